"""The C-ABI library builds, loads and exports every entry point that
include/polyline.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polyline.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pl_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2109_02842_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pl_plan_create", "pl_execute", "pl_execute_host", "pl_plan_destroy",
                 "pl_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert set(declared_functions()) <= exported


def test_binding_knows_every_symbol(lib_path):
    from paper_2109_02842_gb300 import binding
    assert set(binding.EXPORTED) == set(declared_functions())


def test_status_strings_without_gpu(lib_path):
    from paper_2109_02842_gb300 import binding
    lib = binding.load()
    assert lib.pl_version() >= 100
    assert binding.status_string(0) == "ok"
    assert "evanescent" in binding.status_string(4)


def test_binding_refuses_missing_library(tmp_path):
    # no silent fallback: a missing library is an error
    from paper_2109_02842_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2109_02842_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f


STRUCTS = {"PlGeometry": "pl_geometry", "PlScan": "pl_scan", "PlFreqs": "pl_freqs",
           "PlGrid": "pl_grid", "PlOptions": "pl_options", "PlInfo": "pl_info",
           "PlBatchOptions": "pl_batch_options", "PlBatchInfo": "pl_batch_info",
           "PlDesignInfo": "pl_design_info"}


def test_binding_structs_match_the_header(tmp_path):
    # a C program compiled against the header prints sizeof and offsetof of
    # every field the ctypes mirror declares; both must agree byte for byte
    from paper_2109_02842_gb300 import binding
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "polyline.h"',
             "int main(void) {"]
    expect = []
    for py, c in STRUCTS.items():
        cls = getattr(binding, py)
        lines.append('printf("%%zu\\n", sizeof(%s));' % c)
        expect.append(ctypes.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (c, name))
            expect.append(getattr(cls, name).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == expect
