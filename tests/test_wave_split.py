"""Host arithmetic of the tensor-core back-projection's split into its full
waves and its last partial wave (csrc/wave_split.h), compiled with the host
C++ compiler and checked against a brute-force walk over the block order:
the pixels handed to the early inverse transform are exactly the whole rows
of tiles whose every channel part ran in the full waves, and no block of the
last wave writes any of them."""
import itertools
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER_DIR = os.path.join(HERE, "..", "paper_2109_02842_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "wave_split.h"
int main() {
    int total, wave, nsplit, nbx, tile_y, nx, ny;
    while (std::scanf("%d %d %d %d %d %d %d", &total, &wave, &nsplit, &nbx, &tile_y, &nx, &ny) == 7) {
        const WaveSplit s = bp_wave_split(total, wave, nsplit, nbx, tile_y, nx, ny);
        std::printf("%d %d\n", s.full, s.cols);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def split_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("wave_split")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", HEADER_DIR, str(src), "-o", str(exe)],
                   check=True)
    return exe


def run_cases(exe, cases):
    inp = "\n".join(" ".join(str(v) for v in c) for c in cases) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True)
    return [tuple(int(v) for v in line.split()) for line in out.stdout.strip().splitlines()]


def brute_force(total, wave, nsplit, tile_x, tile_y, nx, ny):
    """Walk the blocks in launch order (tile x fastest, then tile y, then the
    channel part) and return (full, cols) as the split should be, plus the
    blocks of the last wave."""
    nbx = -(-nx // tile_x)
    nby = -(-ny // tile_y)
    assert total == nbx * nby * nsplit
    full = total // wave * wave
    parts_done = {}
    for b in range(full):
        t = b % (nbx * nby)
        parts_done[t] = parts_done.get(t, 0) + 1
    rows_of_tiles = 0
    while rows_of_tiles < nby and all(parts_done.get(rows_of_tiles * nbx + x, 0) == nsplit
                                      for x in range(nbx)):
        rows_of_tiles += 1
    rows = min(ny, rows_of_tiles * tile_y)
    if not (0 < full < total and rows > 0):
        return (0, 0), []
    return (full, rows * nx), list(range(full, total))


def pixels_of_block(b, nsplit, tile_x, tile_y, nx, ny):
    nbx = -(-nx // tile_x)
    nby = -(-ny // tile_y)
    t = b % (nbx * nby)
    bx, by = t % nbx, t // nbx
    for py in range(by * tile_y, min(ny, by * tile_y + tile_y)):
        for px in range(bx * tile_x, min(nx, bx * tile_x + tile_x)):
            yield py * nx + px


def case_args(wave, nsplit, tile_x, tile_y, nx, ny):
    nbx = -(-nx // tile_x)
    nby = -(-ny // tile_y)
    return (nbx * nby * nsplit, wave, nsplit, nbx, tile_y, nx, ny)


def test_full_size_split_is_six_waves_and_200_pixel_rows(split_exe):
    # 256 x 256 pixels in 16 x 8 tiles, two channel parts: 1024 blocks on 152
    # SMs (one block each) -> 912 blocks in six full waves; tiles 0..399 have
    # both parts in them, i.e. 25 rows of tiles = pixel rows 0..199
    (got,) = run_cases(split_exe, [case_args(152, 2, 16, 8, 256, 256)])
    assert got == (912, 200 * 256)


def test_no_split_without_a_partial_wave_or_a_finished_row(split_exe):
    cases = [
        case_args(152, 2, 16, 8, 64, 64),     # 64 blocks: fewer than one wave
        case_args(128, 2, 16, 8, 128, 128),   # 256 blocks = two whole waves
        case_args(152, 2, 16, 8, 16 * 100, 8),  # 200 blocks, one row of 100 tiles: part 1 of
                                              # the row's first tiles is in the last wave
    ]
    assert run_cases(split_exe, cases) == [(0, 0)] * len(cases)


def test_matches_brute_force_and_last_wave_is_disjoint(split_exe):
    cases, params = [], []
    for (nx, ny), nsplit, wave in itertools.product(
            [(256, 256), (128, 128), (17, 33), (40, 24), (48, 48), (192, 192), (100, 7)],
            [1, 2, 3], [152, 304, 100, 37]):
        args = case_args(wave, nsplit, 16, 8, nx, ny)
        cases.append(args)
        params.append((wave, nsplit, nx, ny))
    got = run_cases(split_exe, cases)
    n_split = 0
    for args, (wave, nsplit, nx, ny), g in zip(cases, params, got):
        want, last = brute_force(args[0], wave, nsplit, 16, 8, nx, ny)
        assert g == want, (wave, nsplit, nx, ny)
        if g[0]:
            n_split += 1
            cols = g[1]
            for b in last:
                assert min(pixels_of_block(b, nsplit, 16, 8, nx, ny)) >= cols
    assert n_split >= 10          # the grid of cases exercises the split
