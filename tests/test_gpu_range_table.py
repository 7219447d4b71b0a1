"""Stage parity of the range table (step (8a) / (19a)) against the oracle's
exact range profile, through the C ABI.

The table b (workspace PL_STAGE_RANGE_TABLE) holds the coefficients of a
type-1 NUFFT on the uniform range grid l_i = l0 + i h (pl_info describes the
layout, the ES kernel and the band centres). Interpolated with the ES kernel,
sum_i ES((l - l_i) / h) b_i(u), it must reproduce the oracle's
q_{c,u}(l) = sum_m S k_m e^{j (kappa - kappa_0) l} up to the change of
reference from kappa_0 = kappa(k_0, k_z) to the band centre kappa_c:
    sum_i ES(...) b_i(u) = q_{c,u}(l) e^{j (kappa_0 - kappa_c) l}.
Every table format is covered: exact sums on the tensor cores (planar and
interleaved; one and two 64-frequency atoms), the NUFFT-built tensor-core
table (more than 128 frequencies),
the FP32 kernels' float32 and bfloat16 tables, monostatic and multistatic.
The spectrum S fed to the oracle is its own FP64 z-DFT of the same echo.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2109_02842_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C0 = 299792458.0


@pytest.fixture(scope="module")
def binding():
    from paper_2109_02842_gb300 import build, binding as b
    build.build()
    b.load()
    assert torch.cuda.is_available()
    return b


def table_values(plan, binding):
    """The table as complex128 [C][L][n_pad] (b_i(u)), whatever its layout;
    the tensor-core tables as hi + lo (BF16-only products: hi, what the
    back-projection reads)."""
    i = plan.info
    C, L, Np = i["n_chan"], i["table_len"], i["n_pad"]
    raw = plan.workspace(binding.PL_STAGE_RANGE_TABLE).float().cpu().numpy()
    lay = i["table_layout"]
    if lay in (0, 1):                                  # [C][L][np2][{re_u, re_u+1, im_u, im_u+1}]
        re = raw[..., 0:2].reshape(C, L, -1)[..., :Np]
        im = raw[..., 2:4].reshape(C, L, -1)[..., :Np]
        return re.astype(np.float64) + 1j * im
    cols = i["table_cols"]
    assert raw.shape == (C, 2, L, cols)
    v = raw[:, 0].astype(np.float64)
    if i["precision"] == 0:
        v = v + raw[:, 1]
    if lay == 3:                                       # planar: Re of the bins | Im of the bins
        return v[..., :Np] + 1j * v[..., cols // 2: cols // 2 + Np]
    return v[..., 0:2 * Np:2] + 1j * v[..., 1:2 * Np:2]


def kappa(mode, k, kz):
    q = 4 * k * k - kz * kz if mode == 0 else k * k - kz * kz / 4
    return np.where(q > 0, np.sqrt(np.maximum(q, 0.0)), np.nan)


def band_centres(mode, f_hz, kz, group):
    """kappa_c of every bin: the centre of the live kappa band of its group."""
    k = 2 * np.pi * np.asarray(f_hz) / C0
    Np = kz.size
    kc = np.zeros(Np)
    for g0 in range(0, Np, group):
        kap = kappa(mode, k[None, :], kz[g0:g0 + group, None])
        kap = kap[np.isfinite(kap)]
        kc[g0:g0 + group] = 0.5 * (kap.min() + kap.max()) if kap.size else 0.0
    return kc


def es(t, w, beta):
    z = 2.0 * t / w
    q = 1.0 - z * z
    return np.where(q > 0, np.exp(beta * (np.sqrt(np.maximum(q, 0.0)) - 1.0)), 0.0)


def check_table(binding, w, echo, tol, n_ch=6, n_l=24, seed=0, **opts):
    plan = binding.Plan.from_workload(w, **opts)
    plan.execute(torch.from_numpy(echo).cuda())
    torch.cuda.synchronize()
    i = plan.info
    b = table_values(plan, binding)
    L, h, l0, W, beta = i["table_len"], i["table_h"], i["table_l0"], i["nufft_w"], i["es_beta"]
    S = oracle.zdft(echo.astype(np.complex128), w.n_pad)
    kz = oracle.kz_bins(w.n_pad, w.dz)
    k0 = 2 * np.pi * w.f_hz[0] / C0
    kc = band_centres(w.mode, w.f_hz, kz, i["band_group"])
    rng = np.random.default_rng(seed)
    chans = rng.choice(i["n_chan"], size=min(n_ch, i["n_chan"]), replace=False)
    bins = sorted(set([0, 1, w.n_pad // 2, w.n_pad - 1] +
                      list(rng.choice(w.n_pad, size=6, replace=False))))
    # ranges whose whole W-tap window lies inside the table
    lo, hi = l0 + (0.5 * W + 1) * h, l0 + (L - 0.5 * W - 2) * h
    got, ref = [], []
    for c in chans:
        for u in bins:
            k0u = kappa(w.mode, k0, kz[u])
            if not np.isfinite(k0u):
                continue
            l = rng.uniform(lo, hi, n_l)
            q = oracle.range_profile(w.mode, S, w.dz, w.f_hz, int(c), int(u), l)
            ref.append(q * np.exp(1j * (k0u - kc[u]) * l))
            pos = (l - l0) / h
            first = np.ceil(pos - 0.5 * W).astype(int)
            acc = np.zeros(l.size, np.complex128)
            for t in range(W):
                rows = first + t
                acc += es(pos - rows, W, beta) * b[c, rows, u]
            got.append(acc)
    got, ref = np.concatenate(got), np.concatenate(ref)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    mx = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print("table layout %d exact %d precision %d: rel L2 %.3e, max |err| / max |ref| %.3e"
          % (i["table_layout"], i["table_exact"], i["precision"], err, mx))
    assert err < tol and mx < tol
    return i


def small_multi():
    w = wl.small_mono(seed=0)
    xy, sec, ptx, prx, L = wl.multistatic_array(0.5, 4, 60.0, 2, 16)
    w.mode, w.elem_xy, w.elem_section, w.pair_tx, w.pair_rx = 1, xy, sec, ptx, prx
    return w


def echo_of(w, seed):
    clean = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, w.pts, w.amp)
    return wl.add_noise(clean, w.snr_db, wl.rng_for(120, seed)).astype(np.complex64)


CASES = {
    # name: (workload maker, options, expected (layout, exact), tolerance)
    "tc_exact_planar": (lambda: wl.small_mono(seed=1), dict(block_config=4), (3, 1), 1e-4),
    "tc_exact_interleaved": (lambda: wl.small_mono(seed=1), dict(block_config=4, tile_u=16),
                             (2, 1), 1e-4),
    "tc_exact_multi": (small_multi, dict(block_config=4), (3, 1), 1e-4),
    "tc_bf16_products": (lambda: wl.small_mono(seed=1), dict(block_config=4, precision=1),
                         (3, 1), 1e-2),
    "fp32_table": (lambda: wl.small_mono(seed=1), dict(block_config=1), (0, 0), 1e-4),
    "fp32_table_multi": (small_multi, dict(block_config=1), (0, 0), 1e-4),
    "bf16_table": (lambda: wl.small_mono(seed=1), dict(block_config=1, precision=1), (1, 0),
                   1e-2),
    "tc_bf16_spectrum": (lambda: wl.small_mono(seed=1), dict(block_config=4, precision=2),
                         (3, 1), 1e-2),
    "bf16_table_spectrum": (lambda: wl.small_mono(seed=1), dict(block_config=1, precision=2),
                            (1, 0), 1e-2),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_range_table_matches_oracle_profile(binding, case):
    make, opts, (layout, exact), tol = CASES[case]
    w = make()
    i = check_table(binding, w, echo_of(w, 1), tol, **opts)
    assert (i["table_layout"], i["table_exact"]) == (layout, exact)


@pytest.mark.parametrize("mode,precision", [(0, 0), (1, 0), (0, 2)])
def test_two_atom_exact_table(binding, mode, precision):
    # 65 to 128 frequencies: the exact sums over two 64-frequency atoms
    # accumulated in tensor memory (precision 2: the spectrum's BF16 part)
    w = wl.small_mono(seed=2) if mode == 0 else small_multi()
    w.f_hz = wl.uniform_freqs(28e9, 33e9, 96)
    i = check_table(binding, w, echo_of(w, 2), 1e-4 if precision == 0 else 1e-2,
                    block_config=4, precision=precision)
    assert i["table_exact"] == 1 and i["table_layout"] in (2, 3) and i["n_f"] == 96


@pytest.mark.parametrize("mode,precision", [(0, 0), (1, 0), (0, 2)])
def test_nufft_built_tensor_core_table_above_128_frequencies(binding, mode, precision):
    # more than 128 frequencies: the tensor-core back-projection's table comes
    # from the type-1 NUFFT (spread, FFT, deconvolution), not the exact sums
    # (precision 2: from a BF16 spectrum)
    w = wl.small_mono(seed=2) if mode == 0 else small_multi()
    w.f_hz = wl.uniform_freqs(28e9, 33e9, 160)
    i = check_table(binding, w, echo_of(w, 2), 1e-4 if precision == 0 else 1e-2,
                    block_config=4, precision=precision)
    assert i["table_exact"] == 0 and i["table_layout"] in (2, 3) and i["n_f"] == 160
