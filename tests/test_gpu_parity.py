"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerance (the FP32 path): relative L2 error <= 1e-4 over the compared
outputs; the maximum per-voxel magnitude error is printed beside it. The
BF16-table variant is held to 1e-2. Inputs are seeded point-target scenes
from the shared generator; echoes come from the oracle's echo model.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2109_02842_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_BF16 = 1e-2


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def report(name, got, ref):
    e = rel(got, ref)
    mx = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print("%s: rel L2 %.3e, max |err| / max |ref| %.3e" % (name, e, mx))
    return e, mx


def check(name, got, ref, tol):
    """Relative L2 error and the largest per-voxel error (relative to the
    largest reference magnitude) both within `tol`; returns the L2 error."""
    e, mx = report(name, got, ref)
    assert e < tol, (name, e)
    assert mx < tol, (name, mx)
    return e


@pytest.fixture(scope="module")
def binding():
    from paper_2109_02842_gb300 import build, binding as b
    build.build()
    b.load()
    assert torch.cuda.is_available()
    return b


def scene_echo(w, seed=0, n_pts=None):
    pts, amp = (w.pts, w.amp) if n_pts is None else (w.pts[:n_pts], w.amp[:n_pts])
    clean = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, pts, amp)
    return wl.add_noise(clean, w.snr_db, wl.rng_for(100, seed)).astype(np.complex64)


def run_gpu(binding, w, echo, **opts):
    plan = binding.Plan.from_workload(w, **opts)
    img = plan.execute(torch.from_numpy(echo).cuda())
    torch.cuda.synchronize()
    return plan, img.cpu().numpy()


def small_multi(n_tx=2, n_rx=16, nx=32, ny=32):
    w = wl.small_mono(seed=0)
    xy, sec, ptx, prx, L = wl.multistatic_array(0.5, 4, 60.0, n_tx, n_rx)
    w.mode, w.elem_xy, w.elem_section, w.pair_tx, w.pair_rx = 1, xy, sec, ptx, prx
    w.grid = dict(w.grid, nx=nx, ny=ny)
    return w


# --- stage parity ------------------------------------------------------------

@pytest.mark.parametrize("n_pad", [64, 67])
def test_zfft_stage_matches_dft(binding, n_pad):
    # the FP32 kernels' path keeps S in its workspace (the tensor-core path
    # feeds the z-FFT's output straight into its range table)
    w = wl.small_mono(seed=0)
    w.n_pad = n_pad                      # 64: Stockham FFT; 67: direct DFT
    echo = scene_echo(w)
    plan, _ = run_gpu(binding, w, echo, block_config=1)
    S = plan.workspace(binding.PL_STAGE_ZFFT).cpu().numpy()
    check("S n_pad=%d" % n_pad, S, oracle.zdft(echo, n_pad), 1e-5)


@pytest.mark.parametrize("bc", [0, 1])
def test_kspace_image_matches_exact_sum(binding, bc):
    w = wl.small_mono(seed=1)
    echo = scene_echo(w, 1)
    plan, _ = run_gpu(binding, w, echo, block_config=bc)
    assert plan.info["block_config"] == (4 if bc == 0 else bc)
    # [parts][n_pad][pixels]: the spectrum is the sum over the channel parts
    G = plan.workspace(binding.PL_STAGE_BACKPROJECT).cpu().numpy()
    G = G.reshape(-1, w.n_pad, w.grid["nx"] * w.grid["ny"]).sum(axis=0)
    S = oracle.zdft(echo, w.n_pad)
    ref = oracle.hybrid_spectral(0, w.tx_xy, w.rx_xy, S, w.dz, w.f_hz, w.pix_xy())
    check("G small mono", G, ref, TOL_FP32)


# --- end-to-end images ----------------------------------------------------------

def image_ref(w, echo, pix=None):
    pix = w.pix_xy() if pix is None else pix
    return oracle.hybrid_exact(w.mode, w.tx_xy, w.rx_xy, echo, w.z_scan, w.f_hz, w.n_pad, pix,
                               w.axis("z"))


@pytest.mark.parametrize("bc", [0, 1, 3])
def test_small_mono_image(binding, bc):
    w = wl.small_mono(seed=0)
    echo = scene_echo(w)
    _, img = run_gpu(binding, w, echo, block_config=bc)
    ref = image_ref(w, echo)
    check("image small mono", img.reshape(w.grid["nz"], -1), ref, TOL_FP32)


@pytest.mark.parametrize("bc", [0, 1])
def test_small_multi_image(binding, bc):
    w = small_multi()
    echo = scene_echo(w)
    _, img = run_gpu(binding, w, echo, block_config=bc)
    ref = image_ref(w, echo)
    check("image small multi", img.reshape(w.grid["nz"], -1), ref, TOL_FP32)


@pytest.mark.parametrize("bc", [0, 1])
def test_gpu_mono_equals_multi_colocated(binding, bc):
    w = wl.small_mono(seed=2)
    echo = scene_echo(w, 2)
    _, g0 = run_gpu(binding, w, echo, block_config=bc)
    w1 = wl.small_mono(seed=2)
    n = w1.elem_xy.shape[0]
    w1.mode, w1.pair_tx, w1.pair_rx = 1, np.arange(n), np.arange(n)
    _, g1 = run_gpu(binding, w1, echo, block_config=bc)
    assert rel(g1, g0) < 2 * TOL_FP32


@pytest.mark.parametrize("bc", [0, 1])
def test_ragged_grid_and_offgrid_z(binding, bc):
    # nx, ny not multiples of the pixel tile; z voxels off the scan grid
    w = wl.small_mono(seed=3)
    w.grid = dict(w.grid, nx=37, ny=23, nz=7, z0=-0.031, dz=0.0093)
    echo = scene_echo(w, 3)
    plan, img = run_gpu(binding, w, echo, block_config=bc)
    assert plan.info["z_transform_fft"] == 0
    check("image ragged", img.reshape(7, -1), image_ref(w, echo), TOL_FP32)


@pytest.mark.parametrize("nz,nx,ny,tile_u", [(7, 37, 23, 0), (50, 32, 32, 0), (50, 32, 32, 16),
                                            (100, 40, 33, 0), (200, 24, 24, 0)])
def test_tensor_core_zidft_stage(binding, nz, nx, ny, tile_u):
    # Eq. (9) at voxel heights off the scan grid on the tensor cores, against
    # the oracle's inverse transform of the plan's own k-space image G: one,
    # two and three blocks of heights, pixel counts that are not multiples of
    # the 128-pixel block, two channel parts (planar) and one (tile_u 16)
    w = wl.small_mono(seed=5)
    zext = w.n_scan * w.dz
    w.grid = dict(w.grid, nx=nx, ny=ny, nz=nz, z0=-0.5 * zext + 0.0013, dz=zext / nz)
    echo = scene_echo(w, 5)
    plan, img = run_gpu(binding, w, echo, block_config=4, tile_u=tile_u)
    assert plan.info["block_config"] == 4 and plan.info["z_transform_fft"] == 0
    G = plan.workspace(binding.PL_STAGE_BACKPROJECT).cpu().numpy()
    G = G.reshape(-1, w.n_pad, nx * ny).sum(axis=0)
    ref = oracle.zidft(G, w.dz, w.z0, w.axis("z"))
    check("tensor-core z-IDFT nz=%d %dx%d tile_u=%d" % (nz, nx, ny, tile_u),
          img.reshape(nz, -1), ref, 3e-5)


def test_scan_grid_ifft_path_with_offset(binding):
    # voxel heights on the scan grid, shifted by 5 scan steps: inverse FFT path
    w = wl.small_mono(seed=4)
    w.grid = dict(w.grid, z0=w.z0 + 5 * w.dz, dz=w.dz, nz=20)
    echo = scene_echo(w, 4)
    plan, img = run_gpu(binding, w, echo)
    assert plan.info["z_transform_fft"] == 1
    check("image ifft path", img.reshape(20, -1), image_ref(w, echo), TOL_FP32)


@pytest.mark.parametrize("bc", [0, 1])
def test_single_frequency_and_single_scan(binding, bc):
    w = wl.small_mono(seed=5)
    w.f_hz = w.f_hz[:1]
    w.n_scan, w.n_pad = 1, 1
    w.grid = dict(w.grid, nz=1, z0=w.z0, dz=w.dz)
    echo = scene_echo(w, 5)
    _, img = run_gpu(binding, w, echo, block_config=bc)
    check("image 1 freq 1 scan", img.reshape(1, -1), image_ref(w, echo), TOL_FP32)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("bc", [0, 1])
def test_bf16_table_variant(binding, bc, precision):
    # precision 1: BF16 table; 2: BF16 table and BF16 spectrum
    w = wl.small_mono(seed=0)
    echo = scene_echo(w)
    plan, img = run_gpu(binding, w, echo, precision=precision, block_config=bc)
    assert plan.info["precision"] == precision
    check("image bf16 precision %d" % precision, img.reshape(w.grid["nz"], -1),
          image_ref(w, echo), TOL_BF16)


@pytest.mark.parametrize("n_pad", [64, 67])
def test_bf16_spectrum_stage(binding, n_pad):
    # precision 2 on the FP32 kernels' path: S stored as bfloat16 (re, im)
    # pairs (64: Stockham FFT; 67: direct DFT), within BF16 rounding of the DFT
    w = wl.small_mono(seed=0)
    w.n_pad = n_pad
    echo = scene_echo(w)
    plan, _ = run_gpu(binding, w, echo, block_config=1, precision=2)
    S = plan.workspace(binding.PL_STAGE_ZFFT).float().cpu().numpy()
    S = S[..., 0] + 1j * S[..., 1]
    check("S bf16 n_pad=%d" % n_pad, S, oracle.zdft(echo, n_pad), 8e-3)


def test_execute_host_matches_device(binding):
    w = wl.small_mono(seed=6)
    echo = scene_echo(w, 6)
    plan, img = run_gpu(binding, w, echo)
    img_h = plan.execute_host(echo)
    assert np.array_equal(img_h, img)


def test_execute_host_stream_matches_device(binding):
    # five different scans through the pipelined host path (two staging pairs
    # and two plans, so each is reused) against one pl_execute each
    import ctypes
    w = wl.small_mono(seed=7)
    plan = binding.Plan.from_workload(w)
    echoes = [torch.from_numpy(scene_echo(w, 70 + i)).pin_memory() for i in range(5)]
    want = [plan.execute(e.cuda()).cpu().numpy() for e in echoes]
    images = [torch.empty(plan.image_shape, dtype=torch.complex64).pin_memory()
              for _ in range(5)]
    plan.execute_host_stream(echoes, images)
    for a, b in zip(images, want):
        assert np.array_equal(a.numpy(), b)
    # one scan (this plan only) and two scans (one each on this plan and on
    # the second plan built from the same inputs), on a fresh plan
    plan2 = binding.Plan.from_workload(w)
    for n in (1, 2):
        out = [torch.empty(plan2.image_shape, dtype=torch.complex64).pin_memory()
               for _ in range(n)]
        plan2.execute_host_stream(echoes[:n], out)
        for a, b in zip(out, want[:n]):
            assert np.array_equal(a.numpy(), b)
    assert plan.execute_host_stream([]) == []
    lib = binding.load()
    null = (ctypes.c_void_p * 1)(None)
    assert lib.pl_execute_host_stream(plan._h, 1, null, null, None) == 1   # PL_ERR_ARG
    assert lib.pl_execute_host_stream(plan._h, -1, None, None, None) == 1


def test_stage_timing(binding):
    w = wl.small_mono(seed=0)
    plan = binding.Plan.from_workload(w)
    e = torch.from_numpy(scene_echo(w)).cuda()
    plan.set_timing(True)
    for _ in range(3):
        plan.execute(e)
    t = plan.stage_times()
    assert all(v[1] == 3 and v[0] > 0 for v in t.values()), t


def test_invalid_inputs_are_rejected(binding):
    w = wl.small_mono(seed=0)
    with pytest.raises(binding.PolylineError) as ei:       # descending frequencies
        binding.Plan(0, w.elem_xy, w.z0, w.dz, w.n_scan, w.f_hz[::-1], w.grid)
    assert ei.value.status == 3
    with pytest.raises(binding.PolylineError) as ei:       # empty grid
        binding.Plan(0, w.elem_xy, w.z0, w.dz, w.n_scan, w.f_hz, dict(w.grid, nx=0))
    assert ei.value.status == 1
    with pytest.raises(binding.PolylineError) as ei:       # pair index out of range
        binding.Plan(1, w.elem_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.grid, pair_tx=[0, 999],
                     pair_rx=[1, 2])
    assert ei.value.status == 2
    with pytest.raises(binding.PolylineError) as ei:       # non-finite position
        xy = w.elem_xy.copy()
        xy[3, 1] = np.nan
        binding.Plan(0, xy, w.z0, w.dz, w.n_scan, w.f_hz, w.grid)
    assert ei.value.status == 5
    with pytest.raises(binding.PolylineError) as ei:       # n_pad < n
        binding.Plan(0, w.elem_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.grid, n_pad=4)
    assert ei.value.status == 1


@pytest.mark.parametrize("bc", [0, 1])
def test_evanescent_bins_are_dropped(binding, bc):
    # dz so coarse that |k_z| > 2k for the outer bins: they contribute nothing,
    # exactly as in the oracle (the k_z = 0 bin always propagates).
    w = wl.small_mono(seed=0)
    w.dz, w.n_scan, w.n_pad = 0.05, 8, 8
    w.z0 = -3.5 * w.dz
    w.f_hz = np.linspace(0.3e9, 0.5e9, 8)
    w.grid = dict(w.grid, nz=8, z0=w.z0, dz=w.dz)
    echo = scene_echo(w, 9)
    _, img = run_gpu(binding, w, echo, block_config=bc)
    check("image evanescent bins", img.reshape(8, -1), image_ref(w, echo), TOL_FP32)


@pytest.mark.parametrize("which", ["small_mono", "full_mono", "multi"])
def test_gpu_echo_synthesis_matches_oracle(binding, which):
    # ranges in FP64, k R as a float-float product reduced modulo 2 pi before
    # the FP32 sin/cos: ~1e-6 rad per phase at k R ~ 1.5e3 rad (full size:
    # the first 48 channels, 64 of the scene's points)
    w = wl.WORKLOADS[which](seed=7)
    tx, rx, pts, amp = w.tx_xy, w.rx_xy, w.pts, w.amp
    if which != "small_mono":
        tx, rx, pts, amp = tx[:48], rx[:48], pts[:64], amp[:64]
    got = binding.synth_echo(tx, rx, w.z0, w.dz, w.n_scan, w.f_hz, pts, amp).cpu().numpy()
    ref = oracle.synth_echo(tx, rx, w.z_scan, w.f_hz, pts, amp)
    check("echo synthesis %s" % which, got, ref, 1e-5)


# --- full sizes, sampled outputs --------------------------------------------------

def sampled_columns(w, n, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(w.grid["nx"] * w.grid["ny"], size=n, replace=False)
    return idx


@pytest.mark.parametrize("which", ["full_mono", "multi"])
def test_full_size_sampled_columns(binding, which):
    # the FP32 kernels at full size (the tensor-core kernel: below)
    w = wl.WORKLOADS[which](seed=0)
    echo = scene_echo(w, 0, n_pts=24)
    _, img = run_gpu(binding, w, echo, block_config=3 if which == "full_mono" else 1)
    idx = sampled_columns(w, 48, 1)
    ref = image_ref(w, echo, w.pix_xy()[idx])
    got = img.reshape(w.grid["nz"], -1)[:, idx]
    check("image %s sampled" % which, got, ref, TOL_FP32)


# --- tensor cores (block_config 4: tcgen05, TMEM accumulators, TMA windows) -------

@pytest.mark.parametrize("case", ["small_mono", "small_multi", "ragged", "npad45", "fine128",
                                  "tile16", "tile48"])
def test_tensor_core_variant_small(binding, case):
    # small_mono, small_multi, ragged, npad45: planar layout (all bins in one
    # block, two channel parts; npad45 pads 45 bins to 48, ragged has voxel
    # heights off the scan grid: the direct inverse DFT adds the two spectra);
    # fine128: a 2 mm grid (one 16-row window step) and 128 bins, one block
    # per SM with three A buffers; tile16, tile48: interleaved blocks
    opts = {}
    if case == "small_multi":
        w = small_multi()
    elif case == "npad45":
        w = wl.small_mono(seed=4)
        w.n_pad = 45
    elif case == "fine128":
        w = wl.small_mono(seed=5)
        w.n_pad = 128
        x0, dx = wl.centred_axis(0.128, 64)
        w.grid = dict(w.grid, x0=x0, dx=dx, nx=64, y0=x0, dy=dx, ny=64, nz=8)
    elif case == "ragged":
        w = wl.small_mono(seed=3)
        w.grid = dict(w.grid, nx=37, ny=23, nz=7, z0=-0.031, dz=0.0093)
    else:
        w = wl.small_mono(seed=0)
        if case != "small_mono":
            opts["tile_u"] = int(case[4:])
    echo = scene_echo(w)
    plan, img = run_gpu(binding, w, echo, block_config=4, **opts)
    i = plan.info
    print("%s: tile_u %d, window rows %d, table rows %d" % (case, i["tile_u"],
                                                          i["slab_rows"], i["table_len"]))
    if "tile_u" not in opts:                 # planar: one block holds every bin
        assert i["tile_u"] >= w.n_pad and i["tile_u"] % 16 == 0
    if case == "fine128":
        assert i["tile_u"] == 128 and i["slab_rows"] == 16
    assert i["nufft_w"] == 6 and i["slab_rows"] in (16, 32)
    ref = image_ref(w, echo)
    check("image tc %s" % case, img.reshape(w.grid["nz"], -1), ref, TOL_FP32)
    # a second execution reports any bounded wait of the first that ran out
    plan.execute(torch.from_numpy(echo).cuda())
    torch.cuda.synchronize()


@pytest.mark.parametrize("taps", [4, 8])
@pytest.mark.parametrize("grid", ["coarse", "fine128"])
def test_tensor_core_other_tap_counts(binding, taps, grid):
    # the 4- and 8-tap kernels (planar layout; fine128: one 16-row window
    # step and 128 bins, two channels per class round). Four taps at
    # sigma 2 resolve the table only to ~1e-3 (the interpolation error of
    # the ES kernel), eight to the FP32 bar
    w = wl.small_mono(seed=6)
    if grid == "fine128":
        w.n_pad = 128
        x0, dx = wl.centred_axis(0.128, 64)
        w.grid = dict(w.grid, x0=x0, dx=dx, nx=64, y0=x0, dy=dx, ny=64, nz=8)
    echo = scene_echo(w, 6)
    plan, img = run_gpu(binding, w, echo, block_config=4, nufft_w=taps)
    assert plan.info["nufft_w"] == taps and plan.info["block_config"] == 4
    check("image tc %d taps %s" % (taps, grid), img.reshape(w.grid["nz"], -1),
          image_ref(w, echo), 2e-3 if taps == 4 else TOL_FP32)


@pytest.mark.parametrize("rows", [0, 12])
@pytest.mark.parametrize("case", ["mono", "multi", "ragged", "npad45", "offgrid", "taps4",
                                  "taps8", "bf16"])
def test_sparse_products_match_dense_and_oracle(binding, case, rows):
    # the 2:4-sparse products (window rows in residue order, K = [Re; Im]
    # rows of the table) against the dense products of the same plan layout
    # and against the oracle, on 2 mm grids (16-row windows): monostatic and
    # multistatic, a ragged pixel grid, 45 bins padded to 48, heights off the
    # scan grid, 4, 6 and 8 taps, BF16-only products; windows of 16 rows, or
    # on request (rows = 12) of 12 rows (residues mod 3) where the taps of
    # every tile span at most 12 rows and w <= 6
    opts = {"sparse_window_rows": rows}
    tol = TOL_FP32
    w = small_multi() if case == "multi" else wl.small_mono(seed=7)
    nx, ny = (37, 23) if case == "ragged" else (64, 64)
    x0, dx = wl.centred_axis(0.128, 64)
    w.grid = dict(w.grid, x0=x0, dx=dx, nx=nx, y0=x0, dy=dx, ny=ny, nz=8)
    if case == "npad45":
        w.n_pad = 45
    elif case == "offgrid":
        w.grid = dict(w.grid, nz=11, z0=-0.047, dz=0.0087)
    elif case.startswith("taps"):
        opts["nufft_w"] = int(case[4:])
        tol = 2e-3 if case == "taps4" else TOL_FP32
    elif case == "bf16":
        opts["precision"] = 1
        tol = TOL_BF16
    echo = scene_echo(w, 7)
    sp, img = run_gpu(binding, w, echo, block_config=4, **opts)
    de, img_d = run_gpu(binding, w, echo, block_config=4, dense_products=True, **opts)
    print("%s: window rows %d, table rows %d, bins %d" % (case, sp.info["slab_rows"],
                                                         sp.info["table_len"], sp.info["tile_u"]))
    assert sp.info["sparse_products"] == 1 and de.info["sparse_products"] == 0
    assert sp.info["slab_rows"] == (12 if rows == 12 and case != "taps8" else 16)
    nz = w.grid["nz"]
    d = float(np.linalg.norm(img - img_d) / np.linalg.norm(img_d))
    print("%s: sparse vs dense rel L2 %.3e" % (case, d))
    assert d < (1e-3 if case == "bf16" else 3e-5)
    check("image tc sparse %s" % case, img.reshape(nz, -1), image_ref(w, echo), tol)


@pytest.mark.parametrize("case", ["tile16", "tile48", "multi", "ragged", "taps8", "bf16",
                                  "fine16", "fine48", "fine_multi", "fine_taps4"])
def test_sparse_products_interleaved_layout(binding, case):
    # the interleaved layout (blocks of tile_u bins, accumulators P and Q).
    # 32-row windows (the 6.25 mm grid of small_mono): one sparse product per
    # real product covers the whole window, rows in residue order mod 4 (K
    # position 8 j + e <-> row j + 4 e). 16-row windows (fine*: a 2 mm grid):
    # the K = 32 operand is the window's hi rows then its lo rows, so
    # [A_hi | A_hi] takes A_hi (b_hi + b_lo) in one sparse product and
    # [A_lo | 0] the A_lo b_hi term
    opts = {"tile_u": 48 if case in ("tile48", "fine48") else 16}
    tol = TOL_FP32
    w = small_multi() if case in ("multi", "fine_multi") else wl.small_mono(seed=8)
    fine = case.startswith("fine")
    if fine:
        x0, dx = wl.centred_axis(0.128, 64)
        w.grid = dict(w.grid, x0=x0, dx=dx, nx=64, y0=x0, dy=dx, ny=64, nz=8)
    if case == "fine_taps4":
        opts["nufft_w"] = 4
        tol = 2e-3
    if case == "ragged":
        # pixel counts off the tile and heights off the scan grid
        w.grid = dict(w.grid, nx=37, ny=23, nz=7, z0=-0.031, dz=0.0093)
    elif case.startswith("taps"):
        opts["nufft_w"] = int(case[4:])
        tol = 2e-3 if case == "taps4" else TOL_FP32
    elif case == "bf16":
        opts["precision"] = 1
        tol = TOL_BF16
    echo = scene_echo(w, 8)
    sp, img = run_gpu(binding, w, echo, block_config=4, **opts)
    de, img_d = run_gpu(binding, w, echo, block_config=4, dense_products=True, **opts)
    print("%s: window rows %d, bins per block %d, table rows %d" % (
        case, sp.info["slab_rows"], sp.info["tile_u"], sp.info["table_len"]))
    assert sp.info["slab_rows"] == (16 if fine else 32) and sp.info["table_layout"] == 2
    assert sp.info["sparse_products"] == 1 and de.info["sparse_products"] == 0
    d = float(np.linalg.norm(img - img_d) / np.linalg.norm(img_d))
    print("%s: sparse vs dense rel L2 %.3e" % (case, d))
    assert d < (1e-3 if case == "bf16" else 3e-5)
    check("image tc sparse interleaved %s" % case, img.reshape(w.grid["nz"], -1),
          image_ref(w, echo), tol)


@pytest.mark.parametrize("case", ["mono", "multi", "ragged", "taps8", "bf16", "np192",
                                  "blocks300", "blocks300_bf16"])
def test_sparse_products_planar_32_row_windows(binding, case):
    # the planar layout with two K steps (the 6.25 mm grid of small_mono:
    # 32-row windows): the K = 32 operands are the window's Re rows and its
    # Im rows (residue order mod 4), so each accumulator takes A S_re and
    # the other A matrix times S_im: Re G += Re A Re b + (-Im A) Im b, Im G
    # += Im A Re b + Re A Im b (twelve sparse products per channel with the
    # hi/lo split). More bins than 192: planar blocks of bins
    opts = {}
    tol = TOL_FP32
    w = small_multi() if case == "multi" else wl.small_mono(seed=11)
    if case == "ragged":
        w.grid = dict(w.grid, nx=37, ny=23, nz=7, z0=-0.031, dz=0.0093)
    elif case == "taps8":
        opts["nufft_w"] = 8             # (4 taps span at most 16 rows here)
    if case.endswith("bf16"):
        opts["precision"] = 1
        tol = TOL_BF16
    if case == "np192":
        w.n_pad = 192
    elif case.startswith("blocks"):
        w.n_pad = int(case[6:9])
    echo = scene_echo(w, 11)
    sp, img = run_gpu(binding, w, echo, block_config=4, **opts)
    de, img_d = run_gpu(binding, w, echo, block_config=4, dense_products=True, **opts)
    i = sp.info
    print("%s: window rows %d, bins per block %d of %d, table rows %d" % (
        case, i["slab_rows"], i["tile_u"], w.n_pad, i["table_len"]))
    assert i["slab_rows"] == 32 and i["table_layout"] == 3 and i["sparse_products"] == 1
    assert de.info["sparse_products"] == 0
    if case.startswith("blocks"):
        assert i["tile_u"] < w.n_pad and i["tile_u"] <= 192
    else:
        assert i["tile_u"] >= w.n_pad
    d = float(np.linalg.norm(img - img_d) / np.linalg.norm(img_d))
    print("%s: sparse vs dense rel L2 %.3e" % (case, d))
    # (BF16 tables: the dense run of 300 bins takes interleaved blocks of
    # other band centres, so the two round different table values; each is
    # held to the BF16 tolerance against the oracle)
    assert d < ((5e-3 if case.startswith("blocks") else 1e-3) if case.endswith("bf16") else 3e-5)
    check("image tc sparse planar 32 rows %s" % case, img.reshape(w.grid["nz"], -1),
          image_ref(w, echo), tol)


@pytest.mark.parametrize("case", ["sparse300", "dense300", "sparse420_bf16", "multi300",
                                  "sparse250"])
def test_planar_layout_in_blocks_of_bins(binding, case):
    # more bins than one planar block holds (N at most 208 next to the A
    # buffers): planar blocks of bins, each with its own band centre, Re and
    # Im columns of the block's bins read at u0 and Im offset + u0
    opts = {}
    tol = TOL_FP32
    w = small_multi() if case == "multi300" else wl.small_mono(seed=10)
    x0, dx = wl.centred_axis(0.128, 64)
    w.grid = dict(w.grid, x0=x0, dx=dx, nx=64, y0=x0, dy=dx, ny=64, nz=8)
    w.n_pad = 420 if "420" in case else (250 if "250" in case else 300)
    if case.startswith("dense"):
        opts["dense_products"] = True
    if case.endswith("bf16"):
        opts["precision"] = 1
        tol = TOL_BF16
    echo = scene_echo(w, 10)
    plan, img = run_gpu(binding, w, echo, block_config=4, **opts)
    i = plan.info
    print("%s: bins per block %d of %d, window rows %d, sparse %d" % (
        case, i["tile_u"], w.n_pad, i["slab_rows"], i["sparse_products"]))
    assert i["table_layout"] == 3 and i["tile_u"] < w.n_pad and i["tile_u"] <= 208
    assert i["sparse_products"] == (0 if case.startswith("dense") else 1)
    check("image tc planar blocks %s" % case, img.reshape(w.grid["nz"], -1), image_ref(w, echo),
          tol)


@pytest.mark.parametrize("case", ["one_channel", "three_channels", "one_pixel", "one_frequency",
                                  "seven_bins"])
def test_sparse_products_degenerate_sizes(binding, case):
    # the sparse kernel at the edges of its sizes (2 mm grid, 16-row
    # windows): fewer channels than channel classes x warp sets (classes and
    # sets without a round), a single pixel (one tile, 127 idle lanes), a
    # single frequency (a band of one wavenumber), seven k_z bins (N = 16)
    w = wl.small_mono(seed=9)
    x0, dx = wl.centred_axis(0.128, 64)
    w.grid = dict(w.grid, x0=x0, dx=dx, nx=64, y0=x0, dy=dx, ny=64, nz=8)
    if case == "one_channel":
        idx = np.array([21])
    elif case == "three_channels":
        idx = np.array([3, 30, 57])
    else:
        idx = None
    if idx is not None:
        w.elem_xy, w.elem_section = w.elem_xy[idx], w.elem_section[idx]
    if case == "one_pixel":
        w.grid = dict(w.grid, x0=0.013, nx=1, y0=-0.021, ny=1, nz=3)
    elif case == "one_frequency":
        w.f_hz = w.f_hz[7:8]
    elif case == "seven_bins":
        w.n_scan, w.n_pad = 7, 7
        w.grid = dict(w.grid, nz=5, z0=w.z0, dz=w.dz)
    echo = scene_echo(w, 9)
    plan, img = run_gpu(binding, w, echo, block_config=4)
    assert plan.info["sparse_products"] == 1, plan.info
    check("image tc sparse %s" % case, img.reshape(w.grid["nz"], -1), image_ref(w, echo),
          TOL_FP32)


@pytest.mark.parametrize("rows", [0, 12])
@pytest.mark.parametrize("which", ["full_mono", "multi"])
def test_sparse_products_full_size(binding, which, rows):
    # full_mono: every tile's taps span at most 12 rows, so 12-row windows
    # apply on request; multi (spans up to 14 rows) keeps 16
    w = wl.WORKLOADS[which](seed=0)
    echo = scene_echo(w, 0, n_pts=24)
    sp, img = run_gpu(binding, w, echo, block_config=4, sparse_window_rows=rows)
    assert sp.info["slab_rows"] == (12 if which == "full_mono" and rows == 12 else 16)
    de, img_d = run_gpu(binding, w, echo, block_config=4, dense_products=True)
    assert sp.info["sparse_products"] == 1
    d = float(np.linalg.norm(img - img_d) / np.linalg.norm(img_d))
    print("%s: sparse vs dense rel L2 %.3e" % (which, d))
    assert d < 3e-5
    idx = sampled_columns(w, 48, 2)
    ref = image_ref(w, echo, w.pix_xy()[idx])
    check("image tc sparse %s sampled" % which, img.reshape(w.grid["nz"], -1)[:, idx], ref,
          TOL_FP32)


def test_tensor_core_bf16_only_products(binding):
    w = wl.small_mono(seed=2)
    echo = scene_echo(w, 2)
    _, img = run_gpu(binding, w, echo, block_config=4, precision=1)
    ref = image_ref(w, echo)
    check("image tc bf16", img.reshape(w.grid["nz"], -1), ref, TOL_BF16)


@pytest.mark.parametrize("which", ["full_mono", "multi"])
def test_tensor_core_variant_full_size_sampled(binding, which):
    w = wl.WORKLOADS[which](seed=0)
    echo = scene_echo(w, 0, n_pts=24)
    plan, img = run_gpu(binding, w, echo, block_config=4)
    print("%s: window rows %d, table rows %d, back-projection launches %d"
          % (which, plan.info["slab_rows"], plan.info["table_len"], plan.info["bp_launches"]))
    if which == "full_mono":
        # 1024 blocks on 152 SMs: the full waves, then the last wave beside the
        # z-IFFT of the pixels they finished (the sampled columns span both)
        assert plan.info["bp_launches"] == 2
        assert plan.info["launches_per_execute"] == 7
    idx = sampled_columns(w, 48, 1)
    ref = image_ref(w, echo, w.pix_xy()[idx])
    got = img.reshape(w.grid["nz"], -1)[:, idx]
    check("image tc %s sampled" % which, got, ref, TOL_FP32)


# --- configurations at the edges of the workloads --------------------------------

@pytest.mark.parametrize("n_f,exact", [(96, 1), (160, 0)])
def test_tensor_core_many_frequencies(binding, n_f, exact):
    # 96 frequencies: the exact-sum table over two 64-frequency atoms; 160:
    # the tensor-core back-projection reads a table built by the type-1 NUFFT
    # (spread, fine FFT, deconvolution)
    w = wl.small_mono(seed=8)
    w.f_hz = wl.uniform_freqs(28e9, 33e9, n_f)
    echo = scene_echo(w, 8)
    plan, img = run_gpu(binding, w, echo)
    assert plan.info["block_config"] == 4 and plan.info["table_exact"] == exact
    check("image tc %d freqs" % n_f, img.reshape(w.grid["nz"], -1), image_ref(w, echo), TOL_FP32)


def test_uneven_scene_at_the_edge_of_the_batch_ranges(binding):
    # the largest scene the batched workload draws: 12 sections x 48 elements
    # (576 channels), 256 scans (N_p 512), 96 frequencies, a 160^3 image;
    # 500 points, 32 sampled columns x all 160 heights
    w = wl.uneven_scene(wl.rng_for(4, 999), 12, 48, 256, 96, 160, 500, "uneven-edge")
    assert (w.n_chan, w.n_scan, w.n_pad, w.n_f, w.grid["nx"]) == (576, 256, 512, 96, 160)
    echo = scene_echo(w, 9, n_pts=64)
    plan, img = run_gpu(binding, w, echo)
    print("edge scene: block_config %d, tile_u %d, window rows %d, table rows %d, exact %d"
          % (plan.info["block_config"], plan.info["tile_u"], plan.info["slab_rows"],
             plan.info["table_len"], plan.info["table_exact"]))
    idx = sampled_columns(w, 32, 3)
    ref = image_ref(w, echo, w.pix_xy()[idx])
    got = img.reshape(w.grid["nz"], -1)[:, idx]
    check("image edge scene sampled", got, ref, TOL_FP32)


def test_coarse_batch_scene_planar_32_row_windows(binding):
    # one of the batched workload's coarse-grid scenes at its own size (135
    # channels, 138 scans, N_p 288, 75 frequencies: two atoms of the exact-sum
    # table, a 79^3 image at 5 mm): planar sparse products with 32-row
    # windows in two blocks of 144 bins, against the dense products and the
    # oracle on 32 sampled columns x all 79 heights
    w = wl.batch_scene(63)
    assert (w.n_chan, w.n_pad, w.n_f, w.grid["nx"]) == (135, 288, 75, 79)
    echo = scene_echo(w, 13, n_pts=48)
    sp, img = run_gpu(binding, w, echo)
    de, img_d = run_gpu(binding, w, echo, dense_products=True)
    i = sp.info
    print("coarse batch scene: bins per block %d, window rows %d, table rows %d, exact %d"
          % (i["tile_u"], i["slab_rows"], i["table_len"], i["table_exact"]))
    assert i["block_config"] == 4 and i["sparse_products"] == 1 and i["table_layout"] == 3
    assert i["slab_rows"] == 32 and i["tile_u"] == 144 and i["table_exact"] == 1
    d = float(np.linalg.norm(img - img_d) / np.linalg.norm(img_d))
    print("coarse batch scene: sparse vs dense rel L2 %.3e" % d)
    assert d < 3e-5
    idx = sampled_columns(w, 32, 4)
    ref = image_ref(w, echo, w.pix_xy()[idx])
    check("image coarse batch scene sampled", img.reshape(w.grid["nz"], -1)[:, idx], ref,
          TOL_FP32)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("bc", [4, 1])
def test_full_size_multistatic_bf16_variants(binding, bc, precision):
    # the BF16 variants at the full multistatic size (1024 pairs, 128 scans,
    # 64 frequencies, 192 x 192 x 128): precision 1, BF16-only products on
    # the tensor cores (bc 4) or a BF16 table with FP32 arithmetic (bc 1);
    # precision 2, the spectrum in BF16 as well
    w = wl.multi(seed=0)
    echo = scene_echo(w, 0, n_pts=24)
    plan, img = run_gpu(binding, w, echo, block_config=bc, precision=precision)
    assert plan.info["precision"] == precision and plan.info["block_config"] == bc
    idx = sampled_columns(w, 48, 1)
    ref = image_ref(w, echo, w.pix_xy()[idx])
    got = img.reshape(w.grid["nz"], -1)[:, idx]
    check("image multi precision %d bc %d sampled" % (precision, bc), got, ref, TOL_BF16)


@pytest.mark.parametrize("mode,cross", [(0, False), (1, False), (1, True)])
def test_paper_table1_geometry(binding, mode, cross):
    # Table I: R0 = 1.0 m, 3 sections, 51 frequencies over 30-35 GHz, dz 0.5 cm;
    # mono 40 elements per section, multi 4 Tx at the joints and ends with 20 Rx
    # per section (pairs within a section; cross: every Tx with every section's
    # Rx); 64 scans and a 64^3 grid over 0.2 m (the paper states neither);
    # 128 sampled columns x all heights
    w = wl.paper_table1(mode, seed=1, cross_section=cross)
    assert w.n_chan == (120 if mode == 0 else (240 if cross else 120))
    echo = scene_echo(w, 1)
    plan, img = run_gpu(binding, w, echo)
    idx = sampled_columns(w, 128, 4)
    ref = image_ref(w, echo, w.pix_xy()[idx])
    got = img.reshape(w.grid["nz"], -1)[:, idx]
    check("image %s sampled" % w.name, got, ref, TOL_FP32)
