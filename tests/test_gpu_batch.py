"""Batched uneven scans (one persistent launch in a CUDA graph), through the
C ABI: each scene's image equals the single-scan path's and the FP64 oracle's;
the autotuner and the per-scene fallback give the same images; a wait that
cannot be satisfied ends with PL_ERR_TIMEOUT and leaves the device usable."""
import numpy as np
import pytest

import oracle
from paper_2109_02842_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


@pytest.fixture(scope="module")
def binding():
    from paper_2109_02842_gb300 import build, binding as b
    build.build()
    b.load()
    assert torch.cuda.is_available()
    return b


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def uneven_scenes():
    """Five small scenes of different array, scan, band and grid sizes."""
    out = []
    w = wl.small_mono(seed=0)
    out.append(w)
    w = wl.small_mono(seed=1)
    w.grid = dict(w.grid, nx=40, ny=24, nz=20)
    w.f_hz = w.f_hz[:12]
    out.append(w)
    w = wl.small_mono(seed=2)
    xy, sec, ptx, prx, _ = wl.multistatic_array(0.5, 4, 60.0, 2, 16)
    w.mode, w.elem_xy, w.elem_section, w.pair_tx, w.pair_rx = 1, xy, sec, ptx, prx
    out.append(w)
    w = wl.small_mono(seed=3)
    xy, sec, L = wl.monostatic_array(0.55, 5, 70.0, 20)
    w.elem_xy, w.elem_section, w.chord_len, w.n_sections = xy, sec, L, 5
    w.n_scan, w.n_pad = 48, 96
    w.z0 = -(w.n_scan - 1) / 2 * w.dz
    w.f_hz = np.linspace(27e9, 33e9, 24)
    w.grid = dict(w.grid, nx=48, ny=48, nz=24, z0=-0.1, dz=0.2 / 24)
    out.append(w)
    w = wl.small_mono(seed=4)
    w.grid = dict(w.grid, nx=17, ny=33, nz=9)
    out.append(w)
    # more than 64 frequencies: the tensor-core path sums this scene's table
    # over two 64-frequency atoms; more than 128: it builds it with the NUFFT
    for seed, n_f in ((5, 80), (6, 136)):
        w = wl.small_mono(seed=seed)
        w.f_hz = np.linspace(26e9, 34e9, n_f)
        w.grid = dict(w.grid, nz=16)
        out.append(w)
    return out


def echoes(scenes):
    out = []
    for i, w in enumerate(scenes):
        clean = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, w.pts, w.amp)
        out.append(wl.add_noise(clean, w.snr_db, wl.rng_for(200, i)).astype(np.complex64))
    return out


@pytest.fixture(scope="module")
def data():
    sc = uneven_scenes()
    return sc, echoes(sc)


def run_batch(binding, scenes, echo_np, **kw):
    b = binding.Batch(scenes, **kw)
    imgs = b.execute([torch.from_numpy(e).cuda() for e in echo_np])
    torch.cuda.synchronize()
    return b, [im.cpu().numpy() for im in imgs]


@pytest.mark.parametrize("kind", ["tensor_core", "tensor_core_per_scene", "persistent"])
def test_batch_matches_single_scan_path_and_oracle(binding, data, kind):
    # tensor_core: the scenes' range tables on parallel streams, then ONE
    # persistent tensor-core back-projection over every scene's blocks;
    # tensor_core_per_scene (the default): each scene's own tensor-core
    # launches on parallel streams; persistent: the FP32 kernels in one
    # persistent launch over all scenes (range tables and back-projections)
    scenes, echo_np = data
    kw = {"tensor_core": dict(tc_launch=1), "tensor_core_per_scene": {},
          "persistent": dict(tile_u=16, block_config=1)}[kind]
    b, imgs = run_batch(binding, scenes, echo_np, **kw)
    info = b.info
    assert info["persistent"] == (0 if kind == "tensor_core_per_scene" else 1)
    assert info["n_scenes"] == len(scenes)
    if kind == "tensor_core":
        assert info["block_config"] == 4 and info["persistent_blocks"] > 0
    for i, w in enumerate(scenes):
        if kind == "tensor_core":
            plan = binding.Plan.from_workload(w, block_config=4, one_block_per_sm=1)
        elif kind == "tensor_core_per_scene":
            plan = binding.Plan.from_workload(w, block_config=4)
        else:
            plan = binding.Plan.from_workload(w, tile_u=info["tile_u"],
                                              block_config=info["block_config"])
        single = plan.execute(torch.from_numpy(echo_np[i]).cuda()).cpu().numpy()
        if kind != "persistent":
            # the batch runs each scene's blocks (one persistent launch for
            # all scenes, or one launch per scene); a plan's own execution
            # may split its back-projection into its full waves and its last
            # wave with part of the z-IFFT beside it: the same arithmetic per
            # output, so the images agree bit for bit
            assert np.array_equal(imgs[i], single), i
        else:
            assert rel(imgs[i], single) < 1e-6, i
    for i in (0, 2, 3, 5, 6):
        w = scenes[i]
        ref = oracle.hybrid_exact(w.mode, w.tx_xy, w.rx_xy, echo_np[i], w.z_scan, w.f_hz,
                                  w.n_pad, w.pix_xy(), w.axis("z"))
        got = imgs[i].reshape(w.grid["nz"], -1)
        e, mx = rel(got, ref), max_err(got, ref)
        print("batch scene %d: rel L2 %.3e, max |err| / max |ref| %.3e" % (i, e, mx))
        assert e < TOL_FP32 and mx < TOL_FP32


def test_batch_replays_with_new_buffers(binding, data):
    scenes, echo_np = data
    b = binding.Batch(scenes)
    first = [im.cpu().numpy() for im in b.execute([torch.from_numpy(e).cuda() for e in echo_np])]
    again = [im.cpu().numpy() for im in b.execute([torch.from_numpy(e).cuda() for e in echo_np])]
    for x, y in zip(first, again):
        assert np.array_equal(x, y)


def test_autotuned_batch(binding, data):
    scenes, echo_np = data
    b, imgs = run_batch(binding, scenes, echo_np, autotune=True)
    info = b.info
    assert info["autotuned"] == 1 and info["tune_best_ms"] > 0
    assert info["block_config"] in (1, 3, 4)
    if info["block_config"] != 4:
        assert info["tile_u"] in (8, 16, 20)
    w = scenes[0]
    ref = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, echo_np[0], w.z_scan, w.f_hz, w.n_pad,
                              w.pix_xy(), w.axis("z"))
    assert rel(imgs[0].reshape(w.grid["nz"], -1), ref) < TOL_FP32
    # the choice is cached: a second batch of the same shapes does not re-time
    b2 = binding.Batch(scenes, autotune=True)
    assert b2.info["tile_u"] == info["tile_u"] and b2.info["tune_best_ms"] == 0


def test_per_scene_fallback_when_not_persistent(binding, data):
    scenes, echo_np = data
    b, imgs = run_batch(binding, scenes[:2], echo_np[:2], nufft_w=8)
    assert b.info["persistent"] == 0
    w = scenes[1]
    ref = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, echo_np[1], w.z_scan, w.f_hz, w.n_pad,
                              w.pix_xy(), w.axis("z"))
    assert rel(imgs[1].reshape(w.grid["nz"], -1), ref) < TOL_FP32


def test_unsatisfiable_wait_times_out_and_device_stays_usable(binding, data):
    scenes, echo_np = data
    b = binding.Batch(scenes, tile_u=16, block_config=1, debug_unsatisfiable=1,
                      wait_timeout_ms=20.0)
    with pytest.raises(binding.PolylineError) as ei:
        b.execute([torch.from_numpy(e).cuda() for e in echo_np])
    assert ei.value.status == 8
    # the context is still good: a normal batch runs and matches
    _, imgs = run_batch(binding, scenes[:1], echo_np[:1])
    w = scenes[0]
    ref = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, echo_np[0], w.z_scan, w.f_hz, w.n_pad,
                              w.pix_xy(), w.axis("z"))
    assert rel(imgs[0].reshape(w.grid["nz"], -1), ref) < TOL_FP32


def test_persistent_tensor_core_wait_times_out(binding, data):
    # the persistent tensor-core back-projection with a wait nothing completes
    # (the test hook of pl_options) and a 2 ms budget: PL_ERR_TIMEOUT, the
    # blocks stop taking items, and the device stays usable
    scenes, echo_np = data
    b = binding.Batch(scenes[:3], tc_launch=1, tc_debug_unsatisfiable=1, tc_wait_timeout_us=2000)
    assert b.info["persistent"] == 1 and b.info["block_config"] == 4
    with pytest.raises(binding.PolylineError) as ei:
        b.execute([torch.from_numpy(e).cuda() for e in echo_np[:3]])
    assert ei.value.status == 8
    _, imgs = run_batch(binding, scenes[:1], echo_np[:1])
    w = scenes[0]
    ref = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, echo_np[0], w.z_scan, w.f_hz, w.n_pad,
                              w.pix_xy(), w.axis("z"))
    assert rel(imgs[0].reshape(w.grid["nz"], -1), ref) < TOL_FP32
