"""The comparison algorithms of Sec. III on the GPU (pl_execute_exact: the
hybrid with exact nonuniform sums; pl_execute_bp_direct: direct
back-projection) against the FP64 oracle's definitions of the same sums, and
the NUFFT path against the exact sum it approximates."""
import numpy as np
import pytest

import oracle
from paper_2109_02842_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_EXACT = 2e-5      # FP32 sums, float-float phases
TOL_FP32 = 1e-4


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def binding():
    from paper_2109_02842_gb300 import build, binding as b
    build.build()
    b.load()
    return b


def small_multi():
    w = wl.small_mono(seed=0)
    xy, sec, ptx, prx, _ = wl.multistatic_array(0.5, 4, 60.0, 2, 16)
    w.mode, w.elem_xy, w.elem_section, w.pair_tx, w.pair_rx = 1, xy, sec, ptx, prx
    w.grid = dict(w.grid, nx=24, ny=20)
    return w


def echo_of(w, seed=0):
    clean = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, w.pts, w.amp)
    return wl.add_noise(clean, w.snr_db, wl.rng_for(300, seed)).astype(np.complex64)


def case(name):
    if name == "mono":
        return wl.small_mono(seed=1)
    if name == "multi":
        return small_multi()
    w = wl.small_mono(seed=2)            # ragged grid, voxel heights off the scan grid
    w.grid = dict(w.grid, nx=21, ny=13, nz=9, z0=-0.037, dz=0.0081)
    return w


@pytest.mark.parametrize("name", ["mono", "multi", "ragged"])
def test_exact_sum_matches_oracle(binding, name):
    w = case(name)
    e = echo_of(w)
    plan = binding.Plan.from_workload(w)
    img = plan.execute_exact(torch.from_numpy(e).cuda()).cpu().numpy()
    ref = oracle.hybrid_exact(w.mode, w.tx_xy, w.rx_xy, e, w.z_scan, w.f_hz, w.n_pad,
                              w.pix_xy(), w.axis("z"))
    err = rel(img.reshape(w.grid["nz"], -1), ref)
    print("exact sum %s: rel L2 %.3e" % (name, err))
    assert err < TOL_EXACT


@pytest.mark.parametrize("name", ["mono", "multi"])
def test_nufft_path_matches_exact_sum(binding, name):
    # the method (NUFFT, tensor-core back-projection) against the exact sum it
    # approximates, both on the GPU
    w = case(name)
    e = torch.from_numpy(echo_of(w)).cuda()
    plan = binding.Plan.from_workload(w)
    a = plan.execute(e).cpu().numpy()
    b = plan.execute_exact(e).cpu().numpy()
    err = rel(a, b)
    print("NUFFT path vs exact sum %s: rel L2 %.3e" % (name, err))
    assert err < TOL_FP32


def sampled_voxels(w, n, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = w.grid["nz"], w.grid["ny"], w.grid["nx"]
    flat = rng.choice(nx * ny * nz, size=n, replace=False)
    iz, rem = np.divmod(flat, nx * ny)
    iy, ix = np.divmod(rem, nx)
    xyz = np.stack([w.axis("x")[ix], w.axis("y")[iy], w.axis("z")[iz]], axis=1)
    return flat, xyz


@pytest.mark.parametrize("name", ["mono", "multi", "uneven_band"])
def test_direct_bp_matches_oracle(binding, name):
    w = case("multi" if name == "multi" else "mono")
    if name == "uneven_band":          # per-term phases instead of the rotation
        rng = np.random.default_rng(5)
        df = w.f_hz[1] - w.f_hz[0]
        w.f_hz = np.sort(w.f_hz + rng.uniform(-0.2, 0.2, w.f_hz.size) * df)
    e = echo_of(w)
    plan = binding.Plan.from_workload(w)
    img = plan.execute_bp_direct(torch.from_numpy(e).cuda()).cpu().numpy().ravel()
    flat, xyz = sampled_voxels(w, 400, 3)
    ref = oracle.bp_direct(w.tx_xy, w.rx_xy, e, w.z_scan, w.f_hz, xyz)
    err = rel(img[flat], ref)
    print("direct BP %s: rel L2 %.3e" % (name, err))
    assert err < TOL_EXACT


def test_bp_and_hybrid_focus_on_the_same_voxel(binding):
    # the method and the comparison BP image the same point target (Sec. III)
    w = wl.small_mono(seed=4)
    w.pts, w.amp = w.pts[:1], w.amp[:1]
    e = torch.from_numpy(echo_of(w)).cuda()
    plan = binding.Plan.from_workload(w)
    g_h = np.abs(plan.execute(e).cpu().numpy())
    g_b = np.abs(plan.execute_bp_direct(e).cpu().numpy())
    ph = np.unravel_index(np.argmax(g_h), g_h.shape)
    pb = np.unravel_index(np.argmax(g_b), g_b.shape)
    assert max(abs(a - b) for a, b in zip(ph, pb)) <= 1, (ph, pb)
    c = np.corrcoef(g_h.ravel(), g_b.ravel())[0, 1]
    print("|g| correlation hybrid vs BP: %.3f" % c)
    assert c > 0.9


def _width_3db(line, step):
    a = np.abs(line) / np.abs(line).max()
    i = int(np.argmax(a))
    lo = hi = i
    while lo > 0 and a[lo] >= 0.5 ** 0.5:
        lo -= 1
    while hi < a.size - 1 and a[hi] >= 0.5 ** 0.5:
        hi += 1
    return (hi - lo) * step


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_point_spread_widths_match_design(binding, axis):
    # -3 dB widths of the GPU image of one point at the scene centre against
    # the Sec. II-D resolutions reported by pl_design (0.5x - 2x, as the
    # formulas are approximations)
    w = wl.small_mono(seed=0)
    step, n = 0.0005, 161
    t0 = -(n // 2) * step
    g = dict(x0=0.0, dx=step, nx=1, y0=0.0, dy=step, ny=1, z0=0.0, dz=step, nz=1)
    g[axis + "0"], g["n" + axis] = t0, n
    w.grid = g
    s = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, np.zeros((1, 3)), np.ones(1))
    plan = binding.Plan.from_workload(w)
    img = plan.execute(torch.from_numpy(s.astype(np.complex64)).cuda()).cpu().numpy().ravel()
    got = _width_3db(img, step)
    want = binding.design(w)["res_" + axis]
    print("point spread %s: -3 dB width %.4f m, Sec. II-D %.4f m" % (axis, got, want))
    assert 0.5 * want <= got <= 2.0 * want
