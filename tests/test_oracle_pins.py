"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (NumPy's FFT), a closed form (Pythagorean distances, exact phase
cancellation), an operator identity (the adjoint of the Eq. (6) forward
model), an algebraic identity between the two modes (Eq. 5 vs Eq. 18), and
the physics the paper demonstrates (point targets focus where they are,
Sec. III; resolutions of Sec. II-D). The pins are chosen so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2109_02842_gb300 import workloads as wl

C0 = 299792458.0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --- z-DFT (Eq. 2) ---------------------------------------------------------

@pytest.mark.parametrize("n,n_pad", [(8, 8), (7, 12), (32, 64), (10, 10)])
def test_zdft_is_numpy_fft(n, n_pad):
    rng = np.random.default_rng(1)
    s = rng.standard_normal((3, n, 5)) + 1j * rng.standard_normal((3, n, 5))
    S = oracle.zdft(s, n_pad)
    ref = np.fft.fft(s, n=n_pad, axis=1)
    assert rel(S, ref) < 1e-13


@pytest.mark.parametrize("n_pad", [8, 9, 64, 200])
def test_kz_bins_are_fftfreq(n_pad):
    dz = 0.005
    ref = 2 * np.pi * np.fft.fftfreq(n_pad, d=dz)
    assert np.allclose(oracle.kz_bins(n_pad, dz), ref, rtol=0, atol=1e-9)


def test_zidft_is_numpy_ifft_on_scan_grid():
    rng = np.random.default_rng(2)
    n_pad, dz, z0 = 16, 0.005, -0.03
    G = rng.standard_normal((n_pad, 7)) + 1j * rng.standard_normal((n_pad, 7))
    z = z0 + dz * np.arange(11)
    g = oracle.zidft(G, dz, z0, z)
    ref = np.fft.ifft(G, axis=0)[:11]
    assert rel(g, ref) < 1e-13


# --- echo model (Eq. 1 / Eq. 10) ---------------------------------------------

def test_echo_pythagorean_closed_form():
    # Target at the origin; Tx at (0.3, 0.4) -> rho = 0.5; scans at z' = 0 and
    # z' = 1.2 give R = 0.5 and R = 1.3 (5-12-13). Rx at (0, -0.5): rho = 0.5.
    f = np.array([28e9, 30e9])
    k = 2 * np.pi * f / C0
    z = np.array([0.0, 1.2])
    pts = np.zeros((1, 3))
    amp = np.array([0.7 - 0.2j])
    tx = np.array([[0.3, 0.4]])
    rx = np.array([[0.0, -0.5]])
    mono = oracle.synth_echo(tx, tx, z, f, pts, amp)[0]
    assert np.allclose(mono[0], amp[0] * np.exp(-2j * k * 0.5), atol=1e-12)
    assert np.allclose(mono[1], amp[0] * np.exp(-2j * k * 1.3), atol=1e-12)
    multi = oracle.synth_echo(tx, rx, z, f, pts, amp)[0]
    assert np.allclose(multi[0], amp[0] * np.exp(-1j * k * 1.0), atol=1e-12)
    assert np.allclose(multi[1], amp[0] * np.exp(-1j * k * 2.6), atol=1e-12)


def test_echo_is_linear_in_amplitudes():
    w = wl.small_mono(seed=3)
    p = w.pts[:3]
    a = np.array([0.5, 1.0 + 0.5j, -0.25j])
    whole = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, p, a)
    parts = sum(oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, p[i:i + 1], a[i:i + 1])
                for i in range(3))
    assert rel(whole, parts) < 1e-13


# --- direct back-projection -----------------------------------------------------

def test_bp_direct_phase_cancels_at_target():
    # At the voxel that coincides with the point, every term of the matched
    # filter is amp * k_m, so g = amp * C * N * sum_m k_m exactly.
    w = wl.small_mono(seed=0)
    tgt = np.array([[w.axis("x")[13], w.axis("y")[17], w.z_scan[9]]])
    amp = np.array([0.8 + 0.1j])
    s = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, tgt, amp)
    g = oracle.bp_direct(w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, tgt)
    k = 2 * np.pi * w.f_hz / C0
    expect = amp[0] * w.n_chan * w.n_scan * k.sum()
    assert abs(g[0] - expect) < 1e-9 * abs(expect)
    # one voxel off, the terms no longer add coherently
    off = tgt + np.array([[0.0, 0.02, 0.0]])
    assert abs(oracle.bp_direct(w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, off)[0]) < 0.5 * abs(expect)


# --- exact-sum hybrid (Eq. 7 / Eq. 17-19) ----------------------------------------

def _forward_model(mode, tx, rx, g, kz, k, pix):
    """Eq. (6) / Eq. (17): s(c, k_z, k) = sum_pix g(pix, k_z) exp(-j kappa a_c(pix)).
    Written independently of the oracle, with NumPy broadcasting."""
    rho_t = np.hypot(pix[None, :, 0] - tx[:, None, 0], pix[None, :, 1] - tx[:, None, 1])
    rho_r = np.hypot(pix[None, :, 0] - rx[:, None, 0], pix[None, :, 1] - rx[:, None, 1])
    a = rho_t if mode == 0 else rho_t + rho_r                       # [c][p]
    if mode == 0:
        ksq = 4 * k[None, :] ** 2 - kz[:, None] ** 2                # [u][m]
    else:
        ksq = k[None, :] ** 2 - kz[:, None] ** 2 / 4
    kap = np.sqrt(np.maximum(ksq, 0.0))
    prop = ksq > 0
    ph = np.exp(-1j * kap[None, :, :, None] * a[:, None, None, :])  # [c][u][m][p]
    return np.einsum("cump,up->cum", ph, g) * prop[None]


@pytest.mark.parametrize("mode", [0, 1])
def test_hybrid_is_adjoint_of_forward_model(mode):
    rng = np.random.default_rng(5)
    n_pad, dz = 8, 0.005
    f = np.linspace(28e9, 33e9, 5)
    k = 2 * np.pi * f / C0
    kz = 2 * np.pi * np.fft.fftfreq(n_pad, d=dz)
    tx = rng.uniform(-0.3, 0.3, (4, 2)) + np.array([0.0, -0.5])
    rx = tx if mode == 0 else rng.uniform(-0.3, 0.3, (4, 2)) + np.array([0.0, -0.5])
    pix = rng.uniform(-0.1, 0.1, (6, 2))
    g = rng.standard_normal((n_pad, 6)) + 1j * rng.standard_normal((n_pad, 6))
    S = rng.standard_normal((4, n_pad, 5)) + 1j * rng.standard_normal((4, n_pad, 5))
    Ag = _forward_model(mode, tx, rx, g, kz, k, pix)
    HS = oracle.hybrid_spectral(mode, tx, rx, S, dz, f, pix)
    lhs = np.vdot(Ag, S * k[None, None, :])       # <A g, K S>
    rhs = np.vdot(g, HS)                           # <g, H S>
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_evanescent_terms_are_zero():
    # dz so coarse that the highest |k_z| exceeds 2 k for every frequency:
    # those bins must come out exactly zero.
    n_pad, dz = 8, 0.05
    f = np.array([3e9, 3.2e9])
    kz = oracle.kz_bins(n_pad, dz)
    S = np.ones((1, n_pad, 2), complex)
    G = oracle.hybrid_spectral(0, [[0, -0.5]], [[0, -0.5]], S, dz, f, [[0.0, 0.0]])
    k = 2 * np.pi * f / C0
    for u in range(n_pad):
        if np.all(4 * k ** 2 <= kz[u] ** 2):
            assert G[u, 0] == 0
        else:
            assert G[u, 0] != 0


def test_mono_equals_multistatic_with_colocated_tx_rx():
    # Eq. (5) with range rho vs Eq. (18) with range rho_T + rho_R = 2 rho:
    # sqrt(k^2 - kz^2/4) * 2 rho == sqrt(4k^2 - kz^2) * rho.
    w = wl.small_mono(seed=1)
    s = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, w.pts, w.amp)
    pix = w.pix_xy()[::37]
    z = w.axis("z")[::5]
    g0 = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, w.n_pad, pix, z)
    g1 = oracle.hybrid_exact(1, w.tx_xy, w.tx_xy, s, w.z_scan, w.f_hz, w.n_pad, pix, z)
    assert rel(g1, g0) < 1e-12


def test_hybrid_is_linear():
    w = wl.small_mono(seed=2)
    pix = w.pix_xy()[::53]
    z = w.axis("z")[::7]
    rng = np.random.default_rng(9)
    s1 = rng.standard_normal((w.n_chan, w.n_scan, w.n_f)) + 0j
    s2 = 1j * rng.standard_normal((w.n_chan, w.n_scan, w.n_f))
    a, b = 0.3 - 1.1j, 2.0
    h = lambda s: oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, w.n_pad, pix, z)
    assert rel(h(a * s1 + b * s2), a * h(s1) + b * h(s2)) < 1e-12


def _peak_index(g, shape):
    return np.unravel_index(int(np.argmax(np.abs(g))), shape)


@pytest.mark.parametrize("mode", [0, 1])
def test_point_target_focuses_within_one_voxel(mode):
    # Sec. III: point targets are focused. A lone point inside the scan span
    # must give the image maximum within one voxel of its true position.
    w = wl.small_mono(seed=0)
    if mode == 1:
        xy, sec, ptx, prx, _ = wl.multistatic_array(0.5, 4, 60.0, 2, 16)
        tx, rx = xy[ptx], xy[prx]
    else:
        tx = rx = w.tx_xy
    xs, ys, zs = w.axis("x"), w.axis("y"), w.axis("z")
    rng = np.random.default_rng(11 + mode)
    for trial in range(3):
        ix, iy = rng.integers(6, 26, 2)
        iz = int(rng.integers(10, 22))
        tgt = np.array([[xs[ix], ys[iy], zs[iz]]])
        if not (w.z_scan[0] < zs[iz] < w.z_scan[-1]):
            continue
        s = oracle.synth_echo(tx, rx, w.z_scan, w.f_hz, tgt, np.array([1.0]))
        g = oracle.hybrid_exact(mode, tx, rx, s, w.z_scan, w.f_hz, w.n_pad, w.pix_xy(), zs)
        pz, py, px = _peak_index(g, (32, 32, 32))
        assert abs(px - ix) <= 1 and abs(py - iy) <= 1 and abs(pz - iz) <= 1, \
            (trial, (px, py, pz), (ix, iy, iz))


def test_range_profile_at_kz0_is_inverse_dft():
    # At k_z = 0 the monostatic kappa' = 2 (k_m - k_0) is uniform for uniform
    # frequencies, so q(l) of step (8a) at l_p = 2 pi p / (2 dk M) is an
    # inverse DFT of S k (NumPy).
    rng = np.random.default_rng(4)
    M = 16
    f = np.linspace(28e9, 33e9, M)
    k = 2 * np.pi * f / C0
    dk = k[1] - k[0]
    S = rng.standard_normal((1, 4, M)) + 1j * rng.standard_normal((1, 4, M))
    l = 2 * np.pi * np.arange(M) / (2 * dk * M)
    q = oracle.range_profile(0, S, 0.005, f, 0, 0, l)
    ref = M * np.fft.ifft(S[0, 0] * k)
    assert rel(q, ref) < 1e-12


@pytest.mark.parametrize("u", [3, 29])
def test_range_profile_mono_at_l_equals_multi_at_2l(u):
    # Eq. (5) vs Eq. (18): kappa_mono(k, k_z) = 2 kappa_multi(k, k_z) for every
    # k and k_z, and so for kappa_0 = kappa(k_0, k_z) too. Hence, at k_z != 0,
    # q_mono(l) = q_multi(2 l) for the same spectrum. A kappa_0 that is wrong
    # in one mode (2 k_0 in both, or the monostatic kappa_0 in mode 1) or a
    # multistatic branch with the monostatic dispersion fails this.
    rng = np.random.default_rng(11)
    M, n_pad, dz = 24, 64, 0.005
    f = np.linspace(24e9, 34e9, M)
    S = rng.standard_normal((2, n_pad, M)) + 1j * rng.standard_normal((2, n_pad, M))
    assert abs(oracle.kz_bins(n_pad, dz)[u]) > 50.0
    l = np.linspace(0.31, 0.93, 17)
    q0 = oracle.range_profile(0, S, dz, f, 1, u, l)
    q1 = oracle.range_profile(1, S, dz, f, 1, u, 2 * l)
    assert np.max(np.abs(q0 - q1)) / np.max(np.abs(q0)) < 1e-12


@pytest.mark.parametrize("mode", [0, 1])
def test_range_profile_times_carrier_is_the_hybrid_sum(mode):
    # Eq. (8a)-(8b) (mode 0) and (19a)-(19b) (mode 1) split the phase as
    # kappa a = kappa' a + kappa_0 a with kappa_0 = kappa(k_0, k_z). For
    # channels whose range a (rho, or rho_T + rho_R) to a pixel is the same,
    # sum_c q_c(a) e^{j kappa_0 a} must equal the exact-sum hybrid G_u at that
    # pixel (Eq. 7 / 19, pinned above by the adjoint identity), at k_z != 0,
    # where kappa_0 differs from 2 k_0 (mode 0) and k_0 (mode 1).
    rng = np.random.default_rng(12 + mode)
    M, n_pad, dz = 20, 32, 0.005
    f = np.linspace(24e9, 34e9, M)
    k0 = 2 * np.pi * f[0] / C0
    S = rng.standard_normal((3, n_pad, M)) + 1j * rng.standard_normal((3, n_pad, M))
    pix = np.array([[0.013, -0.021]])
    phis = np.array([-1.1, -0.4, 0.7])
    if mode == 0:
        rho = 0.55                                   # three elements at range 0.55 m
        tx = pix + rho * np.stack([np.sin(phis), -np.cos(phis)], 1)
        rx = tx
        a = rho
    else:
        # Tx at 0.50 m and Rx at 0.62 m from the pixel: a = 1.12 m per pair
        tx = pix + 0.50 * np.stack([np.sin(phis), -np.cos(phis)], 1)
        rx = pix + 0.62 * np.stack([np.sin(phis + 0.05), -np.cos(phis + 0.05)], 1)
        a = 1.12
    G = oracle.hybrid_spectral(mode, tx, rx, S, dz, f, pix)
    kz = oracle.kz_bins(n_pad, dz)
    for u in (0, 5, 17, 31):
        kap0 = math.sqrt(4 * k0 ** 2 - kz[u] ** 2) if mode == 0 else math.sqrt(k0 ** 2 - kz[u] ** 2 / 4)
        q = sum(oracle.range_profile(mode, S, dz, f, c, u, [a])[0] for c in range(3))
        got = q * np.exp(1j * kap0 * a)
        assert abs(got - G[u, 0]) / abs(G[u, 0]) < 1e-10, (u, got, G[u, 0])


def test_bp_and_hybrid_agree_on_tiny_grid():
    # Sec. III: the proposed method's focusing is very similar to BP. Each
    # point alone peaks at the same voxel under both; for the whole scene the
    # image magnitudes are strongly correlated.
    w = wl.small_mono(seed=4, n_pts=3)
    xs, ys, zs = w.axis("x")[::2], w.axis("y")[::2], w.axis("z")[::2]
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    vox = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    XX, YY = np.meshgrid(xs, ys)
    pix = np.stack([XX.ravel(), YY.ravel()], 1)
    shape = (zs.size, ys.size, xs.size)

    def both(pts, amp):
        s = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, pts, amp)
        gb = oracle.bp_direct(w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, vox)
        gh = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, w.n_pad, pix,
                                 zs).ravel()
        return gb, gh

    for i in range(3):
        gb, gh = both(w.pts[i:i + 1], w.amp[i:i + 1])
        pb, ph = np.array(_peak_index(gb, shape)), np.array(_peak_index(gh, shape))
        assert np.all(np.abs(pb - ph) <= 1), (i, pb, ph)
    gb, gh = both(w.pts, w.amp)
    ab, ah = np.abs(gb), np.abs(gh)
    corr = float(np.dot(ab - ab.mean(), ah - ah.mean()) /
                 (np.linalg.norm(ab - ab.mean()) * np.linalg.norm(ah - ah.mean())))
    assert corr >= 0.9, corr


def _width_3db(line, step):
    a = np.abs(line) / np.abs(line).max()
    i = int(np.argmax(a))
    lo = i
    while lo > 0 and a[lo] >= 0.5 ** 0.5:
        lo -= 1
    hi = i
    while hi < a.size - 1 and a[hi] >= 0.5 ** 0.5:
        hi += 1
    return (hi - lo) * step


def test_resolutions_match_sec_2d_formulas():
    # Sec. II-D: dx ~ lambda_c / (4 sin(theta_h/2)), dy = c / (2B),
    # dz = lambda_c / (4 sin(theta_z/2)). Checked loosely (0.5x - 2x) on the
    # -3 dB width of a point response, sampled finely along each axis.
    w = wl.small_mono(seed=0)
    tgt = np.array([[0.0, 0.0, 0.0]])
    s = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, tgt, np.array([1.0]))
    fc = 0.5 * (w.f_hz[0] + w.f_hz[-1])
    lam = C0 / fc
    B = w.f_hz[-1] - w.f_hz[0]
    theta_h = math.radians(60.0)
    span = w.z_scan[-1] - w.z_scan[0]
    theta_z = 2 * math.atan(span / 2 / 0.5)
    d = 0.0005
    t = d * np.arange(-80, 81)
    zero = np.zeros_like(t)
    gx = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, w.n_pad,
                             np.stack([t, zero], 1), [0.0])[0]
    gy = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, w.n_pad,
                             np.stack([zero, t], 1), [0.0])[0]
    gz = oracle.hybrid_exact(0, w.tx_xy, w.rx_xy, s, w.z_scan, w.f_hz, w.n_pad,
                             [[0.0, 0.0]], t)[:, 0]
    for got, want in [(_width_3db(gx, d), lam / (4 * math.sin(theta_h / 2))),
                      (_width_3db(gy, d), C0 / (2 * B)),
                      (_width_3db(gz, d), lam / (4 * math.sin(theta_z / 2)))]:
        assert 0.5 * want <= got <= 2.0 * want, (got, want)
