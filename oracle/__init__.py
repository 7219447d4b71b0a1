"""FP64 CPU oracle for the polyline-array hybrid reconstruction.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA product path
never imports, links or calls it, and it shares no code with that path.

The arithmetic lives in ``polyline_oracle.c`` (plain loops, double precision);
this module only marshals NumPy arrays into it. Every function cites the
passage of Wang, Li, Zhao, Sun, "Near-Field Millimeter-Wave Imaging via Arrays
in the Shape of Polyline" (arXiv 2109.02842) that it follows.

Parity status: the echo model, the z-DFT, the exact-sum hybrid (Eq. 7 / 17-19),
the z inverse transform, the direct back-projection and the range profile of
step (8a)/(19a) are each pinned by tests in ``tests/test_oracle_pins.py``
(closed forms, library routines, adjoint identity, mono/multi identity,
point-target focusing; the range profile by the inverse DFT at k_z = 0, the
mono/multi identity q_mono(l) = q_multi(2 l) at k_z != 0, and the split
kappa a = kappa' a + kappa_0 a against the exact-sum hybrid in both modes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polyline_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

C0 = 299792458.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.or_num_threads.restype = I
        lib.or_kz.restype = D
        lib.or_kz.argtypes = [I, I, D]
        lib.or_synth_echo.argtypes = [I, P, P, I, P, I, P, I, P, P, P]
        lib.or_zdft.argtypes = [I, I, I, I, P, P]
        lib.or_hybrid_spectral.argtypes = [I, I, P, P, I, D, I, P, P, I, P, P]
        lib.or_zidft.argtypes = [I, D, D, I, P, I, P, P]
        lib.or_bp_direct.argtypes = [I, P, P, I, P, I, P, P, I, P, P]
        lib.or_range_profile.argtypes = [I, I, D, I, P, P, I, I, I, P, P]
        _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().or_num_threads())


def kz_bins(n_pad: int, dz: float) -> np.ndarray:
    """k_z of each DFT bin (fftfreq order, Nyquist negative), Sec. II-A Eq. (2)."""
    lib = _load()
    return np.array([lib.or_kz(u, n_pad, dz) for u in range(n_pad)])


def synth_echo(tx_xy, rx_xy, z_scan, f_hz, pts, amp) -> np.ndarray:
    """Echo of point scatterers, Eq. (1) (mono: Tx = Rx) and Eq. (10) (multi).

    Returns complex128 [n_chan][n_scan][n_f]:
    s = sum_t amp_t exp(-j k (R_T + R_R)).
    """
    tx = _f64(tx_xy).reshape(-1, 2)
    rx = _f64(rx_xy).reshape(-1, 2)
    z = _f64(z_scan).ravel()
    f = _f64(f_hz).ravel()
    p = _f64(pts).reshape(-1, 3)
    a = _c128(np.broadcast_to(np.asarray(amp, dtype=np.complex128), (p.shape[0],)))
    out = np.zeros((tx.shape[0], z.size, f.size), dtype=np.complex128)
    _load().or_synth_echo(tx.shape[0], _ptr(tx), _ptr(rx), z.size, _ptr(z), f.size,
                          _ptr(f), p.shape[0], _ptr(p), _ptr(a), _ptr(out))
    return out


def zdft(s, n_pad: int) -> np.ndarray:
    """Zero-padded DFT along the scan axis, Eq. (2): [c][n][m] -> [c][u][m]."""
    s = _c128(s)
    c, n, m = s.shape
    out = np.zeros((c, n_pad, m), dtype=np.complex128)
    _load().or_zdft(c, n, m, n_pad, _ptr(s), _ptr(out))
    return out


def hybrid_spectral(mode: int, tx_xy, rx_xy, S, dz: float, f_hz, pix_xy) -> np.ndarray:
    """Exact-sum inversion in the k_z domain, Eq. (7) (mode 0) / Eq. (17)-(19) (mode 1).

    Returns complex128 G[u][pix].
    """
    S = _c128(S)
    c, n_pad, m = S.shape
    tx = _f64(tx_xy).reshape(-1, 2)
    rx = _f64(rx_xy).reshape(-1, 2)
    f = _f64(f_hz).ravel()
    pix = _f64(pix_xy).reshape(-1, 2)
    G = np.zeros((n_pad, pix.shape[0]), dtype=np.complex128)
    _load().or_hybrid_spectral(mode, c, _ptr(tx), _ptr(rx), n_pad, dz, m, _ptr(f),
                               _ptr(S), pix.shape[0], _ptr(pix), _ptr(G))
    return G


def zidft(G, dz: float, z0_scan: float, z_vox) -> np.ndarray:
    """Inverse transform over k_z at arbitrary heights, Eq. (9): G[u][pix] -> g[z][pix]."""
    G = _c128(G)
    n_pad, n_pix = G.shape
    z = _f64(z_vox).ravel()
    g = np.zeros((z.size, n_pix), dtype=np.complex128)
    _load().or_zidft(n_pad, dz, z0_scan, n_pix, _ptr(G), z.size, _ptr(z), _ptr(g))
    return g


def hybrid_exact(mode: int, tx_xy, rx_xy, s, z_scan, f_hz, n_pad: int, pix_xy, z_vox,
                 return_spectral: bool = False):
    """The paper's hybrid method with exact nonuniform sums (Sec. II-A/B).

    z-DFT (Eq. 2) -> exact time-domain inversion per k_z (Eq. 7 / 19) ->
    inverse transform over k_z (Eq. 9). Returns g[z][pix] (complex128), and
    optionally (S, G) as well.
    """
    z_scan = _f64(z_scan).ravel()
    dz = float(z_scan[1] - z_scan[0]) if z_scan.size > 1 else 1.0
    S = zdft(s, n_pad)
    G = hybrid_spectral(mode, tx_xy, rx_xy, S, dz, f_hz, pix_xy)
    g = zidft(G, dz, float(z_scan[0]), z_vox)
    if return_spectral:
        return g, S, G
    return g


def bp_direct(tx_xy, rx_xy, s, z_scan, f_hz, vox_xyz) -> np.ndarray:
    """Direct back-projection (Sec. III comparison algorithm), g[vox]."""
    s = _c128(s)
    c, n, m = s.shape
    tx = _f64(tx_xy).reshape(-1, 2)
    rx = _f64(rx_xy).reshape(-1, 2)
    z = _f64(z_scan).ravel()
    f = _f64(f_hz).ravel()
    v = _f64(vox_xyz).reshape(-1, 3)
    g = np.zeros(v.shape[0], dtype=np.complex128)
    _load().or_bp_direct(c, _ptr(tx), _ptr(rx), n, _ptr(z), m, _ptr(f), _ptr(s),
                         v.shape[0], _ptr(v), _ptr(g))
    return g


def range_profile(mode: int, S, dz: float, f_hz, c: int, u: int, l) -> np.ndarray:
    """Range profile q_{c,u}(l) of step (8a)/(19a), evaluated exactly at ranges l."""
    S = _c128(S)
    nc, n_pad, m = S.shape
    f = _f64(f_hz).ravel()
    l = _f64(l).ravel()
    q = np.zeros(l.size, dtype=np.complex128)
    _load().or_range_profile(mode, n_pad, dz, m, _ptr(f), _ptr(S), c, u, l.size,
                             _ptr(l), _ptr(q))
    return q
