"""Seeded synthetic inputs: array geometry, scan, frequencies, image grid, scenes.

This module is the one place both sides of every parity test take their
inputs from. It holds none of the reconstruction's arithmetic: no dispersion,
no transforms, no back-projection and no echo model (the echo of a scene is
computed by the caller, by the CPU oracle in tests or by the library's scene
synthesis kernel in the benchmark). Random numbers come from NumPy's PCG64,
one stream per (workload, scene index).

Array topology (Sec. I, II-A and Fig. 1 of the paper): ``n_sections`` equal
chords of a circle of radius R, scanned along z. The circle centre is the
origin and the image centre; chord joints sit at azimuth
phi_j = -span/2 + j*span/n_sections at (R sin phi, -R cos phi), so y is the
down-range direction. Elements are cell-centred on each chord, at
(i + 1/2) L / n along it.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import numpy as np

C0 = 299792458.0


@dataclass
class Workload:
    """One reconstruction problem (geometry + scan + band + grid + scene)."""
    name: str
    mode: int                      # 0 monostatic, 1 multistatic
    radius: float
    n_sections: int
    chord_len: float
    elem_xy: np.ndarray            # [n_elem][2] element positions (m)
    elem_section: np.ndarray       # [n_elem] section index of each element
    pair_tx: np.ndarray            # [n_pairs] element index of each Tx (multi)
    pair_rx: np.ndarray            # [n_pairs] element index of each Rx (multi)
    z0: float                      # first scan position z'_0 (m)
    dz: float                      # scan step (m)
    n_scan: int
    n_pad: int                     # z-FFT length N_p >= n_scan
    f_hz: np.ndarray               # [n_f] ascending
    grid: dict                     # x0,dx,nx,y0,dy,ny,z0,dz,nz (voxel centres)
    pts: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    amp: np.ndarray = field(default_factory=lambda: np.zeros(0, np.complex128))
    snr_db: float | None = 30.0
    seed: int = 0

    # channel positions ------------------------------------------------------
    @property
    def n_chan(self) -> int:
        return self.elem_xy.shape[0] if self.mode == 0 else self.pair_tx.size

    @property
    def tx_xy(self) -> np.ndarray:
        return self.elem_xy if self.mode == 0 else self.elem_xy[self.pair_tx]

    @property
    def rx_xy(self) -> np.ndarray:
        return self.elem_xy if self.mode == 0 else self.elem_xy[self.pair_rx]

    @property
    def z_scan(self) -> np.ndarray:
        return self.z0 + self.dz * np.arange(self.n_scan)

    @property
    def n_f(self) -> int:
        return self.f_hz.size

    def axis(self, a: str) -> np.ndarray:
        g = self.grid
        return g[a + "0"] + g["d" + a] * np.arange(g["n" + a])

    def pix_xy(self) -> np.ndarray:
        """[ny*nx][2] pixel centres, x fastest."""
        xs, ys = self.axis("x"), self.axis("y")
        X, Y = np.meshgrid(xs, ys)
        return np.stack([X.ravel(), Y.ravel()], axis=1)

    def updates_per_scan(self) -> float:
        """Element-voxel-frequency terms of the exact sum: C * Nx * Ny * Nz * M."""
        g = self.grid
        return float(self.n_chan) * g["nx"] * g["ny"] * g["nz"] * self.n_f


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------
def chord_joints(radius: float, n_sections: int, span_deg: float) -> np.ndarray:
    """[n_sections+1][2] chord end points on the circle (Fig. 1 topology)."""
    span = math.radians(span_deg)
    phi = -span / 2 + span * np.arange(n_sections + 1) / n_sections
    return np.stack([radius * np.sin(phi), -radius * np.cos(phi)], axis=1)


def cell_centred(p0: np.ndarray, p1: np.ndarray, n: int) -> np.ndarray:
    t = (np.arange(n) + 0.5) / n
    return p0[None, :] + t[:, None] * (p1 - p0)[None, :]


def monostatic_array(radius, n_sections, span_deg, per_chord):
    j = chord_joints(radius, n_sections, span_deg)
    xy = np.concatenate([cell_centred(j[s], j[s + 1], per_chord) for s in range(n_sections)])
    sec = np.repeat(np.arange(n_sections), per_chord)
    return xy, sec, float(np.linalg.norm(j[1] - j[0]))


def multistatic_array(radius, n_sections, span_deg, n_tx, n_rx, cross_section=False):
    """Tx and Rx interleaved on each chord; pairs = all Tx x Rx within a chord,
    and with ``cross_section`` also every Tx with every Rx of the neighbouring
    chords (s - 1 and s + 1), the cross-section pairs Sec. II-C allows.

    Element order: for each section, its n_tx transmitters then its n_rx
    receivers. Pair order: section, then Tx, then Rx (the within-chord pairs
    of all sections first, then the cross-section pairs in the same order,
    neighbouring chord s - 1 before s + 1).
    """
    j = chord_joints(radius, n_sections, span_deg)
    xy, sec, ptx, prx = [], [], [], []
    base = 0
    for s in range(n_sections):
        xy.append(cell_centred(j[s], j[s + 1], n_tx))
        xy.append(cell_centred(j[s], j[s + 1], n_rx))
        sec += [s] * (n_tx + n_rx)
        for t in range(n_tx):
            for r in range(n_rx):
                ptx.append(base + t)
                prx.append(base + n_tx + r)
        base += n_tx + n_rx
    if cross_section:
        per = n_tx + n_rx
        for s in range(n_sections):
            for t in range(n_tx):
                for nb in (s - 1, s + 1):
                    if 0 <= nb < n_sections:
                        for r in range(n_rx):
                            ptx.append(s * per + t)
                            prx.append(nb * per + n_tx + r)
    return (np.concatenate(xy), np.array(sec), np.array(ptx), np.array(prx),
            float(np.linalg.norm(j[1] - j[0])))


def centred_axis(extent: float, n: int, centre: float = 0.0):
    d = extent / n
    return centre - extent / 2 + 0.5 * d, d


def uniform_freqs(f0: float, f1: float, n: int) -> np.ndarray:
    return np.linspace(f0, f1, n)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------
def rng_for(workload_id: int, scene: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([workload_id, scene]))


def uniform_points(rng, lo, hi, n):
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    return lo + (hi - lo) * rng.random((n, 3))


def elliptic_cylinder_points(rng, sx, sy, z_lo, z_hi, n):
    """Points uniform in arclength on the ellipse (semi-axes sx, sy) and in z."""
    out = np.empty((n, 3))
    got = 0
    vmax = max(sx, sy)
    while got < n:
        th = rng.uniform(0, 2 * np.pi, 2 * (n - got) + 8)
        speed = np.sqrt((sx * np.sin(th)) ** 2 + (sy * np.cos(th)) ** 2)
        keep = th[rng.random(th.size) * vmax < speed][: n - got]
        out[got:got + keep.size, 0] = sx * np.cos(keep)
        out[got:got + keep.size, 1] = sy * np.sin(keep)
        got += keep.size
    out[:, 2] = rng.uniform(z_lo, z_hi, n)
    return out


def bright_points(rng, lo, hi, n, sx, sy, min_gap):
    """Isolated points uniform in the box, at least ``min_gap`` off the ellipse."""
    pts = []
    while len(pts) < n:
        p = uniform_points(rng, lo, hi, 1)[0]
        r = math.hypot(p[0] / sx, p[1] / sy)
        if abs(r - 1.0) * min(sx, sy) > min_gap:
            pts.append(p)
    return np.array(pts)


def complex_noise(rng, shape) -> np.ndarray:
    """Unit-variance circular complex Gaussian noise (variance split re/im)."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def add_noise(clean: np.ndarray, snr_db: float | None, rng) -> np.ndarray:
    """Noise power = 10^(-SNR/10) * mean |s_clean|^2 over the whole cube."""
    if snr_db is None:
        return clean
    p = float(np.mean(np.abs(clean) ** 2))
    return clean + math.sqrt(p * 10 ** (-snr_db / 10)) * complex_noise(rng, clean.shape)


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------
def small_mono(seed: int = 0, n_pts: int = 5) -> Workload:
    """Monostatic, 4 chords of R = 0.5 m over 60 deg, 16 elements per chord;
    32 scans at 5 mm; 16 frequencies 28-33 GHz; 32^3 voxels over a 0.2 m
    cube at the circle centre; 5 points, amplitudes U(0.5, 1); 30 dB SNR."""
    xy, sec, L = monostatic_array(0.5, 4, 60.0, 16)
    n, dz = 32, 0.005
    z0 = -(n - 1) / 2 * dz
    x0, dx = centred_axis(0.2, 32)
    rng = rng_for(1, seed)
    span = (z0, z0 + (n - 1) * dz)
    pts = uniform_points(rng, (-0.1, -0.1, span[0]), (0.1, 0.1, span[1]), n_pts)
    amp = rng.uniform(0.5, 1.0, n_pts).astype(np.complex128)
    return Workload("mono-4x16-32scan-16f-32^3", 0, 0.5, 4, L, xy, sec,
                    np.zeros(0, int), np.zeros(0, int), z0, dz, n, 64,
                    uniform_freqs(28e9, 33e9, 16),
                    dict(x0=x0, dx=dx, nx=32, y0=x0, dy=dx, ny=32, z0=x0, dz=dx, nz=32),
                    pts, amp, 30.0, seed)


def _cylinder_scene(rng, n_surf, n_bright, height, zc, box_xy, z_span, vox):
    surf = elliptic_cylinder_points(rng, 0.15, 0.10, zc - height / 2, zc + height / 2, n_surf)
    br = bright_points(rng, (-box_xy, -box_xy, z_span[0]), (box_xy, box_xy, z_span[1]),
                       n_bright, 0.15, 0.10, 2 * vox)
    pts = np.concatenate([surf, br])
    a = rng.lognormal(0.0, 0.5, n_surf + n_bright)
    a[n_surf:] *= 5.0
    return pts, a.astype(np.complex128)


def full_mono(seed: int = 0, n_surf: int = 2000, n_bright: int = 20) -> Workload:
    """Monostatic, 8 chords of R = 0.6 m over 120 deg, 48 elements per chord
    (384); 200 scans at 5 mm; 64 frequencies 24-34 GHz; 256 x 256 x 200
    voxels over 0.4 x 0.4 x 1.0 m (z on the scan grid); elliptic cylinder
    (0.15 / 0.10 m, 0.9 m high) with 2000 surface points + 20 bright points,
    lognormal(0, 0.5) amplitudes; 30 dB SNR."""
    xy, sec, L = monostatic_array(0.6, 8, 120.0, 48)
    n, dz = 200, 0.005
    z0 = -(n - 1) / 2 * dz
    x0, dx = centred_axis(0.4, 256)
    rng = rng_for(2, seed)
    pts, amp = _cylinder_scene(rng, n_surf, n_bright, 0.9, 0.0, 0.2,
                               (z0, z0 + (n - 1) * dz), dx)
    return Workload("mono-8x48-200scan-64f-256x256x200", 0, 0.6, 8, L, xy, sec,
                    np.zeros(0, int), np.zeros(0, int), z0, dz, n, 200,
                    uniform_freqs(24e9, 34e9, 64),
                    dict(x0=x0, dx=dx, nx=256, y0=x0, dy=dx, ny=256, z0=z0, dz=dz, nz=200),
                    pts, amp, 30.0, seed)


def multi(seed: int = 0, n_surf: int = 500, n_bright: int = 10) -> Workload:
    """Multistatic, 8 chords of R = 0.6 m over 120 deg, 4 Tx + 32 Rx per chord,
    all Tx-Rx pairs within a chord (1024); 128 scans at 5 mm; 64 frequencies
    24-34 GHz; 192 x 192 x 128 voxels over 0.4 x 0.4 x 0.64 m (z on the scan
    grid); 500 surface + 10 bright points."""
    xy, sec, ptx, prx, L = multistatic_array(0.6, 8, 120.0, 4, 32)
    n, dz = 128, 0.005
    z0 = -(n - 1) / 2 * dz
    x0, dx = centred_axis(0.4, 192)
    rng = rng_for(3, seed)
    span = (z0, z0 + (n - 1) * dz)
    pts, amp = _cylinder_scene(rng, n_surf, n_bright, 0.9 * (span[1] - span[0]), 0.0,
                               0.2, span, dx)
    return Workload("multi-8x(4tx,32rx)-128scan-64f-192x192x128", 1, 0.6, 8, L, xy, sec,
                    ptx, prx, z0, dz, n, 128, uniform_freqs(24e9, 34e9, 64),
                    dict(x0=x0, dx=dx, nx=192, y0=x0, dy=dx, ny=192, z0=z0, dz=dz, nz=128),
                    pts, amp, 30.0, seed)


def paper_table1(mode: int, seed: int = 0, n_scan: int = 64, n_grid: int = 64,
                 cross_section: bool = False) -> Workload:
    """Table I of the paper: R0 = 1.0 m, 3 sections, 30-35 GHz in 51 steps,
    dz = 0.5 cm; mono 40 elements per section at 0.48 cm; multi 4 Tx in total
    (at the joints and ends) with 20 Rx per section, pairs within a section
    (each section's Rx with the two Tx at its ends); with ``cross_section``
    also every Tx with the Rx of the sections it does not bound (Sec. II-C:
    a joint transmitter may also serve the farther sections).
    The paper gives no scan count and no image grid: ``n_scan`` scans and an
    ``n_grid``^3 grid over a 0.2 m cube are this module's choice. The chord
    length is set by the element count times the stated spacing (0.192 m),
    which fixes the span angle."""
    L = 40 * 0.0048
    span = math.degrees(3 * 2 * math.asin(L / 2 / 1.0))
    j = chord_joints(1.0, 3, span)
    if mode == 0:
        xy, sec, L = monostatic_array(1.0, 3, span, 40)
        ptx = prx = np.zeros(0, int)
    else:
        rx = [cell_centred(j[s], j[s + 1], 20) for s in range(3)]
        xy = np.concatenate([j] + rx)                      # 4 Tx at joints/ends
        sec = np.array([0, 0, 1, 2] + sum(([s] * 20 for s in range(3)), []))
        ptx, prx = [], []
        for s in range(3):
            for t in (s, s + 1):
                for r in range(20):
                    ptx.append(t)
                    prx.append(4 + 20 * s + r)
        if cross_section:
            for s in range(3):
                for t in range(4):
                    if t not in (s, s + 1):
                        for r in range(20):
                            ptx.append(t)
                            prx.append(4 + 20 * s + r)
        ptx, prx = np.array(ptx), np.array(prx)
    dz = 0.005
    z0 = -(n_scan - 1) / 2 * dz
    x0, dx = centred_axis(0.2, n_grid)
    rng = rng_for(6, seed)
    span_z = (z0, z0 + (n_scan - 1) * dz)
    pts = uniform_points(rng, (-0.1, -0.1, max(span_z[0], -0.1)),
                         (0.1, 0.1, min(span_z[1], 0.1)), 5)
    amp = rng.uniform(0.5, 1.0, 5).astype(np.complex128)
    n_pad = 1 << int(math.ceil(math.log2(2 * n_scan)))
    name = "table1-%s%s" % ("mono" if mode == 0 else "multi", "-cross" if cross_section else "")
    return Workload(name, mode, 1.0, 3, L, xy,
                    sec, ptx, prx, z0, dz, n_scan, n_pad, uniform_freqs(30e9, 35e9, 51),
                    dict(x0=x0, dx=dx, nx=n_grid, y0=x0, dy=dx, ny=n_grid, z0=x0, dz=dx,
                         nz=n_grid), pts, amp, 30.0, seed)


def smooth_at_least(n: int) -> int:
    """Smallest 2^a 3^b 5^c >= n."""
    best = None
    p2 = 1
    while p2 < 2 * n:
        p3 = p2
        while p3 < 2 * n:
            p5 = p3
            while p5 < 2 * n:
                if p5 >= n and (best is None or p5 < best):
                    best = p5
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return best


def batch_scene(index: int, seed: int = 0) -> Workload:
    """One of the uneven monostatic scenes of the batched workload: sections
    4-12, 16-48 elements per chord, 64-256 scans, 32-96 frequencies within
    24-34 GHz, a cubic image of 64-160 voxels a side, 50-500 points, 30 dB.
    Radius 0.6 m over 120 deg; the image z extent is the scene's scan span."""
    rng = rng_for(4, 1000 * seed + index)
    ns = int(rng.integers(4, 13))
    per = int(rng.integers(16, 49))
    n = int(rng.integers(64, 257))
    nf = int(rng.integers(32, 97))
    ng = int(rng.integers(64, 161))
    npts = int(rng.integers(50, 501))
    return uneven_scene(rng, ns, per, n, nf, ng, npts, "batch-scene-%d" % index, seed)


def uneven_scene(rng, ns: int, per: int, n: int, nf: int, ng: int, npts: int,
                 name: str = "uneven-scene", seed: int = 0) -> Workload:
    """A monostatic scene of the batched workload's family with the given
    sizes: ``ns`` chords of R = 0.6 m over 120 deg with ``per`` elements each,
    ``n`` scans at 5 mm (N_p the smallest 5-smooth length >= 2 n), ``nf``
    frequencies over 24-34 GHz, an ``ng``^3 image (0.4 x 0.4 m, z over the
    scan span) and ``npts`` points U(0.5, 1) drawn from ``rng``."""
    xy, sec, L = monostatic_array(0.6, ns, 120.0, per)
    dz = 0.005
    z0 = -(n - 1) / 2 * dz
    zext = n * dz
    x0, dx = centred_axis(0.4, ng)
    zz0, zdz = centred_axis(zext, ng)
    pts = uniform_points(rng, (-0.15, -0.15, z0), (0.15, 0.15, z0 + (n - 1) * dz), npts)
    amp = rng.uniform(0.5, 1.0, npts).astype(np.complex128)
    return Workload(name, 0, 0.6, ns, L, xy, sec, np.zeros(0, int),
                    np.zeros(0, int), z0, dz, n, smooth_at_least(2 * n),
                    uniform_freqs(24e9, 34e9, nf),
                    dict(x0=x0, dx=dx, nx=ng, y0=x0, dy=dx, ny=ng, z0=zz0, dz=zdz, nz=ng),
                    pts, amp, 30.0, seed)


WORKLOADS = {
    "small_mono": small_mono,
    "full_mono": full_mono,
    "multi": multi,
}
