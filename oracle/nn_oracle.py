"""FP64 CPU oracle for the learned fast path's layers (test infrastructure only).

Plain NumPy definitions, one per layer, written from the textbook definitions
(no blocking, no fusion): channels-last volumes x[z][y][x][c], 'same'
zero padding, stride 1, 3x3x3 kernels, weights w[co][tap][ci] with
tap = (dz*3 + dy)*3 + dx and an input offset of (dz-1, dy-1, dx-1).
Pinned in tests/test_nn_oracle.py against scipy.signal.correlate (a library
routine) and against central finite differences of the forward functions.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in range(3) for dy in range(3) for dx in range(3)]


def _shifted(x, dz, dy, dx):
    """x[z + dz - 1][y + dy - 1][x + dx - 1], zero outside."""
    D, H, W = x.shape[:3]
    out = np.zeros_like(x)
    zs = slice(max(0, 1 - dz), min(D, D + 1 - dz))
    ys = slice(max(0, 1 - dy), min(H, H + 1 - dy))
    xs = slice(max(0, 1 - dx), min(W, W + 1 - dx))
    zi = slice(zs.start + dz - 1, zs.stop + dz - 1)
    yi = slice(ys.start + dy - 1, ys.stop + dy - 1)
    xi = slice(xs.start + dx - 1, xs.stop + dx - 1)
    out[zs, ys, xs] = x[zi, yi, xi]
    return out


def conv3d(x, w, b=None):
    """y[v][co] = b[co] + sum_tap sum_ci w[co][tap][ci] x[v + off(tap)][ci]."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += _shifted(x, dz, dy, dx) @ w[:, t, :].T
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3d_backward(x, w, gy):
    """Gradients of sum(gy * conv3d(x, w, b)) w.r.t. x, w and b."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    gy = np.asarray(gy, np.float64)
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(TAPS):
        xs = _shifted(x, dz, dy, dx)
        gw[:, t, :] = np.einsum("zyxo,zyxi->oi", gy, xs)
        # adjoint of the shift: move gy back by the opposite offset
        gx += _shifted(gy @ w[:, t, :], 2 - dz, 2 - dy, 2 - dx)
    gb = gy.sum(axis=(0, 1, 2))
    return gx, gw, gb


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    """Mean over 2 x 2 x 2 blocks (even sizes)."""
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def upsample2(x):
    """Nearest-neighbour x2 in every spatial axis."""
    return x.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def features(g):
    """Re g / s, Im g / s, |g| / s of a complex volume, s = max |g| -> [D,H,W,3]."""
    a = np.abs(g)
    s = a.max() if a.max() > 0 else 1.0
    return np.stack([g.real / s, g.imag / s, a / s], axis=-1), s


def rel_l2_loss(pred, target):
    """sum |pred - target|^2 / sum |target|^2 and its gradient w.r.t. pred."""
    d = np.asarray(pred, np.float64) - np.asarray(target, np.float64)
    den = float(np.sum(np.asarray(target, np.float64) ** 2))
    return float(np.sum(d * d)) / den, 2.0 * d / den


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015), bias-corrected."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
