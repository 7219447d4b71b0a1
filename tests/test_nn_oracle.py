"""Pins of the learned path's CPU oracle (oracle/nn_oracle.py): conv3d against
scipy.signal.correlate, its gradients against central finite differences, the
pooling/upsampling adjoint pair, the loss gradient, and Adam's first step
(which moves every parameter by lr against the sign of its gradient)."""
import numpy as np
import pytest

from oracle import nn_oracle as nn

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3d_is_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 6, 7, 3))
    w = rng.standard_normal((4, 27, 3))
    b = rng.standard_normal(4)
    y = nn.conv3d(x, w, b)
    for co in range(4):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            k = w[co, :, ci].reshape(3, 3, 3)
            ref += scipy_signal.correlate(x[..., ci], k, mode="same")
        assert np.allclose(y[..., co], ref, atol=1e-12)


def test_conv3d_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 2))
    w = rng.standard_normal((3, 27, 2))
    b = rng.standard_normal(3)
    gy = rng.standard_normal((3, 4, 5, 3))
    gx, gw, gb = nn.conv3d_backward(x, w, gy)
    f = lambda xx, ww, bb: float(np.sum(gy * nn.conv3d(xx, ww, bb)))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 3, 1), (2, 3, 4, 0), (0, 3, 0, 1)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert abs((f(x + e, w, b) - f(x - e, w, b)) / (2 * h) - gx[idx]) < 1e-6
    for idx in [(0, 0, 0), (2, 13, 1), (1, 26, 0)]:
        e = np.zeros_like(w)
        e[idx] = h
        assert abs((f(x, w + e, b) - f(x, w - e, b)) / (2 * h) - gw[idx]) < 1e-6
    assert np.allclose(gb, gy.sum(axis=(0, 1, 2)))


def test_pool_and_upsample_are_adjoint_up_to_8():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((4, 6, 8, 3))
    c = rng.standard_normal((2, 3, 4, 3))
    # <avgpool(a), c> = <a, upsample(c)> / 8
    assert abs(np.vdot(nn.avgpool2(a), c) - np.vdot(a, nn.upsample2(c)) / 8) < 1e-12


def test_loss_gradient_and_features():
    rng = np.random.default_rng(3)
    p = rng.standard_normal((2, 3, 4, 2))
    t = rng.standard_normal((2, 3, 4, 2))
    L, g = nn.rel_l2_loss(p, t)
    h = 1e-7
    e = np.zeros_like(p)
    e[1, 2, 3, 0] = h
    assert abs((nn.rel_l2_loss(p + e, t)[0] - nn.rel_l2_loss(p - e, t)[0]) / (2 * h)
               - g[1, 2, 3, 0]) < 1e-6
    z = rng.standard_normal((2, 3, 4)) + 1j * rng.standard_normal((2, 3, 4))
    f, s = nn.features(z)
    assert np.isclose(f[..., 2].max(), 1.0)
    assert np.allclose(f[..., 0] ** 2 + f[..., 1] ** 2, f[..., 2] ** 2)
    assert np.allclose(s * (f[..., 0] + 1j * f[..., 1]), z)


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(4)
    p = rng.standard_normal(10)
    g = rng.standard_normal(10)
    p1, m, v = nn.adam(p, g, np.zeros(10), np.zeros(10), 1, 1e-3)
    assert np.allclose(p - p1, 1e-3 * np.sign(g), rtol=1e-4)
