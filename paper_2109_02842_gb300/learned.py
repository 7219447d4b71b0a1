"""Learned fast path: a 3-D convolutional encoder-decoder that maps a cheap
reconstruction to the full one (the paper has no learned component; the plain
hybrid method stays the fallback and the yardstick for the network's error).

Cheap reconstruction: every other frequency and a coarse range table (NUFFT
oversampling 1.25, 4 taps). Full reconstruction: all frequencies, sigma = 2,
6 taps. Both come from the library's plain path (`binding.Plan`).

Network (channels-last BF16 activations, FP32 master weights):
    features of the cheap image (Re g / s, Im g / s, |g| / s), s = max |g|
    enc1: 3 -> 16 -> 16         (full resolution)         -> skip1
    enc2: pool, 16 -> 32 -> 32  (1/2)                     -> skip2
    enc3: pool, 32 -> 64 -> 64  (1/4)                     -> skip3
    bottleneck: pool, 64 -> 128 -> 128 (1/8)
    dec3: up, 128 -> 64, + skip3, 64 -> 64
    dec2: up, 64 -> 32, + skip2, 32 -> 32
    dec1: up, 32 -> 16, + skip1, 16 -> 16
    head: 16 -> 2 (linear), added to gain * (Re, Im) of the cheap image / s
          (gain = full / cheap frequency count): the prediction of the full
          image / s is the cheap image plus a learned correction
All 3 x 3 x 3 convolutions with ReLU except the head; pooling is a 2 x 2 x 2
mean, upsampling nearest. Loss: relative L2 between the prediction and the
full image / s. Every layer runs in the library's kernels (pl_nn_* in
include/polyline.h); this module only allocates tensors and sequences calls.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import binding as B

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_S = ctypes.c_size_t

_ARGTYPES = {
    "pl_nn_padded_k": ([_I], _I),
    "pl_nn_conv3d": ([_P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _P], _I),
    "pl_nn_wgrad_workspace": ([_I, _I, _I, _I, _I], _S),
    "pl_nn_conv3d_wgrad": ([_P, _P, _P, _P, _P, _S, _I, _I, _I, _I, _I, _P], _I),
    "pl_nn_weight_flip": ([_P, _P, _I, _I, _P], _I),
    "pl_nn_elementwise": ([_I, _P, _P, _P, _S, _P], _I),
    "pl_nn_resample": ([_I, _P, _P, _I, _I, _I, _I, _P], _I),
    "pl_nn_features": ([_P, _P, _P, _S, _P], _I),
    "pl_nn_loss": ([_P, _P, _P, _P, _P, _S, _P], _I),
    "pl_nn_residual": ([_P, _P, _P, _F, _S, _P], _I),
    "pl_nn_check": ([_P, _P, _P, _F, _S, _P, _P], _I),
    "pl_nn_to_complex": ([_P, _P, _P, _S, _P], _I),
    "pl_nn_adam": ([_P, _P, _P, _P, _P, _S, _F, _F, _F, _F, _I, _P], _I),
}


def lib():
    L = B.load()
    if not getattr(L, "_nn_ready", False):
        for name, (args, res) in _ARGTYPES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        L._nn_ready = True
    return L


def _p(t):
    return None if t is None else _P(t.data_ptr())


def _s():
    import torch
    return _P(torch.cuda.current_stream().cuda_stream)


def conv3d(x, w, bias, dims, cin, cout, relu, out_bf16):
    """Launch pl_nn_conv3d; returns the output tensor."""
    import torch
    D, H, W = dims
    out = torch.empty((D * H * W, cout), dtype=torch.bfloat16 if out_bf16 else torch.float32,
                      device="cuda")
    B._check(lib().pl_nn_conv3d(_p(x), _p(w), _p(bias), _p(out), D, H, W, cin, cout,
                                1 if relu else 0, 1 if out_bf16 else 0, _s()))
    return out


def pool(x, dims, c):
    import torch
    D, H, W = dims
    y = torch.empty((D * H * W // 8, c), dtype=torch.bfloat16, device="cuda")
    B._check(lib().pl_nn_resample(0, _p(x), _p(y), D, H, W, c, _s()))
    return y


def pool_bwd_accum(gy, gx, fine_dims, c):
    D, H, W = fine_dims
    B._check(lib().pl_nn_resample(1, _p(gy), _p(gx), D, H, W, c, _s()))


def upsample(x, coarse_dims, c):
    import torch
    D, H, W = coarse_dims
    y = torch.empty((8 * D * H * W, c), dtype=torch.bfloat16, device="cuda")
    B._check(lib().pl_nn_resample(2, _p(x), _p(y), D, H, W, c, _s()))
    return y


def upsample_bwd(gy, coarse_dims, c):
    import torch
    D, H, W = coarse_dims
    gx = torch.empty((D * H * W, c), dtype=torch.float32, device="cuda")
    B._check(lib().pl_nn_resample(3, _p(gy), _p(gx), D, H, W, c, _s()))
    return gx


def elementwise(op, a, b, out):
    B._check(lib().pl_nn_elementwise(op, _p(a), _p(b), _p(out), out.numel(), _s()))
    return out


class Conv:
    """One 3 x 3 x 3 convolution with FP32 master weights, a BF16 copy and Adam state."""

    def __init__(self, cin, cout, relu, rng):
        import torch
        self.cin, self.cout, self.relu = cin, cout, relu
        self.kp = lib().pl_nn_padded_k(cin)
        std = math.sqrt((2.0 if relu else 1.0) / (27 * cin))
        w = np.zeros((cout, self.kp), np.float32)
        w[:, :27 * cin] = rng.standard_normal((cout, 27 * cin)) * std
        self.w = torch.from_numpy(w).cuda()
        self.b = torch.zeros(cout, dtype=torch.float32, device="cuda")
        self.wb = self.w.to(torch.bfloat16)
        self.gw = torch.zeros_like(self.w)
        self.gb = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.wt = torch.empty((cin, lib().pl_nn_padded_k(cout)), dtype=torch.bfloat16,
                              device="cuda")

    def forward(self, x, dims, out_bf16=True):
        return conv3d(x, self.wb, self.b, dims, self.cin, self.cout, self.relu, out_bf16)

    def backward(self, gy, y, x, dims, need_gx=True):
        """gy: FP32 gradient of this layer's output y; x its BF16 input.
        Accumulates gw, gb; returns the FP32 gradient of x (or None)."""
        import torch
        gyb = torch.empty(gy.shape, dtype=torch.bfloat16, device="cuda")
        if self.relu:
            elementwise(0, gy, y, gyb)
        else:
            elementwise(1, gy, None, gyb)
        D, H, W = dims
        nbytes = lib().pl_nn_wgrad_workspace(D, H, W, self.cin, self.cout)
        work = torch.empty(nbytes // 4 + 1, dtype=torch.float32, device="cuda")
        B._check(lib().pl_nn_conv3d_wgrad(_p(x), _p(gyb), _p(self.gw), _p(self.gb), _p(work),
                                          nbytes, D, H, W, self.cin, self.cout, _s()))
        if not need_gx:
            return None
        B._check(lib().pl_nn_weight_flip(_p(self.wb), _p(self.wt), self.cin, self.cout, _s()))
        return conv3d(gyb, self.wt, None, dims, self.cout, self.cin, False, False)

    def params(self):
        return [(self.w, self.gw, self.mw, self.vw, self.wb), (self.b, self.gb, self.mb, self.vb, None)]


class UNet3D:
    """The encoder-decoder of the module docstring."""

    WIDTHS = (16, 32, 64, 128)

    def __init__(self, seed=0, widths=WIDTHS):
        rng = np.random.default_rng(seed)
        c1, c2, c3, c4 = widths
        self.widths = widths
        self.enc1 = [Conv(3, c1, True, rng), Conv(c1, c1, True, rng)]
        self.enc2 = [Conv(c1, c2, True, rng), Conv(c2, c2, True, rng)]
        self.enc3 = [Conv(c2, c3, True, rng), Conv(c3, c3, True, rng)]
        self.bott = [Conv(c3, c4, True, rng), Conv(c4, c4, True, rng)]
        self.dec3 = [Conv(c4, c3, True, rng), Conv(c3, c3, True, rng)]
        self.dec2 = [Conv(c3, c2, True, rng), Conv(c2, c2, True, rng)]
        self.dec1 = [Conv(c2, c1, True, rng), Conv(c1, c1, True, rng)]
        self.head = Conv(c1, 2, False, rng)
        # the head starts at zero: the prediction starts as the scaled cheap
        # image and training learns the correction
        self.head.w.zero_()
        self.head.wb.zero_()
        self.step_count = 0

    def layers(self):
        return (self.enc1 + self.enc2 + self.enc3 + self.bott + self.dec3 + self.dec2 + self.dec1
                + [self.head])

    # -- forward / backward ------------------------------------------------------
    def forward(self, feat, dims, keep=False):
        """feat: BF16 [V][3]; returns FP32 [V][2] (and the activations if keep)."""
        c1, c2, c3, c4 = self.widths
        d1 = dims
        d2 = tuple(n // 2 for n in d1)
        d3 = tuple(n // 2 for n in d2)
        d4 = tuple(n // 2 for n in d3)
        a = {}
        a["e1a"] = self.enc1[0].forward(feat, d1)
        a["s1"] = self.enc1[1].forward(a["e1a"], d1)
        a["p1"] = pool(a["s1"], d1, c1)
        a["e2a"] = self.enc2[0].forward(a["p1"], d2)
        a["s2"] = self.enc2[1].forward(a["e2a"], d2)
        a["p2"] = pool(a["s2"], d2, c2)
        a["e3a"] = self.enc3[0].forward(a["p2"], d3)
        a["s3"] = self.enc3[1].forward(a["e3a"], d3)
        a["p3"] = pool(a["s3"], d3, c3)
        a["b1"] = self.bott[0].forward(a["p3"], d4)
        a["b2"] = self.bott[1].forward(a["b1"], d4)
        a["u3"] = upsample(a["b2"], d4, c4)
        a["d3a"] = self.dec3[0].forward(a["u3"], d3)
        a["a3"] = elementwise(2, a["d3a"], a["s3"], a["d3a"].clone())
        a["d3"] = self.dec3[1].forward(a["a3"], d3)
        a["u2"] = upsample(a["d3"], d3, c3)
        a["d2a"] = self.dec2[0].forward(a["u2"], d2)
        a["a2"] = elementwise(2, a["d2a"], a["s2"], a["d2a"].clone())
        a["d2"] = self.dec2[1].forward(a["a2"], d2)
        a["u1"] = upsample(a["d2"], d2, c2)
        a["d1a"] = self.dec1[0].forward(a["u1"], d1)
        a["a1"] = elementwise(2, a["d1a"], a["s1"], a["d1a"].clone())
        a["d1"] = self.dec1[1].forward(a["a1"], d1)
        pred = self.head.forward(a["d1"], d1, out_bf16=False)
        if keep:
            a["feat"] = feat
            return pred, a
        return pred

    def backward(self, gpred, a, dims):
        """Accumulates every layer's gradients from gpred (FP32 [V][2])."""
        c1, c2, c3, c4 = self.widths
        d1 = dims
        d2 = tuple(n // 2 for n in d1)
        d3 = tuple(n // 2 for n in d2)
        d4 = tuple(n // 2 for n in d3)
        g = self.head.backward(gpred, None, a["d1"], d1)
        g_a1 = self.dec1[1].backward(g, a["d1"], a["a1"], d1)
        g_s1 = g_a1.clone()                                   # skip of a1 = d1a + s1
        g_u1 = self.dec1[0].backward(g_a1, a["d1a"], a["u1"], d1)
        g = upsample_bwd(g_u1, d2, c2)
        g_a2 = self.dec2[1].backward(g, a["d2"], a["a2"], d2)
        g_s2 = g_a2.clone()
        g_u2 = self.dec2[0].backward(g_a2, a["d2a"], a["u2"], d2)
        g = upsample_bwd(g_u2, d3, c3)
        g_a3 = self.dec3[1].backward(g, a["d3"], a["a3"], d3)
        g_s3 = g_a3.clone()
        g_u3 = self.dec3[0].backward(g_a3, a["d3a"], a["u3"], d3)
        g = upsample_bwd(g_u3, d4, c4)
        g = self.bott[1].backward(g, a["b2"], a["b1"], d4)
        g_p3 = self.bott[0].backward(g, a["b1"], a["p3"], d4)
        pool_bwd_accum(g_p3, g_s3, d3, c3)
        g = self.enc3[1].backward(g_s3, a["s3"], a["e3a"], d3)
        g_p2 = self.enc3[0].backward(g, a["e3a"], a["p2"], d3)
        pool_bwd_accum(g_p2, g_s2, d2, c2)
        g = self.enc2[1].backward(g_s2, a["s2"], a["e2a"], d2)
        g_p1 = self.enc2[0].backward(g, a["e2a"], a["p1"], d2)
        pool_bwd_accum(g_p1, g_s1, d1, c1)
        g = self.enc1[1].backward(g_s1, a["s1"], a["e1a"], d1)
        self.enc1[0].backward(g, a["e1a"], a["feat"], d1, need_gx=False)

    def zero_grad(self):
        for L in self.layers():
            L.gw.zero_()
            L.gb.zero_()

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for L in self.layers():
            for p, g, m, v, pb in L.params():
                B._check(lib().pl_nn_adam(_p(p), _p(g), _p(m), _p(v), _p(pb), p.numel(), lr, b1,
                                          b2, eps, self.step_count, _s()))

    # -- checkpoints -----------------------------------------------------------------
    def state(self):
        out = {"step": np.array(self.step_count), "widths": np.array(self.widths)}
        for i, L in enumerate(self.layers()):
            for name in ("w", "b", "mw", "vw", "mb", "vb"):
                out["%d_%s" % (i, name)] = getattr(L, name).cpu().numpy()
        return out

    def save(self, path):
        np.savez(path, **self.state())

    def load(self, path):
        import torch
        z = np.load(path)
        self.step_count = int(z["step"])
        for i, L in enumerate(self.layers()):
            for name in ("w", "b", "mw", "vw", "mb", "vb"):
                getattr(L, name).copy_(torch.from_numpy(z["%d_%s" % (i, name)]))
            L.wb.copy_(L.w.to(torch.bfloat16))


class FastPath:
    """Cheap reconstruction + network, with the full plain reconstruction as
    training target and fallback."""

    def __init__(self, workload, net=None, cheap_sigma=1.25, cheap_w=4):
        from . import workloads as wl
        self.w = workload
        self.full = B.Plan.from_workload(workload)
        cheap = wl.Workload(**{k: getattr(workload, k) for k in workload.__dataclass_fields__})
        cheap.f_hz = workload.f_hz[::2]
        self.cheap_w = cheap
        self.cheap = B.Plan.from_workload(cheap, nufft_sigma=cheap_sigma, nufft_w=cheap_w)
        self.gain = float(workload.f_hz.size) / float(cheap.f_hz.size)
        g = workload.grid
        self.dims = (g["nz"], g["ny"], g["nx"])
        self.V = g["nz"] * g["ny"] * g["nx"]
        self.net = net if net is not None else UNet3D()

    def cheap_echo(self, echo):
        return echo[:, :, ::2].contiguous()

    def features(self, img_cheap):
        import torch
        feat = torch.empty((self.V, 3), dtype=torch.bfloat16, device="cuda")
        scale = torch.empty(1, dtype=torch.float32, device="cuda")
        B._check(lib().pl_nn_features(_p(img_cheap), _p(feat), _p(scale), self.V, _s()))
        return feat, scale

    def train_step(self, echo, lr=1e-3):
        """One step on one scene; returns the (device) loss sums."""
        import torch
        full = self.full.execute(echo)
        cheap = self.cheap.execute(self.cheap_echo(echo))
        feat, scale = self.features(cheap)
        pred, acts = self.net.forward(feat, self.dims, keep=True)
        B._check(lib().pl_nn_residual(_p(pred), _p(cheap), _p(scale), self.gain, self.V, _s()))
        sums = torch.empty(2, dtype=torch.float32, device="cuda")
        grad = torch.empty_like(pred)
        B._check(lib().pl_nn_loss(_p(pred), _p(full), _p(scale), _p(sums), _p(grad), self.V, _s()))
        self.net.zero_grad()
        self.net.backward(grad, acts, self.dims)
        self.net.adam_step(lr)
        return sums

    def infer(self, echo_cheap, echo_full=None, max_correction=1.0):
        """Learned image (complex64 volume) from the cheap echo (every other
        frequency of the full echo, see cheap_echo).

        Returns (image, cheap image, fell_back). The network's correction is
        accepted only if it is finite and its L2 norm is at most
        max_correction times that of the scaled cheap image it is added to
        (pl_nn_check). Otherwise the plain reconstruction of echo_full, the
        full echo, is returned with fell_back = True; without echo_full a
        rejected correction raises RuntimeError."""
        import torch
        cheap = self.cheap.execute(echo_cheap)
        feat, scale = self.features(cheap)
        pred = self.net.forward(feat, self.dims)
        stats = torch.empty(3, dtype=torch.float32, device="cuda")
        B._check(lib().pl_nn_check(_p(pred), _p(cheap), _p(scale), self.gain, self.V, _p(stats),
                                   _s()))
        bad, corr2, base2 = (float(v) for v in stats.cpu())
        if bad > 0 or not math.isfinite(corr2) or corr2 > max_correction ** 2 * base2:
            if echo_full is None:
                raise RuntimeError("learned correction rejected (%d non-finite values, "
                                   "|corr|^2 = %.3e vs %.3e) and no full echo to fall back on"
                                   % (bad, corr2, max_correction ** 2 * base2))
            return self.full.execute(echo_full).view(self.dims), cheap, True
        B._check(lib().pl_nn_residual(_p(pred), _p(cheap), _p(scale), self.gain, self.V, _s()))
        img = torch.empty(self.V, dtype=torch.complex64, device="cuda")
        B._check(lib().pl_nn_to_complex(_p(pred), _p(scale), _p(img), self.V, _s()))
        return img.view(self.dims), cheap, False
