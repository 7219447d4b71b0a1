"""Learned fast path on the GPU, through the C ABI (pl_nn_*): every layer's
forward and backward kernels against the CPU oracle (oracle/nn_oracle.py),
the whole network's gradients against the oracle's layers composed the same
way, checkpoint round trip, and a short training run showing what the
network gains over the cheap reconstruction without it."""
import math

import numpy as np
import pytest

from oracle import nn_oracle as nn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2109_02842_gb300 import build, binding
    build.build()
    binding.load()
    from paper_2109_02842_gb300 import learned
    learned.lib()
    return learned


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def to_dev_bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def pack_w(w, kp):
    """oracle w[co][tap][ci] -> kernel layout [co][kp]"""
    co, taps, ci = w.shape
    out = np.zeros((co, kp), np.float32)
    out[:, :taps * ci] = w.reshape(co, taps * ci)
    return out


# the mma.sync kernel (odd sizes, 3 input or 2 output channels) and the
# tcgen05 kernel (Cin a multiple of 16, Cout 16..128, rows of 16..128 voxels
# with 128 / W dividing H: the shapes of the network at full size; their input
# gradients, convolutions with swapped channel roles, take it too)
@pytest.mark.parametrize("dims,cin,cout", [((5, 6, 7), 3, 16), ((4, 5, 9), 16, 2),
                                           ((8, 8, 8), 16, 32), ((6, 4, 4), 32, 64),
                                           ((4, 4, 4), 64, 128), ((16, 16, 17), 16, 16),
                                           ((4, 8, 16), 16, 16), ((3, 4, 32), 32, 64),
                                           ((2, 2, 64), 64, 128), ((2, 1, 128), 128, 64),
                                           ((5, 16, 16), 16, 32), ((2, 8, 16), 128, 32),
                                           ((4, 8, 16), 16, 2), ((2, 4, 32), 32, 5)])
def test_conv3d_forward_and_gradients(L, dims, cin, cout):
    rng = np.random.default_rng(cin * 1000 + cout)
    x = bf16_round(rng.standard_normal(dims + (cin,)))
    w = bf16_round(rng.standard_normal((cout, 27, cin)) / math.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    gy = bf16_round(rng.standard_normal(dims + (cout,)))
    kp = L.lib().pl_nn_padded_k(cin)
    xd, wd = to_dev_bf16(x.reshape(-1, cin)), to_dev_bf16(pack_w(w, kp))
    bd = torch.from_numpy(b).cuda()
    D, H, W = dims
    y = L.conv3d(xd, wd, bd, dims, cin, cout, False, False).cpu().numpy()
    assert rel(y, nn.conv3d(x, w, b).reshape(-1, cout)) < 1e-5
    yr = L.conv3d(xd, wd, bd, dims, cin, cout, True, False).cpu().numpy()
    assert rel(yr, nn.relu(nn.conv3d(x, w, b)).reshape(-1, cout)) < 1e-5
    # gradients of sum(gy * conv(x)) (linear layer)
    conv = L.Conv(cin, cout, False, rng)
    conv.w.copy_(torch.from_numpy(pack_w(w, kp)))
    conv.wb.copy_(wd)
    gx = conv.backward(torch.from_numpy(gy.reshape(-1, cout)).cuda(), None, xd, dims)
    rgx, rgw, rgb = nn.conv3d_backward(x, w, gy)
    assert rel(gx.cpu().numpy(), rgx.reshape(-1, cin)) < 1e-5
    gw = conv.gw.cpu().numpy()[:, :27 * cin].reshape(cout, 27, cin)
    assert rel(gw, rgw) < 1e-5
    assert rel(conv.gb.cpu().numpy(), rgb) < 1e-5


def test_pool_upsample_and_their_adjoints(L):
    rng = np.random.default_rng(7)
    dims, c = (4, 6, 8), 16
    x = bf16_round(rng.standard_normal(dims + (c,)))
    y = L.pool(to_dev_bf16(x.reshape(-1, c)), dims, c).float().cpu().numpy()
    assert rel(y, bf16_round(nn.avgpool2(x)).reshape(-1, c)) < 4e-3
    small = tuple(n // 2 for n in dims)
    gy = rng.standard_normal(small + (c,)).astype(np.float32)
    gx = torch.zeros(int(np.prod(dims)), c, device="cuda")
    L.pool_bwd_accum(torch.from_numpy(gy.reshape(-1, c)).cuda(), gx, dims, c)
    assert rel(gx.cpu().numpy(), (nn.upsample2(gy) / 8).reshape(-1, c)) < 1e-6
    z = bf16_round(rng.standard_normal(small + (c,)))
    u = L.upsample(to_dev_bf16(z.reshape(-1, c)), small, c).float().cpu().numpy()
    assert np.array_equal(u, nn.upsample2(z).reshape(-1, c).astype(np.float32))
    gu = rng.standard_normal(dims + (c,)).astype(np.float32)
    gz = L.upsample_bwd(torch.from_numpy(gu.reshape(-1, c)).cuda(), small, c).cpu().numpy()
    assert rel(gz, (8 * nn.avgpool2(gu)).reshape(-1, c)) < 1e-6


def test_features_loss_adam(L):
    from paper_2109_02842_gb300 import binding as B
    rng = np.random.default_rng(8)
    n = 3000
    g = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    gd = torch.from_numpy(g).cuda()
    feat = torch.empty((n, 3), dtype=torch.bfloat16, device="cuda")
    scale = torch.empty(1, device="cuda")
    B._check(L.lib().pl_nn_features(L._p(gd), L._p(feat), L._p(scale), n, L._s()))
    rf, rs = nn.features(g.astype(np.complex128))
    assert abs(scale.item() - rs) < 1e-6 * rs
    assert np.abs(feat.float().cpu().numpy() - rf.reshape(n, 3)).max() < 4e-3
    pred = rng.standard_normal((n, 2)).astype(np.float32)
    pd = torch.from_numpy(pred).cuda()
    sums = torch.empty(2, device="cuda")
    grad = torch.empty_like(pd)
    B._check(L.lib().pl_nn_loss(L._p(pd), L._p(gd), L._p(scale), L._p(sums), L._p(grad), n,
                                L._s()))
    t = np.stack([g.real, g.imag], 1) / rs
    loss, rgrad = nn.rel_l2_loss(pred, t)
    assert abs(sums[1].item() / sums[0].item() - loss) < 1e-5 * loss
    assert rel(grad.cpu().numpy(), rgrad) < 1e-5
    p = rng.standard_normal(100).astype(np.float32)
    gr = rng.standard_normal(100).astype(np.float32)
    P, G = torch.from_numpy(p).cuda(), torch.from_numpy(gr).cuda()
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    rp, rm, rv = p.astype(np.float64), np.zeros(100), np.zeros(100)
    for step in (1, 2, 3):
        B._check(L.lib().pl_nn_adam(L._p(P), L._p(G), L._p(M), L._p(V), None, 100, 1e-2, 0.9,
                                    0.999, 1e-8, step, L._s()))
        rp, rm, rv = nn.adam(rp, gr, rm, rv, step, 1e-2)
    assert rel(P.cpu().numpy(), rp) < 1e-6
    out = pd.clone()
    B._check(L.lib().pl_nn_residual(L._p(out), L._p(gd), L._p(scale), 2.0, n, L._s()))
    assert rel(out.cpu().numpy(), pred + 2.0 * np.stack([g.real, g.imag], 1) / rs) < 1e-6


def test_correction_check_kernel(L):
    # pl_nn_check against NumPy: non-finite count, sum of squares of the
    # finite correction entries, and of the scaled cheap image
    from paper_2109_02842_gb300 import binding as B
    rng = np.random.default_rng(21)
    n = 5000
    corr = rng.standard_normal((n, 2)).astype(np.float32)
    corr[17, 1] = np.nan
    corr[4000, 0] = np.inf
    img = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    scale = torch.tensor([2.5], device="cuda")
    out = torch.empty(3, device="cuda")
    corr_d, img_d = torch.from_numpy(corr).cuda(), torch.from_numpy(img).cuda()
    B._check(L.lib().pl_nn_check(L._p(corr_d), L._p(img_d), L._p(scale), 2.0, n, L._p(out),
                                 L._s()))
    got = out.cpu().numpy().astype(np.float64)
    fin = np.isfinite(corr)
    assert got[0] == 2
    assert abs(got[1] - np.sum(corr[fin].astype(np.float64) ** 2)) < 1e-5 * got[1]
    ref_i = np.sum(np.abs(2.0 * img.astype(np.complex128) / 2.5) ** 2)
    assert abs(got[2] - ref_i) < 1e-5 * ref_i


def _oracle_unet(net, feat, target_over_s):
    """Forward + backward of the same network with the oracle's layers (FP64)."""
    def W(conv):
        return conv.w.cpu().numpy()[:, :27 * conv.cin].reshape(conv.cout, 27, conv.cin).astype(np.float64)

    def Bv(conv):
        return conv.b.cpu().numpy().astype(np.float64)

    c = {}
    acts = {}

    def fwd(name, conv, x):
        z = nn.conv3d(x, W(conv), Bv(conv))
        y = nn.relu(z) if conv.relu else z
        c[name] = (conv, x, z)
        return y

    e1a = fwd("e1a", net.enc1[0], feat)
    s1 = fwd("s1", net.enc1[1], e1a)
    e2a = fwd("e2a", net.enc2[0], nn.avgpool2(s1))
    s2 = fwd("s2", net.enc2[1], e2a)
    e3a = fwd("e3a", net.enc3[0], nn.avgpool2(s2))
    s3 = fwd("s3", net.enc3[1], e3a)
    b1 = fwd("b1", net.bott[0], nn.avgpool2(s3))
    b2 = fwd("b2", net.bott[1], b1)
    d3a = fwd("d3a", net.dec3[0], nn.upsample2(b2))
    d3 = fwd("d3", net.dec3[1], d3a + s3)
    d2a = fwd("d2a", net.dec2[0], nn.upsample2(d3))
    d2 = fwd("d2", net.dec2[1], d2a + s2)
    d1a = fwd("d1a", net.dec1[0], nn.upsample2(d2))
    d1 = fwd("d1", net.dec1[1], d1a + s1)
    pred = fwd("pred", net.head, d1)
    loss, gp = nn.rel_l2_loss(pred, target_over_s)
    grads = {}

    def bwd(name, gy):
        conv, x, z = c[name]
        if conv.relu:
            gy = gy * (z > 0)
        gx, gw, gb = nn.conv3d_backward(x, W(conv), gy)
        grads[id(conv)] = (gw, gb)
        return gx

    g_a1 = bwd("d1", bwd("pred", gp))
    g_s1 = g_a1.copy()
    g = nn.avgpool2(bwd("d1a", g_a1)) * 8
    g_a2 = bwd("d2", g)
    g_s2 = g_a2.copy()
    g = nn.avgpool2(bwd("d2a", g_a2)) * 8
    g_a3 = bwd("d3", g)
    g_s3 = g_a3.copy()
    g = nn.avgpool2(bwd("d3a", g_a3)) * 8
    g = bwd("b1", bwd("b2", g))
    g_s3 = g_s3 + nn.upsample2(g) / 8
    g = bwd("e3a", bwd("s3", g_s3))
    g_s2 = g_s2 + nn.upsample2(g) / 8
    g = bwd("e2a", bwd("s2", g_s2))
    g_s1 = g_s1 + nn.upsample2(g) / 8
    bwd("e1a", bwd("s1", g_s1))
    return loss, grads


@pytest.mark.parametrize("widths", [(4, 8, 16, 16), (16, 32, 64, 128)])
def test_network_gradients_match_oracle(L, widths):
    # (16, 32, 64, 128): the widths of the learned fast path itself
    from paper_2109_02842_gb300 import binding as B
    dims = (8, 8, 16)
    net = L.UNet3D(seed=3, widths=widths)
    rng = np.random.default_rng(9)
    # the head starts at zero (no gradient would reach the other layers)
    hw = np.zeros(tuple(net.head.w.shape), np.float32)
    hw[:, :27 * net.head.cin] = rng.standard_normal((2, 27 * net.head.cin)) * 0.1
    net.head.w.copy_(torch.from_numpy(hw))
    net.head.wb.copy_(net.head.w.to(torch.bfloat16))
    feat = bf16_round(rng.standard_normal(dims + (3,)) * 0.5)
    g = (rng.standard_normal(dims) + 1j * rng.standard_normal(dims)).astype(np.complex64)
    scale = torch.tensor([1.0], device="cuda")
    pred, acts = net.forward(to_dev_bf16(feat.reshape(-1, 3)), dims, keep=True)
    V = int(np.prod(dims))
    sums = torch.empty(2, device="cuda")
    grad = torch.empty_like(pred)
    gd = torch.from_numpy(g.reshape(-1)).cuda()
    B._check(L.lib().pl_nn_loss(L._p(pred), L._p(gd), L._p(scale), L._p(sums), L._p(grad), V,
                                L._s()))
    net.zero_grad()
    net.backward(grad, acts, dims)
    loss, ref = _oracle_unet(net, feat.astype(np.float64), np.stack([g.real, g.imag], -1))
    assert abs(sums[1].item() / sums[0].item() - loss) < 0.02 * loss
    for conv in net.layers():
        gw, gb = ref[id(conv)]
        got = conv.gw.cpu().numpy()[:, :27 * conv.cin].reshape(gw.shape)
        cos = float(np.sum(got * gw) / (np.linalg.norm(got) * np.linalg.norm(gw) + 1e-30))
        # BF16 activations between layers: directions agree, magnitudes within a few %
        assert cos > 0.99, (conv.cin, conv.cout, cos)
        assert rel(got, gw) < 0.1, (conv.cin, conv.cout, rel(got, gw))


def _small_fastpath(L):
    from paper_2109_02842_gb300 import workloads as wl
    w = wl.small_mono(seed=0)
    w.f_hz = np.linspace(28e9, 33e9, 32)
    x0, dx = wl.centred_axis(0.2, 32)
    w.grid = dict(x0=x0, dx=dx, nx=32, y0=x0, dy=dx, ny=32, z0=x0, dz=0.2 / 16, nz=16)
    return L.FastPath(w, net=L.UNet3D(seed=1, widths=(8, 16, 32, 32)))


def _scene_echo(fp, seed):
    from paper_2109_02842_gb300 import binding as B, workloads as wl
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 8))
    w = fp.w
    pts = wl.uniform_points(rng, (-0.08, -0.08, w.z_scan[0]), (0.08, 0.08, w.z_scan[-1]), n)
    amp = rng.uniform(0.5, 1.0, n)
    return B.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, pts, amp)


def test_checkpoint_round_trip(L, tmp_path):
    fp = _small_fastpath(L)
    echo = _scene_echo(fp, 0)
    fp.train_step(echo)
    path = str(tmp_path / "ckpt.npz")
    fp.net.save(path)
    other = L.UNet3D(seed=99, widths=(8, 16, 32, 32))
    other.load(path)
    fp2 = _small_fastpath(L)
    fp2.net = other
    fp.train_step(echo)
    fp2.train_step(echo)
    for a, b in zip(fp.net.layers(), other.layers()):
        assert torch.equal(a.w, b.w) and torch.equal(a.b, b.b)


def test_training_beats_the_cheap_reconstruction(L):
    """After a short training run on generated scenes, on held-out scenes the
    network's image is clearly closer to the full reconstruction than the
    cheap reconstruction is, even with the cheap image's best scalar scaling."""
    fp = _small_fastpath(L)
    steps = 600
    for step in range(1, steps + 1):
        lr = 1e-3 * 0.5 * (1 + math.cos(math.pi * step / steps))
        fp.train_step(_scene_echo(fp, 1000 + step), lr=lr)
    e_net, e_cheap = [], []
    for s in range(8):
        echo = _scene_echo(fp, 50000 + s)
        full = fp.full.execute(echo).cpu().numpy().ravel()
        img, cheap, fell_back = fp.infer(fp.cheap_echo(echo), echo)
        assert not fell_back
        img, cheap = img.cpu().numpy().ravel(), cheap.cpu().numpy().ravel()
        a = np.vdot(cheap, full) / np.vdot(cheap, cheap)
        e_cheap.append(rel(a * cheap, full))
        e_net.append(rel(img, full))
    print("held-out rel L2 vs full: network %.3f, cheap (best-scaled) %.3f"
          % (np.mean(e_net), np.mean(e_cheap)))
    assert np.mean(e_net) < 0.85 * np.mean(e_cheap)


def test_rejected_correction_falls_back_to_the_plain_image(L):
    """The plain hybrid method stays the fallback: a network whose correction
    is non-finite (a NaN written into the head's bias on the host side) or
    implausibly large (a huge head bias) returns the full plain image, the
    same bits as the plain path's own execution."""
    fp = _small_fastpath(L)
    echo = _scene_echo(fp, 3)
    full = fp.full.execute(echo).cpu().numpy()
    img, _, fell_back = fp.infer(fp.cheap_echo(echo), echo)
    assert not fell_back                       # zero head: no correction yet
    for bad in (float("nan"), 1e6):
        b = np.zeros(2, np.float32)
        b[0] = bad
        fp.net.head.b.copy_(torch.from_numpy(b))
        img, _, fell_back = fp.infer(fp.cheap_echo(echo), echo)
        assert fell_back
        assert np.array_equal(img.cpu().numpy(), full)
        with pytest.raises(RuntimeError):
            fp.infer(fp.cheap_echo(echo))
