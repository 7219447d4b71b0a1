"""Train and evaluate the learned fast path on generated scenes.

    python -m paper_2109_02842_gb300.train_fastpath [--scenes 2000] [--eval 200]
           [--out fastpath.npz] [--json summary.json]

Workload (the cheap/full pair of learned.py): the 4-chord x 16-element array
of R = 0.5 m over 60 deg, 32 scans at 5 mm, 64 frequencies 28-33 GHz (the
cheap reconstruction takes every other one, NUFFT oversampling 1.25, 4 taps),
128 x 128 x 96 voxels over the 0.2 m cube. Scenes: 3-30 seeded points in the
cube within the scan span, amplitudes U(0.5, 1), 30 dB noise. Training scene
i uses seed i, evaluation scene j seed 1_000_000 + j (disjoint). Each training
scene is reconstructed by the plain method (cheap and full) on the GPU and used
for one step. Evaluation reports, on the held-out scenes, the relative L2
error against the full plain reconstruction of (a) the network, (b) the cheap
reconstruction with its best scalar scaling, and the time of the learned path
(cheap reconstruction + network) against the full plain reconstruction.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def fastpath_workload():
    from . import workloads as wl
    w = wl.small_mono(seed=0)
    w.f_hz = np.linspace(28e9, 33e9, 64)
    x0, dx = wl.centred_axis(0.2, 128)
    z0, dz = wl.centred_axis(0.2, 96)
    w.grid = dict(x0=x0, dx=dx, nx=128, y0=x0, dy=dx, ny=128, z0=z0, dz=dz, nz=96)
    return w


def scene_echo(w, seed, snr_db=30.0):
    import torch
    from . import binding as B, workloads as wl
    rng = wl.rng_for(5, seed)
    n = int(rng.integers(3, 31))
    pts = wl.uniform_points(rng, (-0.09, -0.09, w.z_scan[0]), (0.09, 0.09, w.z_scan[-1]), n)
    amp = rng.uniform(0.5, 1.0, n)
    e = B.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, pts, amp)
    if snr_db is not None:
        p = float(torch.mean(e.abs() ** 2))
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        e += math.sqrt(p * 10 ** (-snr_db / 10)) * torch.randn(e.shape, dtype=torch.complex64,
                                                               device="cuda", generator=g)
    return e


def evaluate(fp, n_eval, first_seed=1_000_000):
    import torch
    en, ec = [], []
    for j in range(n_eval):
        e = scene_echo(fp.w, first_seed + j)
        full = fp.full.execute(e)
        img, cheap, _ = fp.infer(fp.cheap_echo(e), e)
        f, i, c = (x.reshape(-1) for x in (full, img, cheap))
        a = torch.vdot(c, f) / torch.vdot(c, c)
        ec.append(float((a * c - f).norm() / f.norm()))
        en.append(float((i - f).norm() / f.norm()))
    return float(np.mean(en)), float(np.mean(ec)), float(np.max(en))


def time_paths(fp, reps=20):
    import torch
    e = scene_echo(fp.w, 7)
    ec = fp.cheap_echo(e)
    out = fp.full.execute(e)
    fp.infer(ec, e)
    torch.cuda.synchronize()

    def timed(fn):
        s, t = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            fn()
        t.record()
        torch.cuda.synchronize()
        return s.elapsed_time(t) / reps

    t_full = timed(lambda: fp.full.execute(e, out))
    t_learned = timed(lambda: fp.infer(ec, e))
    t_cheap = timed(lambda: fp.cheap.execute(ec))
    return t_full, t_learned, t_cheap


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=None)
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    import torch
    from . import binding as B, build, learned as L
    build.build()
    B.load()
    L.lib()
    fp = L.FastPath(fastpath_workload(), net=L.UNet3D(seed=0))
    e0 = evaluate(fp, min(args.eval, 20))
    t0 = time.time()
    losses = []
    for i in range(args.scenes):
        lr = args.lr * 0.5 * (1 + math.cos(math.pi * (i + 1) / args.scenes))
        sums = fp.train_step(scene_echo(fp.w, i), lr=lr)
        if (i + 1) % 100 == 0:
            s = sums.cpu().numpy()
            losses.append((i + 1, float(s[1] / s[0])))
            print("step %d loss %.5f (%.1f s)" % (i + 1, s[1] / s[0], time.time() - t0), flush=True)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    e_net, e_cheap, e_max = evaluate(fp, args.eval)
    t_full, t_learned, t_cheap = time_paths(fp)
    summary = {
        "workload": "mono-4x16-32scan-64f-128x128x96 (cheap: 32 f, sigma 1.25, w 4)",
        "train_scenes": args.scenes, "eval_scenes": args.eval, "train_seconds": t_train,
        "ms_per_train_step": 1e3 * t_train / max(args.scenes, 1),
        "loss_curve": losses,
        "before_training": {"rel_l2_network": e0[0], "rel_l2_cheap_best_scaled": e0[1]},
        "rel_l2_network_vs_full": e_net, "rel_l2_network_max": e_max,
        "rel_l2_cheap_best_scaled_vs_full": e_cheap,
        "ms_full_plain": t_full, "ms_learned_path": t_learned, "ms_cheap_plain": t_cheap,
        "speedup_learned_over_full": t_full / t_learned,
    }
    print(json.dumps(summary), flush=True)
    if args.out:
        fp.net.save(args.out)
    if args.json:
        with open(args.json, "w") as f:
            json.dump(summary, f, indent=1)


if __name__ == "__main__":
    main()
