"""Reconstruct one synthetic workload a few times on cuda:0 and print the plan
and per-stage times: a quick check and the driver the committed profiles are
captured with.

    python -m paper_2109_02842_gb300.run --workload full_mono [--block-config 4]
        [--precision 0] [--tile-u 0] [--repeat 4]
    python -m paper_2109_02842_gb300.run --workload batch64 [--repeat 2]
        (the 64 uneven scenes of the batched workload, default batch options)
    python -m paper_2109_02842_gb300.run --workload conv:CIN:COUT [--repeat 10]
        (one learned-path convolution on 96 x 128 x 128 voxels)
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="full_mono")
    ap.add_argument("--block-config", type=int, default=0)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--tile-u", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=4)
    a = ap.parse_args(argv)

    import torch
    from . import binding, build, workloads as wl
    build.build()
    binding.load()
    if a.workload.startswith("conv"):
        # one learned-path convolution layer on 96 x 128 x 128 voxels:
        # --workload conv:CIN:COUT
        from . import learned as L
        _, cin, cout = a.workload.split(":")
        cin, cout = int(cin), int(cout)
        D, H, W = 96, 128, 128
        L.lib()
        x = torch.randn(D * H * W, cin, device="cuda").to(torch.bfloat16)
        kp = L.lib().pl_nn_padded_k(cin)
        wt = (torch.randn(cout, kp, device="cuda") * 0.05).to(torch.bfloat16)
        bias = torch.zeros(cout, device="cuda")
        for _ in range(3):
            L.conv3d(x, wt, bias, (D, H, W), cin, cout, True, True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(a.repeat):
            L.conv3d(x, wt, bias, (D, H, W), cin, cout, True, True)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / a.repeat
        print(json.dumps({"workload": a.workload, "ms": ms,
                          "tflops": 2 * D * H * W * 27 * cin * cout / ms / 1e9}))
        return
    if a.workload == "batch64-stages":
        # the 64 scenes one after another through their own plans, with the
        # per-stage CUDA-event times summed over the scenes
        tot, rows = {}, []
        for i in range(64):
            w = wl.batch_scene(i)
            e = binding.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.pts, w.amp)
            plan = binding.Plan.from_workload(w, block_config=a.block_config,
                                              precision=a.precision)
            img = plan.execute(e)
            plan.set_timing(True)
            for _ in range(a.repeat):
                plan.execute(e, img)
            torch.cuda.synchronize()
            t = {k: v[0] / max(v[1], 1) for k, v in plan.stage_times().items()}
            for k, v in t.items():
                tot[k] = tot.get(k, 0.0) + v
            inf = plan.info
            rows.append({"scene": i, "C": w.n_chan, "Np": w.n_pad, "M": w.n_f,
                         "grid": w.grid["nx"], "exact": inf["table_exact"],
                         "tile_u": inf["tile_u"], "rows": inf["slab_rows"],
                         "layout": inf["table_layout"], "zfft_inv": inf["z_transform_fft"],
                         "ms": t})
            plan.close()
        print(json.dumps({"workload": "batch64-stages", "total_ms": tot, "scenes": rows}))
        return
    if a.workload == "batch64":
        scenes = [wl.batch_scene(i) for i in range(64)]
        echos = [binding.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.pts, w.amp)
                 for w in scenes]
        b = binding.Batch(scenes, block_config=a.block_config, tile_u=a.tile_u,
                          precision=a.precision)
        imgs = b.execute(echos)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(max(a.repeat - 1, 0)):
            b.execute(echos, imgs)
        ev[1].record()
        torch.cuda.synchronize()
        print(json.dumps({"workload": "batch64", "info": b.get_info(),
                          "ms_per_batch": ev[0].elapsed_time(ev[1]) / max(a.repeat - 1, 1)}))
        b.close()
        return
    w = wl.WORKLOADS[a.workload](seed=0)
    echo = binding.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.pts, w.amp)
    plan = binding.Plan.from_workload(w, block_config=a.block_config, precision=a.precision,
                                      tile_u=a.tile_u)
    img = plan.execute(echo)
    plan.set_timing(True)
    for _ in range(max(a.repeat - 1, 0)):
        plan.execute(echo, img)
    torch.cuda.synchronize()
    t = plan.stage_times()
    info = plan.info
    print(json.dumps({"workload": w.name, "block_config": info["block_config"],
                      "tile_u": info["tile_u"], "table_len": info["table_len"],
                      "stage_ms": {k: v[0] / max(v[1], 1) for k, v in t.items()}}))
    plan.close()


if __name__ == "__main__":
    main()
