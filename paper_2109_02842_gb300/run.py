"""Reconstruct one synthetic workload a few times on cuda:0 and print the plan
and per-stage times: a quick check and the driver the committed profiles are
captured with.

    python -m paper_2109_02842_gb300.run --workload full_mono [--block-config 4]
        [--precision 0] [--tile-u 0] [--repeat 4]
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
