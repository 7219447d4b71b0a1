"""Benchmark of the polyline-array hybrid reconstruction on GB300.

One step = one full reconstruction of one scan (z-FFT, NUFFT range table,
back-projection with the coherent channel sum, z inverse FFT) of the
full-size monostatic workload: 8 chords of R = 0.6 m over 120 deg with 48
elements each (384), 200 scans at 5 mm, 64 frequencies 24-34 GHz,
256 x 256 x 200 voxels; elliptic-cylinder scene of 2000 + 20 points, 30 dB.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. `value` = element-voxel-frequency updates per second
(C * Nx * Ny * Nz * M per scan) with inputs resident in HBM, timed with CUDA
events on the launch stream; `e2e` = the same through pl_execute_host_stream
over K scans with pinned host buffers (every scan's upload and download inside
the timed call, overlapped with the reconstruction of its neighbours), with
the latency of a single pl_execute_host call beside it. For N > 1 (torchrun)
each rank reconstructs its own scans (independent replicas, no collective on
the data path); `value` is the sum over ranks over the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0
MUFU_PER_SM_CLK = 16
# the metric of both arms (the reference arm times the FP64 oracle on it)
METRIC = "element-voxel-freq updates/s at rel. L2 err <= 1e-3 vs FP64 oracle"
CLOCK_QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--workload", default="full_mono",
                    choices=["full_mono", "multi", "batch64", "table2"],
                    help="full_mono (default), multi, batch64 (64 uneven scenes), or table2 "
                         "(Table I geometry: the method vs the exact sum vs direct BP)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of the kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(kernel, {})
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_2109_02842_gb300", "csrc", d.get("source", "x"))
    if not os.path.exists(src) or d.get("workload") != workload:
        return None
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    return d.get("bytes_per_launch") if sha == d.get("sha1") else None


class ClockSampler:
    """nvidia-smi clock / throttle samples (every 20 ms) during the timed
    region: samples stamped outside [t_begin, t_end] (host wall clock) are
    dropped."""

    def __init__(self, index: int, path: str):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + CLOCK_QUERY,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)          # nvidia-smi is polling before the region starts
        except Exception:
            self.proc = None

    def stop(self, t_begin: float, t_end: float):
        """Median SM clock and throttle reasons over the samples stamped in
        [t_begin, t_end] (time.time() values)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        total = 0
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                stamp = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                stamp += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                clk, clk_max = float(parts[2]), float(parts[3])
            except (ValueError, IndexError):
                continue
            total += 1
            if not (t_begin - 0.02 <= stamp <= t_end + 0.02):
                continue
            sm.append(clk)
            smax.append(clk_max)
            for n, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "samples_outside_region": total - len(sm), "interval_ms": 20}


def dtype_of(info: dict, precision: int) -> str:
    if info["block_config"] == 4:
        return ("bf16x3+f32acc", "bf16+f32acc", "bf16+f32acc,bf16-spectrum")[precision]
    return ("f32", "f32+bf16-table", "f32+bf16-table+bf16-spectrum")[precision]


def tc_flops_per_launch(info: dict, precision: int) -> float:
    """Dense BF16 flops of one tensor-core back-projection launch: per (pixel,
    channel, bin) 16 ks window rows x 2 columns (re, im) x 2 accumulators
    (Re A, Im A) x split products (3 with the hi/lo split, 1 in BF16), over
    16 x 8 pixel tiles and whole tile_u-bin blocks (the padding is executed)."""
    ks = max(info["slab_rows"] // 16, 1)
    split = 3 if precision == 0 else 1
    ut = info["tile_u"]
    bins = -(-info["n_pad"] // ut) * ut
    pix = -(-info["nx"] // 16) * 16 * (-(-info["ny"] // 8) * 8)
    return 2.0 * pix * info["n_chan"] * bins * 4 * split * 16 * ks


# the method's work per (pixel, channel, k_z bin) update of the back-projection
# at w = 6 taps: 2w FMA for the interpolation, ~8 FMA for the split-float
# carrier phase and its reduction, 4 FMA for the complex multiply-accumulate,
# i.e. 24 FMA = 48 flop
METHOD_FLOP_PER_UPDATE = 48


def measure_unit_peaks(binding) -> dict:
    """FP32 FMA, MUFU sine and shared-memory peaks measured on this device
    (pl_measure_peak), or {} if the call fails."""
    try:
        return {"fp32_tflops": binding.measure_peak(0), "mufu_gsin": binding.measure_peak(1),
                "smem_gbs": binding.measure_peak(2), "source": "pl_measure_peak, this run"}
    except Exception as e:          # reported, not fatal for the bench line
        return {"error": str(e)}


def backproject_flops_per_update(w_taps: int) -> int:
    # w complex-by-real MACs (4w flop) + complex multiply-accumulate by the
    # carrier (8); the carrier's phase and sine/cosine pair are formed once per
    # (pixel, channel) and shared by the block's bins.
    return 4 * w_taps + 8


def oracle_baseline(w, echo_np, gpu_image=None, n_cols=256, n_chan=None, seed=1):
    """Time the FP64 oracle on a bounded sample -- P sampled (x, y) columns x
    all z, optionally over the first n_chan channels only -- and scale to the
    metric's unit; optionally return the GPU image's error on those columns
    (only when every channel is used)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    P = w.grid["nx"] * w.grid["ny"]
    C = w.n_chan
    cs = C if n_chan is None else min(n_chan, C)
    idx = np.sort(rng.choice(P, size=min(n_cols, P), replace=False))
    pix = w.pix_xy()[idx]
    t0 = time.perf_counter()
    S = oracle.zdft(echo_np[:cs], w.n_pad)
    t1 = time.perf_counter()
    G = oracle.hybrid_spectral(w.mode, w.tx_xy[:cs], w.rx_xy[:cs], S, w.dz, w.f_hz, pix)
    g = oracle.zidft(G, w.dz, w.z0, w.axis("z"))
    t2 = time.perf_counter()
    # full-scan time: z-DFT over all channels + per-column work over all columns
    t_full = (t1 - t0) * C / cs + (t2 - t1) * (C / cs) * (P / idx.size)
    upd = w.updates_per_scan()
    out = {"value": upd / t_full, "unit": "updates/s", "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": "FP64 exact-sum hybrid on %d of %d channels: z-DFT (%.2f s) + %d of %d "
                     "(x,y) columns x all %d z (%.2f s), scaled to the full scan" %
                     (cs, C, t1 - t0, idx.size, P, w.grid["nz"], t2 - t1),
           "seconds": t2 - t0}
    err = None
    if gpu_image is not None and cs == C:
        err = column_error(gpu_image, w, idx, g)
    return out, err, (idx, g)


def column_error(image, w, idx, ref):
    """Relative L2 and largest per-voxel error of an image's sampled columns
    against the oracle's values there."""
    import numpy as np
    got = image.reshape(w.grid["nz"], -1)[:, idx]
    return {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_abs_over_max_ref": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
            "columns": int(idx.size)}


def max_over_ranks(values, world: int, device):
    """The per-rank floats reduced to their maximum over all ranks (the
    slowest rank's times); unchanged for one rank."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank processes its own units)."""
    return world * units_per_rank / seconds


def workload_config(w, world, precision, l2):
    """The `config` of both arms: the workload's name and sizes, the options
    and how the timing treats the L2 cache."""
    return {"workload": w.name, "mode": "monostatic" if w.mode == 0 else "multistatic",
            "n_chan": int(w.n_chan), "n_scan": int(w.n_scan), "n_f": int(w.n_f),
            "grid": [w.grid["nx"], w.grid["ny"], w.grid["nz"]], "n_pad": int(w.n_pad),
            "precision": ("fp32", "bf16-table", "bf16-table+spectrum")[precision],
            "nufft_w": 6, "nufft_sigma": 2.0,
            "parallelism": "replicas%d" % world, "l2": l2}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2109_02842_gb300 import workloads as wl
    oracle.build()
    w = wl.full_mono(seed=0)
    rng = np.random.default_rng(7)
    echo = (rng.standard_normal((w.n_chan, w.n_scan, w.n_f)) +
            1j * rng.standard_normal((w.n_chan, w.n_scan, w.n_f)))
    for _ in range(args.warmup):
        oracle_baseline(w, echo, n_cols=64, n_chan=48)
    vals, secs = [], []
    for _ in range(args.steps):
        b, _, _ = oracle_baseline(w, echo, n_cols=64, n_chan=48)
        vals.append(b["value"])
        secs.append(b["seconds"])
    v = statistics.mean(vals)
    base = b
    base["value"] = v
    line = {"impl": "reference", "metric": METRIC,
            "value": v, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(w, world, args.precision,
                                      "CPU oracle on host cores (no GPU cache involved)"),
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch64(args, world, rank, local):
    """64 uneven monostatic scenes in one persistent launch (CUDA graph);
    autotuned block shape vs the fixed default shape."""
    import numpy as np
    import torch
    from paper_2109_02842_gb300 import binding, build as nbuild, workloads as wl
    torch.cuda.set_device(local)
    nbuild.build()
    binding.load()
    scenes = [wl.batch_scene(i, seed=rank) for i in range(64)]
    echos = [binding.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.pts, w.amp)
             for w in scenes]
    upd = sum(w.updates_per_scan() for w in scenes)
    pix_upd = sum(w.n_chan * w.grid["nx"] * w.grid["ny"] * w.n_pad for w in scenes)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    for name, kw in (("fixed", dict(tile_u=16, block_config=1)), ("default", {}),
                     ("persistent_tc", dict(tc_launch=1)), ("autotuned", dict(autotune=True))):
        b = binding.Batch(scenes, **kw)
        imgs = b.execute(echos)
        for _ in range(max(0, args.warmup - 1)):
            b.execute(echos, imgs)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            b.execute(echos, imgs)
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        ms = statistics.mean(ts)
        res[name] = {"ms_per_batch": ms, "value": upd / (ms * 1e-3), "info": b.get_info()}
        b.close()
    best = res["autotuned"]
    tc = best["info"]["block_config"] == 4
    peaks, peak_src = measured_peaks()
    unit_peaks = measure_unit_peaks(binding)
    if tc:
        peak, bound = float(peaks.get("bf16_tflops", 1900.0)), "tensor"
        basis = "dense BF16 burst, %s" % ("of measured" if peak_src == "measured" else "of fallback")
    else:
        peak, bound = (unit_peaks.get("fp32_tflops")
                       or N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e-6), "alu"
        basis = "FP32 FMA pipe (pl_measure_peak)" if unit_peaks.get("fp32_tflops") else "FP32 unit counts"
    achieved = pix_upd * METHOD_FLOP_PER_UPDATE / (best["ms_per_batch"] * 1e-3) / 1e12
    line = {"metric": METRIC,
            "value": best["value"], "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms_per_batch"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f32acc" if tc else "f32",
            "data": "synthetic",
            "config": {"workload": "batch-64-uneven-mono", "scenes": 64,
                       "l2": "flushed before every batch (256 MiB write, outside the events)"},
            "scans_per_s": 64 / (best["ms_per_batch"] * 1e-3),
            "fixed_vs_autotuned": {k: {"ms_per_batch": v["ms_per_batch"], "value": v["value"],
                                       "tile_u": v["info"]["tile_u"],
                                       "block_config": v["info"]["block_config"],
                                       "persistent": v["info"]["persistent"]}
                                   for k, v in res.items()},
            "autotune_speedup": res["fixed"]["ms_per_batch"] / best["ms_per_batch"],
            "gpu_launches": best["info"]["launches_per_execute"] * args.steps,
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "peak_basis": basis,
                         "kernel": "whole batch, the method's %d flop per (pixel, channel, "
                                   "k_z bin) update" % METHOD_FLOP_PER_UPDATE
                                   + ("; tensor-core back-projection" if tc else
                                      "; persistent FP32 kernel")},
            "unit_peaks": unit_peaks,
            "batch_info": best["info"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_table2(args, world, rank, local):
    """Table II restated on the GPU: the method (NUFFT + tensor-core
    back-projection), the exact-sum hybrid ("omega-K-BP") and direct BP on
    the Table I geometry (monostatic and multistatic; 64 scans and a 64^3
    grid over 0.2 m chosen here, the paper states neither)."""
    import numpy as np
    import torch
    from paper_2109_02842_gb300 import binding, build as nbuild, workloads as wl

    torch.cuda.set_device(local)
    nbuild.build()
    binding.load()
    paper = {"mono": {"omegaK_NUFFT_BP_s": 28.0, "omegaK_BP_s": 370.0, "BP_s": 2779.0},
             "multi": {"omegaK_NUFFT_BP_s": 62.0, "omegaK_BP_s": 685.0, "BP_s": 5824.0}}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    out = {}
    for mode, name in ((0, "mono"), (1, "multi")):
        w = wl.paper_table1(mode, seed=rank)
        echo = binding.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.pts, w.amp)
        plan = binding.Plan.from_workload(w)
        img = plan.execute(echo)
        ex = plan.execute_exact(echo)
        bp = plan.execute_bp_direct(echo)
        for _ in range(max(args.warmup - 1, 0)):
            plan.execute(echo, img)
        torch.cuda.synchronize()
        t_h = timed(lambda: plan.execute(echo, img), max(args.steps, 5))
        t_e = timed(lambda: plan.execute_exact(echo, ex), 3)
        t_b = timed(lambda: plan.execute_bp_direct(echo, bp), 2)
        a, e, b = (x.cpu().numpy() for x in (img, ex, bp))
        err = float(np.linalg.norm(a - e) / np.linalg.norm(e))
        corr = float(np.corrcoef(np.abs(a).ravel(), np.abs(b).ravel())[0, 1])
        out[name] = {"workload": w.name, "n_chan": w.n_chan,
                     "grid": [w.grid["nx"], w.grid["ny"], w.grid["nz"]],
                     "n_scan": w.n_scan, "n_f": w.n_f,
                     "omegaK_NUFFT_BP_ms": t_h, "omegaK_BP_ms": t_e, "BP_ms": t_b,
                     "ratio_omegaK_BP": t_e / t_h, "ratio_BP": t_b / t_h,
                     "paper_ratio_omegaK_BP": paper[name]["omegaK_BP_s"] / paper[name]["omegaK_NUFFT_BP_s"],
                     "paper_ratio_BP": paper[name]["BP_s"] / paper[name]["omegaK_NUFFT_BP_s"],
                     "paper_seconds": paper[name],
                     "nufft_vs_exact_rel_l2": err, "abs_corr_vs_BP": corr,
                     "updates_per_s": w.updates_per_scan() / (t_h * 1e-3),
                     "block_config": plan.info["block_config"]}
        plan.close()
    m = out["mono"]
    line = {"metric": METRIC,
            "value": m["updates_per_s"], "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["omegaK_NUFFT_BP_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3+f32acc", "data": "synthetic",
            "config": {"workload": "table2-paper-table1",
                       "l2": "flushed before every timed call (256 MiB write, outside the events)"},
            "table2": out}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batch64":
        run_batch64(args, world, rank, local)
        return
    if args.workload == "table2":
        run_table2(args, world, rank, local)
        return
    import numpy as np
    import torch
    from paper_2109_02842_gb300 import binding, build as nbuild, workloads as wl

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    nbuild.build()
    binding.load()
    dev = torch.device("cuda", local)

    w = wl.WORKLOADS[args.workload](seed=rank)
    plan = binding.Plan.from_workload(w, precision=args.precision)
    info = plan.info
    # inputs resident in HBM: scene echo synthesised on the GPU + 30 dB noise
    echo = binding.synth_echo(w.tx_xy, w.rx_xy, w.z0, w.dz, w.n_scan, w.f_hz, w.pts, w.amp)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)
    p_sig = float(torch.mean(echo.abs() ** 2))
    noise = torch.randn(echo.shape, dtype=torch.complex64, device=dev, generator=gen)
    echo += math.sqrt(p_sig * 10 ** (-w.snr_db / 10)) * noise
    del noise
    image = torch.empty(plan.image_shape, dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        flush.zero_()
        plan.execute(echo, image)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    plan.set_timing(True)
    clocks = ClockSampler(local, os.path.join(tempfile.gettempdir(),
                                              "pl_bench_clocks_rank%d.csv" % rank))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_begin = time.time()
    for i in range(args.steps):
        flush.zero_()                       # L2 flush between steps, outside the events
        starts[i].record(stream)
        plan.execute(echo, image)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop(t_begin, time.time())
    stage = plan.stage_times()
    plan.set_timing(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = max_over_ranks([statistics.mean(step_ms)], world, dev)[0]
    upd = w.updates_per_scan()
    value = whole_job_rate(upd, world, ms * 1e-3)

    # end to end through the C ABI with pinned host buffers: a stream of K
    # scans through pl_execute_host_stream (every scan's echo uploaded and
    # image downloaded inside the timed call, the copies overlapped with the
    # reconstruction of the neighbouring scans), host wall clock around the
    # call; beside it the latency of one pl_execute_host call
    ring = 3
    echo_h = [echo.cpu().pin_memory() for _ in range(ring)]
    image_h = [torch.empty(plan.image_shape, dtype=torch.complex64).pin_memory()
               for _ in range(ring)]
    plan.execute_host_stream([echo_h[i % ring] for i in range(args.warmup)],
                             [image_h[i % ring] for i in range(args.warmup)])
    if world > 1:
        torch.distributed.barrier()
    ta = time.perf_counter()
    plan.execute_host_stream([echo_h[i % ring] for i in range(args.steps)],
                             [image_h[i % ring] for i in range(args.steps)])
    e2e_s = (time.perf_counter() - ta) / args.steps
    lat = []
    for _ in range(3):
        ta = time.perf_counter()
        plan.execute_host(echo_h[0], image_h[0])
        lat.append(time.perf_counter() - ta)
    e2e_s, lat_s = max_over_ranks([e2e_s, statistics.mean(lat)], world, dev)

    # roofline of the dominant kernel (back-projection), live CUDA-event times
    bp_ms, bp_n = stage["backproject"]
    bp_avg_s = bp_ms / max(bp_n, 1) * 1e-3
    pix_updates = info["n_chan"] * info["nx"] * info["ny"] * info["n_pad"]
    method_flops = pix_updates * METHOD_FLOP_PER_UPDATE
    peaks, peak_src = measured_peaks()
    unit_peaks = measure_unit_peaks(binding)
    if info["block_config"] == 4:
        # tensor cores: the method's work (48 flop per (pixel, channel, bin)
        # update) against the dense BF16 peak; beside it the dense MMA work the
        # formulation issues (window rows x split products), i.e. how busy the
        # tensor pipe is kept
        dense = tc_flops_per_launch(info, args.precision)
        peak = float(peaks.get("bf16_tflops", 1900.0))
        achieved = method_flops / bp_avg_s / 1e12
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": kernel_traffic("backproject_tc", w.name),
                    "launch_ms": bp_avg_s * 1e3,
                    "flop_per_launch": method_flops,
                    "flop_basis": "%d flop per (pixel, channel, k_z bin) update: w-tap "
                                  "interpolation, split-float carrier phase and the complex "
                                  "multiply-accumulate (x %d updates per pass)"
                                  % (METHOD_FLOP_PER_UPDATE, pix_updates),
                    "launches_per_pass": info.get("bp_launches", 1),
                    "pass": "launch_ms, flop_per_launch and traffic are per back-projection "
                            "pass: from the start of its first launch to the end of its last",
                    "peak_basis": "dense BF16 burst, %s" % ("of measured" if peak_src == "measured"
                                                            else "of fallback"),
                    "kernel": "k_backproject_tc_sp" if info.get("sparse_products") else
                              "k_backproject_tc",
                    # the 2:4-sparse products issue the same logical MMA work
                    # (K = 32 per sparse product over [Re; Im] rows) at twice
                    # the dense rate: their pipe fraction is taken against 2x
                    # the dense peak
                    "mma_pipe_frac": dense / bp_avg_s / 1e12 / (peak * (2 if info.get(
                        "sparse_products") else 1)),
                    "mma_dense_flop_per_launch": dense,
                    "mma_basis": "BF16 MMA work issued (logical, dense-equivalent): 16 window "
                                 "rows x 4 real products x %d split products x 2 per (pixel, "
                                 "channel, bin) over padded tiles; only %d of the 16 rows carry "
                                 "a tap%s" % (3 if args.precision == 0 else 1, info["nufft_w"],
                                              "; 2:4-sparse products, against 2x the dense "
                                              "peak" if info.get("sparse_products") else "")}
    else:
        fp32_peak = unit_peaks.get("fp32_tflops") or N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e-6
        achieved = method_flops / bp_avg_s / 1e12
        executed = pix_updates * backproject_flops_per_update(info["nufft_w"])
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak, "traffic": kernel_traffic("backproject", w.name),
                    "kernel": "k_backproject", "launch_ms": bp_avg_s * 1e3,
                    "flop_per_launch": method_flops,
                    "flop_basis": "%d flop per (pixel, channel, k_z bin) update"
                                  % METHOD_FLOP_PER_UPDATE,
                    "peak_basis": ("FP32 FMA pipe, measured by pl_measure_peak in this run"
                                   if unit_peaks.get("fp32_tflops") else
                                   "FP32: 152 SM x 128 lanes x 2 flop x 2070 MHz (unit counts)"),
                    "executed_flop_frac": executed / bp_avg_s / 1e12 / fp32_peak,
                    "executed_basis": "%d flop per update actually executed (the carrier's phase "
                                      "and sin/cos once per (pixel, channel, bin block))"
                                      % backproject_flops_per_update(info["nufft_w"]),
                    "mufu_frac": (2 * pix_updates / max(info["tile_u"], 1) / bp_avg_s / 1e9) /
                                 unit_peaks["mufu_gsin"] if unit_peaks.get("mufu_gsin") else None}
    stage_avg = {k: v[0] / max(v[1], 1) for k, v in stage.items()}

    cpu, acc, variants = None, None, None
    if rank == 0 and world == 1 and not args.no_oracle:
        # accuracy leg and CPU baseline on an oracle-made echo (24 of the
        # scene's points: the operator is linear, so the error of the timed
        # 2020-point echo's image is of the same kind)
        import oracle
        oracle.build()
        clean = oracle.synth_echo(w.tx_xy, w.rx_xy, w.z_scan, w.f_hz, w.pts[:24], w.amp[:24])
        e_np = wl.add_noise(clean, w.snr_db, wl.rng_for(100, 0)).astype(np.complex64)
        e_dev = torch.from_numpy(e_np).to(dev)
        img = plan.execute(e_dev).cpu().numpy()
        cpu, acc, (idx, ref) = oracle_baseline(w, e_np, img, n_cols=256)
        acc["echo"] = "oracle echo of 24 of the scene's points, 30 dB noise"
        # every precision variant of both kernel families on the same columns
        variants = {}
        for name, kw in (("tensor_core_bf16x3", dict(block_config=4, precision=0)),
                         ("tensor_core_bf16", dict(block_config=4, precision=1)),
                         ("tensor_core_bf16_spectrum", dict(block_config=4, precision=2)),
                         ("fp32", dict(block_config=3 if w.mode == 0 else 1, precision=0)),
                         ("fp32_bf16_table", dict(block_config=1, precision=1)),
                         ("fp32_bf16_table_spectrum", dict(block_config=1, precision=2))):
            try:
                pv = binding.Plan.from_workload(w, **kw)
            except binding.PolylineError as ex:
                variants[name] = {"unavailable": str(ex)}
                continue
            iv = pv.execute(e_dev).cpu().numpy()
            variants[name] = dict(column_error(iv, w, idx, ref), dtype=dtype_of(pv.info, kw["precision"]),
                                  block_config=pv.info["block_config"], precision=kw["precision"])
            pv.close()

    line = {
        "metric": METRIC,
        "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(info, args.precision),
        "data": "synthetic",
        "config": workload_config(w, world, args.precision,
                                  "flushed before every step (256 MiB write, outside the "
                                  "step events)"),
        "scans_per_s": world / (ms * 1e-3),
        "e2e": {"value": whole_job_rate(upd, world, e2e_s), "unit": "updates/s",
                "h2d_bytes_per_step": int(echo.numel() * 8),
                "d2h_bytes_per_step": int(image.numel() * 8),
                "scans_per_s": world / e2e_s,
                "api": "pl_execute_host_stream over %d scans (pinned host buffers, "
                       "copies overlapped with compute, alternate scans on two "
                       "plans and streams)" % args.steps,
                "single_scan_latency_ms": lat_s * 1e3},
        "gpu_launches": info["launches_per_execute"] * args.steps,
        "roofline": roofline,
        "stage_ms": stage_avg,
        "clocks": clk,
        "wall_s_timed_region": wall,
        "accuracy_vs_oracle": acc,
        "accuracy_by_variant": variants,
        "unit_peaks": unit_peaks,
        "cpu_baseline": cpu,
        "peaks_source": peak_src,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
