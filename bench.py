"""Benchmark: one step = one full debiased Sinkhorn solve (sinkhorn_divergence)
on the synthetic track-density workload (two 64^3 density volumes, ~100k
weighted voxels each, masses 1.0 vs 1.2, p = 2, blur = 1 voxel, reach = 10
voxels, eps-scaling q = 0.5, multiscale with 4-voxel grid cells), run to the
stopping rule (estimated remaining relative change of S below 1e-6).

Prints ONE JSON line.  `value` is softmin pairs evaluated per second of solve
time (all four symmetric instances, whole solve: clustering, coarse phase,
extrapolation, truncation, fine steps, final FP64 sums).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Other workloads (not the default line; each prints its own JSON line):
    --workload fibers [--n N] [--precision fp32|tc]   60-D fiber bundles, k-means multiscale,
        blur 2 mm, reach 20 mm (FP32 or the BF16 hi/lo tensor-core cross term)
    --workload mlp [--n N]    warm-start network: inference and training throughput
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Measured per-SM, per-clock rates on GB300 (sm_103a): ex2.approx 32/clk (the
# MUFU unit), FP32 FMA 128 lanes/clk (f32x2 packing halves issue, not FP32 work).
# A pair of a stable log-sum-exp in the dot-product form costs D FMAs, one add
# (the row's reference), one add (accumulate) and one ex2 on the CUDA cores; in
# the tensor-core forms the exponent comes from the tensor core and the CUDA
# cores keep one ex2 and one add per pair, so the MUFU unit bounds them.
SFU_EX2_PER_CLK_SM = 32
FP32_LANES_PER_CLK_SM = 128
# D <= 3, default precision: tensor-core dot product of K = 32 BF16 slots per pair
TC3_TENSOR_FLOP_PER_PAIR = 2 * 32
# DRAM bytes (read + write) of one fine-step launch of softmin3_tc_kernel on this
# workload, from one ncu capture (profiles/softmin3_tc_trackdensity_100k_multiscale.md);
# to be re-measured whenever that kernel changes
SOFTMIN3_TC_DRAM_BYTES = 172.6e6


def workload(args):
    from paper_2107_02010_gb300 import synth

    x, a, y, b = synth.density_maps(grid=args.grid, n_keep=args.n_keep)
    return x, a, y, b


def fiber_workload(args):
    from paper_2107_02010_gb300 import synth

    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(args.n, seed=4, ctrl=ctrl, perturb=3.0)
    y, b, _ = synth.fiber_bundles(args.n, seed=5, ctrl=ctrl)
    return x, a, y, b


def fiber_params(args, otgb):
    return otgb.default_params(blur=2.0, reach=20.0, scaling=0.5, multiscale=1, cluster=1,
                               k_clusters=max(20, args.n // 1000), kmeans_iters=10, tol=args.tol,
                               max_iters=args.max_iters, precision=1 if args.precision == "tc" else 0)


def params_for(args, otgb):
    return otgb.default_params(blur=1.0, reach=10.0, scaling=0.5, multiscale=int(args.multiscale), cluster=0,
                               cell=4.0, tol=args.tol, max_iters=args.max_iters, check_every=10,
                               rows_per_thread=args.rows_per_thread)


def start_clock_sampler():
    try:
        # the raw samples go to the file named by OTGB_CLOCKS_CSV, if set
        f = open(os.environ.get("OTGB_CLOCKS_CSV") or os.devnull, "w")
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
            text=True)
        return p, f
    except Exception:
        return None, None


def stop_clock_sampler(p, f, dev_index=0):
    if p is None:
        return None
    time.sleep(0.3)
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        out = ""
    rows = []
    for line in out.splitlines():
        parts = [s.strip() for s in line.split(",")]
        if len(parts) < 9 or parts[0] != str(dev_index):
            continue
        rows.append(parts)
        if f:
            f.write(line + "\n")
    if f:
        f.close()
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


def flush_l2(buf):
    buf.add_(1.0)  # touches 256 MB (> 129 MB L2)


def cpu_baseline(x, a, y, b, rows=0, target_s=10.0):
    """The FP64 oracle's softmin on a bounded sample: `rows` rows of the
    alpha->beta instance against all columns, at eps = blur^2.  rows = 0: a
    calibration run of 2048 rows sets the row count for about target_s seconds
    (at most every row).  Returns (the cpu_baseline object, rows used)."""
    import oracle

    oracle.build()
    pot = np.zeros(y.shape[0])

    def run(n):
        idx = np.linspace(0, x.shape[0] - 1, n).astype(np.int64)
        t0 = time.perf_counter()
        oracle.softmin(x[idx], y, b, pot, 1.0, 1.0 / 1.01)
        return time.perf_counter() - t0

    if rows <= 0:
        dt0 = run(2048)
        rows = int(min(x.shape[0], max(2048, 2048 * target_s / max(dt0, 1e-6))))
    dt = run(rows)
    pairs = rows * y.shape[0]
    return {"value": pairs / dt, "unit": "pairs/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": "FP64 oracle softmin: %d rows x %d columns of the track-density workload (%.1f s)" %
                      (rows, y.shape[0], dt)}, rows


def peak_pairs_per_s(D, clock_mhz, n_sm):
    per_clk = min(SFU_EX2_PER_CLK_SM, FP32_LANES_PER_CLK_SM / (D + 2))
    return per_clk * n_sm * clock_mhz * 1e6


def run_mlp(args):
    """Warm-start network throughput: inference over n rows and one training
    epoch over n rows (batches of 16384), FLOPs counted as 2 per multiply-add of
    the four layers (input padded to 64); training = 3 x forward."""
    import torch
    from paper_2107_02010_gb300 import otgb

    ctx = otgb.Context()
    D, H = 60, 256
    net = otgb.Mlp(ctx, D, H, seed=1)
    r = np.random.default_rng(0)
    n = args.n
    x = torch.from_numpy(r.normal(0, 1, (n, D)).astype(np.float32)).cuda()
    f = torch.from_numpy(r.normal(0, 1, n).astype(np.float32)).cuda()
    fwd = 2.0 * n * (64 * H + 2 * H * H + H)
    for _ in range(args.warmup):
        net.infer(x)
        net.train_epoch(x, f, 16384, 1e-4, seed=0)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    l0 = otgb.kernel_launches()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(st)
    for _ in range(args.steps):
        net.infer(x)
    ev[1].record(st)
    ev[2].record(st)
    for k in range(args.steps):
        net.train_epoch(x, f, 16384, 1e-4, seed=k + 1)
    ev[3].record(st)
    torch.cuda.synchronize()
    inf_ms = ev[0].elapsed_time(ev[1]) / args.steps
    tr_ms = ev[2].elapsed_time(ev[3]) / args.steps
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    peak = peaks.get("bf16_tflops", 1900.0)
    line = {"metric": "warm-start network TFLOP/s", "workload": "mlp", "unit": "TFLOP/s",
            "value": fwd / inf_ms / 1e9, "steps": args.steps, "warmup": args.warmup, "dtype": "bf16",
            "data": "synthetic", "higher_is_better": True,
            "config": {"workload": "MLP %d->%d->%d->%d->1 SiLU, %d rows" % (D, H, H, H, n)},
            "inference_ms": inf_ms, "inference_tflops": fwd / inf_ms / 1e9,
            "train_epoch_ms": tr_ms, "train_tflops": 3 * fwd / tr_ms / 1e9,
            "roofline": {"bound": "tensor", "peak": peak, "unit": "TFLOP/s",
                         "frac_inference": fwd / inf_ms / 1e9 / peak, "frac_train": 3 * fwd / tr_ms / 1e9 / peak,
                         "peak_basis": "bf16 burst, of measured"},
            "gpu_launches": int(otgb.kernel_launches() - l0)}
    print(json.dumps(line))
    return 0


def run_fibers(args):
    """60-D fiber bundles (N = M = n), k-means multiscale, FP32 or tensor-core
    form; one step = one solve to the stopping rule."""
    import torch
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = fiber_workload(args)
    X, A, Y, B = (torch.from_numpy(v).cuda() for v in (x, a, y, b))
    ctx = otgb.Context()
    p = fiber_params(args, otgb)
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        out = otgb.sinkhorn_divergence(ctx, X, A, Y, B, p, raise_on_noconv=False)
    torch.cuda.synchronize()
    sampler, sf = start_clock_sampler()
    st = torch.cuda.current_stream()
    l0 = otgb.kernel_launches()
    ms, pairs, smin = [], 0.0, 0.0
    for _ in range(args.steps):
        flush_l2(l2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        out = otgb.sinkhorn_divergence(ctx, X, A, Y, B, p, raise_on_noconv=False)
        e1.record(st)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        pairs += out["stats"]["pairs_evaluated"]
        smin += out["stats"]["softmin_ms"]
    clocks = stop_clock_sampler(sampler, sf)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    clk = peaks.get("sm_max_mhz", 2070.0)
    D = x.shape[1]
    if args.precision == "tc":
        # three K = 64 BF16 MMAs per pair (hi.hi, hi.lo, lo.hi); the MUFU bound is higher
        peak = min(peaks.get("bf16_tflops", 1929.8) * 1e12 / (3 * 2 * 64), SFU_EX2_PER_CLK_SM * n_sm * clk * 1e6)
        basis = "tensor: bf16 of measured / 384 flop per pair (MUFU %d SMs x 32/clk is higher)" % n_sm
        bound = "tensor"
    else:
        peak = peak_pairs_per_s(D, clk, n_sm)
        basis = "FP32 form: %d SMs x min(32, 128/(D+2)) pairs/clk x %.0f MHz" % (n_sm, clk)
        bound = "alu"
    achieved = pairs / (smin / 1e3) if smin > 0 else None
    line = {"metric": "softmin pairs/s", "workload": "fibers", "value": pairs / (sum(ms) / 1e3), "unit": "pairs/s",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
            "higher_is_better": True, "dtype": "f32" if args.precision == "fp32" else "bf16x3+f32",
            "data": "synthetic",
            "config": {"workload": "fiber bundles 60-D, N=M=%d, k-means %d clusters, blur 2, reach 20, q 0.5, %s" %
                                   (args.n, max(20, args.n // 1000), args.precision)},
            "time_to_solve_ms": statistics.mean(ms), "iters_per_solve": out["stats"]["iters_total"],
            "S": out["S"], "last_stats": out["stats"],
            "roofline": {"bound": bound, "achieved": achieved / 1e9 if achieved else None, "peak": peak / 1e9,
                         "unit": "Gpairs/s", "frac": achieved / peak if achieved else None, "peak_basis": basis},
            "gpu_launches": int(otgb.kernel_launches() - l0), "clocks": clocks}
    print(json.dumps(line))
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    x, a, y, b = workload(args)
    cb = None
    vals = []
    rows = args.ref_rows
    for k in range(args.warmup + args.steps):
        r, rows = cpu_baseline(x, a, y, b, rows=rows, target_s=5.0)  # calibrated once, then fixed
        if k >= args.warmup:
            vals.append(r["value"])
            cb = r
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": "softmin pairs/s", "value": v, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "track-density maps 64^3, ~%d voxels per side, FP64 oracle softmin sample" %
                                   x.shape[0]},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--n-keep", type=int, default=100_000)
    ap.add_argument("--multiscale", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iters", type=int, default=20000)
    ap.add_argument("--ref-rows", type=int, default=0, help="oracle sample rows (0: about 5-10 s of host work)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows-per-thread", type=int, default=0)
    ap.add_argument("--workload", default="density", choices=["density", "fibers", "mlp"])
    ap.add_argument("--n", type=int, default=0, help="fibers: points per side (200000); mlp: rows (1048576)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tc"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "fibers":
        args.n = args.n or 200_000
        args.max_iters = min(args.max_iters, 5000)
        return run_fibers(args)
    if args.workload == "mlp":
        args.n = args.n or (1 << 20)
        return run_mlp(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2107_02010_gb300 import otgb

    # Independent replicas: every rank solves its own copy of the workload; no
    # data-path collective exists in the method on one problem.
    x, a, y, b = workload(args)
    dev = torch.device("cuda", local)
    X, A, Y, B = (torch.from_numpy(v).to(dev) for v in (x, a, y, b))
    ctx = otgb.Context()
    p = params_for(args, otgb)
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    solve = lambda *t: otgb.sinkhorn_divergence(ctx, *t, p, raise_on_noconv=False)
    for _ in range(args.warmup):
        out = solve(X, A, Y, B)
    torch.cuda.synchronize()

    sampler, sf = start_clock_sampler()
    st = torch.cuda.current_stream()
    launches0 = otgb.kernel_launches()
    step_ms, pairs, smin_ms, iters, S_vals, statuses = [], 0.0, 0.0, [], [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush_l2(l2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        out = solve(X, A, Y, B)
        e1.record(st)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        s = out["stats"]
        pairs += s["pairs_evaluated"]
        smin_ms += s["softmin_ms"]
        iters.append(s["iters_total"])
        S_vals.append(out["S"])
        statuses.append(out["status"])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    launches = otgb.kernel_launches() - launches0
    clocks = stop_clock_sampler(sampler, sf, local)

    ms_per_step = statistics.mean(step_ms)
    t_total = sum(step_ms) / 1e3
    from paper_2107_02010_gb300 import replicas

    t_total, pairs = replicas.aggregate(t_total, pairs, dev)
    value = pairs / t_total

    # end to end through the public API with host buffers: pinned host inputs
    # copied in, the solve, and S plus the potentials f, g read back
    hx, ha, hy, hb = (torch.from_numpy(v).pin_memory() for v in (x, a, y, b))
    e2e_ms = []
    for k in range(args.steps + 1):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        Xd, Ad, Yd, Bd = (h.to(dev, non_blocking=True) for h in (hx, ha, hy, hb))
        o = solve(Xd, Ad, Yd, Bd)
        fh, gh = o["f"].cpu(), o["g"].cpu()
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append((time.perf_counter() - t1) * 1e3)
    pairs_per = pairs / args.steps / max(world, 1)
    e2e_val = pairs_per / (statistics.mean(e2e_ms) / 1e3) * max(world, 1)
    h2d = sum(v.nbytes for v in (x, a, y, b))
    d2h = 4 * (x.shape[0] + y.shape[0]) + 8

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = peaks.get("sm_max_mhz", 2070.0)
    # the default D <= 3 kernel (softmin3_tc_kernel): min(MUFU ex2, tensor pipe)
    peak_mufu = SFU_EX2_PER_CLK_SM * n_sm * clk * 1e6
    peak_tensor = peaks.get("bf16_tflops", 1929.8) * 1e12 / TC3_TENSOR_FLOP_PER_PAIR
    peak = min(peak_mufu, peak_tensor)
    peak_fp32_form = peak_pairs_per_s(3, clk, n_sm)
    achieved = pairs / max(world, 1) / (smin_ms / 1e3) if smin_ms > 0 else None

    if rank != 0:
        return 0
    line = {
        "metric": "softmin pairs/s", "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "track-density maps: two 64^3 volumes of 30 Gaussian tubes, %d voxels per side, "
                               "masses 1.0/1.2, p=2, blur=1, reach=10, q=0.5, %s, stop at est. rel. change of "
                               "S < %g" % (x.shape[0], "multiscale grid cells of 4 voxels" if args.multiscale
                                           else "dense single scale", args.tol),
                   "N": int(x.shape[0]), "M": int(y.shape[0]), "D": 3,
                   "l2": "256 MB buffer written between timed steps (inputs are smaller than L2)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "time_to_solve_ms": ms_per_step,
        "iters_per_solve": statistics.mean(iters),
        "S": S_vals[-1],
        "converged": all(v == 0 for v in statuses),
        "last_stats": out["stats"],
        "softmin_ms_per_solve": smin_ms / args.steps,
        "pairs_per_solve": pairs_per,
        "roofline": {"bound": "alu", "kernel": "softmin3_tc_kernel (+ fallback), per softmin launch",
                     "achieved": achieved / 1e9 if achieved else None, "peak": peak / 1e9, "unit": "Gpairs/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": SOFTMIN3_TC_DRAM_BYTES,
                     "traffic_unit": "bytes per fine-step launch (ncu dram__bytes_read + write)",
                     "peak_basis": "MUFU ex2: %d SMs x 32 ex2/clk x %.0f MHz (measured per-clock rate; clock = "
                                   "sm_max_mhz of MEASURED_PEAKS.json), below the tensor bound %.3g pairs/s "
                                   "(bf16, of measured, %d flop per pair)" % (n_sm, clk, peak_tensor,
                                                                            TC3_TENSOR_FLOP_PER_PAIR),
                     "fp32_form_peak": peak_fp32_form / 1e9,
                     "frac_of_fp32_form_peak": (achieved / peak_fp32_form) if achieved else None},
        "e2e": {"value": e2e_val, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s": wall,
    }
    if not args.no_cpu_baseline and world <= 1:
        line["cpu_baseline"] = cpu_baseline(x, a, y, b)[0]
    print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
