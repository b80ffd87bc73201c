#!/usr/bin/env python3
"""Benchmark: Moore-Penrose inverse of a rank-deficient 4096 x 3072 matrix.

Workload (seeded, synthetic): A = U diag(s) V^T, Haar U (4096 x 2304) and
V (3072 x 2304), s log-spaced in [1e-4, 1] (rank 2304, kappa 1e4 on the
range), X0 = alpha A^T with alpha = 1/s_1^2 (Section 4: any 0 < alpha <
2/s_1^2 converges; this end of the range keeps every residual eigenvalue in
[0, 1), which low-precision loops need), stabilised variant (Section 7) with
the cleanup finish.

Settings: mixed precision -- FP32-class products while the iterate grows,
FP64-class products from the loop after the first step below 1 -- the
stabilised product in the FP64-class loops after a step below 0.9, order-18
stop (step < 1e-2 keeps that loop's result: the next step would be below
rounding), cleanup finish (projection + order-2 step in FP64 class).

One step = one full solve through pinv_solve on device-resident A.  The
metric counts a solve only if it reaches the 1e-9 Penrose residual; the
accuracy of the last timed result is checked after the timed region
(Penrose residuals on the device and sampled rows against the closed form
V diag(1/s) U^T).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64_tc|fp64|mixed_bf16]

The default (--prec fp32) is the mixed form: FP32-class slice products (4
exact BF16 slices per operand, 10 slice products) in the growth loops,
FP64-class ones (7 slices, 28 slice products) in the last loops and the
finish, all on the BF16 tensor cores.  Beside it the line carries the same
solve with every product FP64-class on the tensor cores (fp64_tc) and the
plain FP64 iteration on native FP64 DMMA products (fp64_gpu), each with its
own loop count.
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Multi-GPU: independent replicas (one solve per rank per step, no collective on
the data path); value = all ranks' solves / max-over-ranks time.
"""

from __future__ import annotations

import argparse
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

# Independent groups of batched and served problems run on their own streams;
# with the default eight hardware connections several streams share one queue
# and a small problem's loop waits behind a large problem's kernels on it
# (measured on the serving sample: p50 latency 305 ms with 8, 136 ms with 32).
# The setting is read when the CUDA context is created, so it is made before
# anything here touches the GPU.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

M, N, RANK, S_MIN, SEED = 4096, 3072, 2304, 1e-4, 1
METRIC = "pseudoinverses/s at 1e-9 Penrose residual"
UNIT = "solves/s"
WORKLOAD = "moore_penrose_rank_deficient_4096x3072_r2304"
# dram__bytes_read.sum + dram__bytes_write.sum of one 3072x3072x4096 launch of
# the dominant kernel in each product class (one ncu capture of the current
# kernel per class), per FP64-equivalent flop of that launch; a solve's mean launch weights them by
# the FP64-equivalent work each class processed (this workload's products are
# n x n x m and n x n x n with n = 3072, m = 4096: the captured shapes).
TRAFFIC_REF_FLOPS = 2.0 * 3072 * 3072 * 4096   # the captured launches' 2MNK
TRAFFIC_PER_FLOP = {"fp32": (964.2e6 + 62.8e6) / TRAFFIC_REF_FLOPS,
                    "fp64_tc": (3.277e9 + 62.8e6) / TRAFFIC_REF_FLOPS}


def mean_launch_traffic(prec, gemm_flops, tensor_flops, launches):
    """DRAM bytes of the mean tensor-core launch of a solve, from the per-class
    figures: the FP64-class and FP32-class work (28 and 10 slice products per
    FP64-equivalent flop) are separated from the totals.  None where the solve
    ran classes without a captured figure (BF16, native FP64)."""
    if not launches or prec not in ("fp32", "fp32_refine", "fp64_tc"):
        return None
    if prec == "fp64_tc":
        f64, f32 = gemm_flops, 0.0
    else:
        f64 = max(0.0, (tensor_flops - 10.0 * gemm_flops) / 18.0)
        f32 = max(0.0, gemm_flops - f64)
    return (f32 * TRAFFIC_PER_FLOP["fp32"] + f64 * TRAFFIC_PER_FLOP["fp64_tc"]) / launches


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def dominant_peak(prec, peaks):
    """Peak of the dominant GEMM's dtype in TFLOP/s.  FP64 has no measured
    figure: the measured BF16 sustained rate times the nominal ratio (1.25/2250)."""
    bf16 = peaks["bf16_tflops_sustained"]
    if prec == "fp64":
        return bf16 * 1.25 / 2250.0, "bf16 sustained x nominal fp64/bf16 (1.25/2250)"
    return bf16, "bf16 sustained (the slice products run on the BF16 tensor cores)"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The slowest rank's value (the timed region ends when every replica has
    finished).  dist: torch.distributed or None for a single process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput of independent replicas: every rank solves `steps`
    problems, all of them in the max-over-ranks time."""
    return world * steps / (max_ms * 1e-3)


def workload():
    from paper_1604_07893_gb300 import workloads as W
    w = W.rectangular(M, N, RANK, 1.0, S_MIN, seed=SEED)
    alpha = 1.0 / w.s[0] ** 2
    return w, alpha


SWITCH_TOL = 0.9


def solve_kwargs(prec, alpha):
    """Stabilised variant in the FP64-class loops after a step below 0.9 (the
    iterate is then within one order-18 contraction of its limit, so X A X
    does not collapse anything), stopped by the order-18 rule at step < 1e-2,
    cleanup finish."""
    return dict(alpha=alpha, tol=1e-2, stop="order18", prec=prec, variant="stabilized",
                switch_tol=SWITCH_TOL, finish="clean")


# Loops of one solve of the headline workload with the bench's settings, as the
# oracle itself runs them (order-18 stop at 1e-2, stabilised after a step
# below 0.9, cleanup finish): 8 loops, one of them stabilised.  The GPU solve
# reports the same counts.
ORACLE_LOOPS, ORACLE_STAB_LOOPS = 8, 1


def cpu_oracle_sample(A, alpha, loops_per_solve=ORACLE_LOOPS, stab_loops=ORACLE_STAB_LOOPS, budget_s=30.0):
    """Time the FP64 oracle as it stands on a bounded sample of the workload:
    its naive order-18 loop (17 products + the update), its stabilised loop
    (the naive loop, then X A X) and the cleanup projection on the full
    4096 x 3072 matrix, then extrapolate to the loops of one solve."""
    from oracle import hyperpower as H
    X0 = H.x0_moore_penrose(A, alpha)
    t0 = time.perf_counter()
    X1 = H.hyperpower_step(A, X0, side="left")
    t_loop = time.perf_counter() - t0
    t_stab = t_clean = None
    if t_loop < budget_s / 3:
        t0 = time.perf_counter()
        H.stabilised_step(A, X0, side="left")
        t_stab = time.perf_counter() - t0
        t0 = time.perf_counter()
        H.cleanup_moore_penrose(A, X1)
        t_clean = time.perf_counter() - t0
    t_stab_ = t_stab if t_stab is not None else t_loop
    per_solve = (t_loop * (loops_per_solve - stab_loops) + t_stab_ * stab_loops
                 + (t_clean if t_clean is not None else t_loop))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": 1.0 / per_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one naive loop ({t_loop:.2f} s), one stabilised loop ({t_stab_:.2f} s) and one "
                       f"cleanup projection ({(t_clean or float('nan')):.2f} s) of the full 4096x3072 "
                       f"problem, extrapolated to {loops_per_solve} loops ({stab_loops} stabilised) "
                       f"+ the cleanup per solve"),
            "s_per_solve": per_solve}


SCHEDULES = {"fp32_refine": "fp32-class loops while the step is >= 1; after the first loop below 1, X A X in "
                            "fp32 class, one fp32-class order-2 step, then fp64-class order-2 steps until "
                            "min(step, previous step^2) < 1e-5; finish fp64-class",
             "fp32": "fp32-class products while the step is >= 1, then fp64-class; finish fp64-class",
             "fp64_tc": "fp64-class products throughout",
             "fp64": "native fp64 (DMMA) products throughout",
             "mixed_bf16": "bf16 while the step is > 0.5, fp32-class, then fp64-class"}


def bench_config(prec, world):
    """The `config` of the headline line, shared by both arms."""
    return {"workload": WORKLOAD, "m": M, "n": N, "rank": RANK, "s_range": [S_MIN, 1.0],
            "alpha": "1/s_1^2", "prec": prec, "schedule": SCHEDULES[prec],
            "variant": "stabilized", "switch_tol": SWITCH_TOL, "stop": "order18",
            "tol": 1e-2, "finish": "clean",
            "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (A 100 MB, workspace 0.8 GB)"}


def run_reference(args):
    rank, local, world = env_rank()
    if rank != 0:
        return 0
    w, alpha = workload()
    times = []
    for i in range(args.warmup + args.steps):
        s = cpu_oracle_sample(w.A, alpha)
        if i >= args.warmup:
            times.append(s["s_per_solve"])
    per = statistics.mean(times)
    value = 1.0 / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args.prec, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                             "sample": s["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, local, world = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1604_07893_gb300 import Handle

    w, alpha = workload()
    A = torch.from_numpy(w.A).to(dev)
    X = torch.empty((N, M), dtype=torch.float64, device=dev)
    h = Handle(local)
    kw = solve_kwargs(args.prec, alpha)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        h.solve(A, X, **kw)
    torch.cuda.synchronize(dev)

    infos = []
    per_step = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            _, info = h.solve(A, X, profile=True, **kw)
            ev[i][1].record(stream)
            infos.append(info)
        t_all1.record(stream)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(t_all0.elapsed_time(t_all1), dist, dev)
    per_step = [a.elapsed_time(b) for a, b in ev]
    clocks = clk.summary()

    # accuracy of the last timed result (untimed)
    Xh = X.cpu().numpy()
    rows = np.random.default_rng(0).choice(N, 32, replace=False)
    ref_rows = (w.V[rows] / w.s) @ w.U.T
    row_err = float(np.linalg.norm(Xh[rows] - ref_rows) / np.linalg.norm(ref_rows))
    _, cinfo = h.solve(A, X, check=True, **kw)
    penrose = max(cinfo["penrose"])
    ok = penrose <= 1e-9 and row_err <= 1e-9

    # end to end through the C ABI with host buffers (pinned)
    A_pin = torch.from_numpy(w.A).pin_memory()
    X_pin = torch.empty((N, M), dtype=torch.float64).pin_memory()
    A_np, X_np = A_pin.numpy(), X_pin.numpy()
    h.solve(A_np, X_np, host=True, **kw)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h.solve(A_np, X_np, host=True, **kw)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    # the same solve with every product FP64-class on the tensor cores, and the
    # plain FP64 GPU iteration (native FP64 DMMA products), beside the mixed form
    def other_arm(prec, reps):
        kwo = solve_kwargs(prec, alpha)
        h.solve(A, X, **kwo)
        torch.cuda.synchronize(dev)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(reps):
            _, io = h.solve(A, X, **kwo)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        _, co = h.solve(A, X, check=True, **kwo)
        ms = s0.elapsed_time(s1) / reps
        return {"value": 1e3 / ms, "unit": UNIT, "ms_per_solve": ms, "loops": io["iters"],
                "stabilized_loops": io["stabilized_loops"], "penrose_max": max(co["penrose"])}
    fp32_loops = other_arm("fp32", 3) if args.prec == "fp32_refine" and not args.no_fp64 else None
    fp64_tc = other_arm("fp64_tc", 3) if args.prec != "fp64_tc" and not args.no_fp64 else None
    fp64 = other_arm("fp64", 1) if args.prec != "fp64" and not args.no_fp64 else None

    if rank != 0:
        h.close()
        if dist:
            dist.destroy_process_group()
        return 0

    peaks, peak_src = load_peaks()
    peak, peak_note = dominant_peak(args.prec, peaks)
    gemm_ms = sum(i["gemm_ms"] for i in infos)
    gemm_flops = sum(i["gemm_flops"] for i in infos)
    gemm_launches = sum(i["gemms"] for i in infos)
    # the dominant kernel's algorithmic work: FP64 products for the DMMA path;
    # for the tensor-core path the BF16 slice products it executes (28 per FP64
    # product at FP64 class), reported beside the FP64-equivalent rate
    work = gemm_flops if args.prec == "fp64" else sum(i["tensor_flops"] for i in infos)
    achieved = work / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    fp64_equiv = gemm_flops / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    traffic = mean_launch_traffic(args.prec, gemm_flops, sum(i["tensor_flops"] for i in infos), gemm_launches)
    value = replica_throughput(world, args.steps, total_ms)
    sorted_ms = sorted(per_step)
    p50 = statistics.median(per_step)
    p99 = sorted_ms[min(len(sorted_ms) - 1, int(math.ceil(0.99 * len(sorted_ms))) - 1)]
    cpu = None
    if not args.no_cpu and world == 1:   # the loop counts this solve ran (the oracle runs the same)
        # (the refine schedule's order-2 steps have no counterpart in the oracle,
        # which converges in its own ORACLE_LOOPS loops)
        cpu = (cpu_oracle_sample(w.A, alpha) if args.prec == "fp32_refine" else
               cpu_oracle_sample(w.A, alpha, infos[-1]["iters"], infos[-1]["stabilized_loops"]))
        cpu.pop("s_per_solve", None)

    line = {
        "metric": METRIC, "value": value if ok else 0.0, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp64_tc": "bf16 slices (fp64-class)",
                  "fp32": "bf16 slices (fp32-class, then fp64-class)",
                  "fp32_refine": "bf16 slices (fp32-class loops, fp64-class refinement)",
                  "mixed_bf16": "bf16 + bf16 slices"}[args.prec],
        "data": "synthetic",
        "config": bench_config(args.prec, world),
        "latency_ms": {"p50": p50, "p99": p99},
        "accuracy": {"penrose_max": penrose, "sampled_rows_rel_err": row_err, "meets_1e-9": ok,
                     "loops": infos[-1]["iters"], "stabilized_loops": infos[-1]["stabilized_loops"],
                     "loop_classes": ["fp64" if p == 0 else {1: "bf16", 3: "fp32-class", 4: "fp64-class", 5: "fp32-class order-2", 6: "fp64-class order-2"}[p]
                                      for p in infos[-1]["precision"]],
                     "step_measures": infos[-1]["history"]},
        "e2e": {"value": world / e2e_s if ok else 0.0, "unit": UNIT,
                "h2d_bytes_per_step": M * N * 8, "d2h_bytes_per_step": N * M * 8},
        "gpu_launches": sum(i["kernels"] for i in infos),
        "roofline": {"bound": "tensor", "kernel": "gemm_f64_kernel" if args.prec == "fp64" else "tc_gemm_kernel",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "fp64_equivalent_tflops": fp64_equiv,
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_source": f"{peak_src}: {peak_note}",
                     "gemm_launches": gemm_launches, "gemm_share_of_step": gemm_ms / total_ms},
        "clocks": clocks,
        "cpu_baseline": cpu,
        "fp32_loops": fp32_loops,
        "fp64_tc": fp64_tc,
        "fp64_gpu": fp64,
    }
    print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()
    return 0




# ---------------------------------------------------------------------------
# further workloads (each prints its own JSON line; not the default run)
# ---------------------------------------------------------------------------

def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


def _emit(line):
    print(json.dumps(line), flush=True)


def run_mp64(args):
    """64 x 48 Moore-Penrose, s log-spaced in [1e-2, 1], alpha = 2/(s1^2 + sr^2):
    per-solve latency (the problem is launch-bound)."""
    import torch
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    w = W.rectangular(64, 48, None, 1.0, 1e-2, seed=0)
    alpha = 2.0 / (w.s[0] ** 2 + w.s[-1] ** 2)
    A = torch.from_numpy(w.A).cuda()
    X = torch.empty(48, 64, dtype=torch.float64, device="cuda")
    h = Handle(0)
    st = torch.cuda.current_stream()
    out = {}
    for key in ("fp64_tc", "autotuned"):
        prec = "fp64_tc"
        if key == "autotuned":   # the engine crossover, measured on this device, routes small products to DMMA
            out["crossover"] = h.autotune()
        for _ in range(args.warmup):
            h.solve(A, X, alpha=alpha, tol=1e-12, prec=prec)
        lat = []
        for _ in range(max(args.steps, 50)):
            e0, e1 = _events(st)
            e0.record(st)
            _, info = h.solve(A, X, alpha=alpha, tol=1e-12, prec=prec)
            e1.record(st)
            torch.cuda.synchronize()
            lat.append(e0.elapsed_time(e1))
        err = float(np.linalg.norm(X.cpu().numpy() - (w.V / w.s) @ w.U.T) / np.linalg.norm((w.V / w.s) @ w.U.T))
        out[key] = {"value": 1e3 / statistics.mean(lat), "p50_ms": statistics.median(lat),
                     "p99_ms": _pct(lat, 0.99), "rel_err_vs_closed_form": err, "loops": info["iters"],
                     "kernels_per_solve": info["kernels"]}
    # roofline of the autotuned solve's products (they run on the FP64 DMMA
    # kernel below the measured crossover): CUDA-event time of the product
    # launches in one profiled (host-driven) solve
    _, pinfo = h.solve(A, X, alpha=alpha, tol=1e-12, prec="fp64_tc", profile=True)
    peaks, src = load_peaks()
    peak64, note64 = dominant_peak("fp64", peaks)
    gemm_s = pinfo["gemm_ms"] * 1e-3
    roof = {"bound": "fp64 (DMMA)", "kernel": "gemm_f64_kernel", "unit": "TFLOP/s",
            "achieved": pinfo["gemm_flops"] / gemm_s / 1e12 if gemm_s > 0 else None, "peak": peak64,
            "frac": pinfo["gemm_flops"] / gemm_s / 1e12 / peak64 if gemm_s > 0 else None,
            "gemm_share_of_solve": pinfo["gemm_ms"] / out["autotuned"]["p50_ms"], "traffic": None,
            "peak_source": f"{src}: {note64}",
            "note": "latency-bound: 48 x 48 x 64 products of a few CTAs each"}
    t0 = time.perf_counter()
    ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    t_cpu = time.perf_counter() - t0
    _emit({"metric": "pseudoinverses/s (64x48, latency-bound)", "value": out["autotuned"]["value"],
           "roofline": roof,
           "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "moore_penrose_64x48", "alpha": alpha, "tol": 1e-12},
           "fp64_tc": out["fp64_tc"], "autotuned": out["autotuned"], "crossover": out["crossover"],
           "cpu_baseline": {"value": 1.0 / t_cpu, "unit": "solves/s", "kind": "oracle", "sample": "full solve",
                            "cores": len(os.sched_getaffinity(0))}})
    h.close()


def _roofline(infos, peaks_prec="bf16"):
    """The dominant kernel's rate over the given solves (profile=True): BF16
    slice-product flops (or FP64 flops for the DMMA path) / CUDA-event time of
    the product kernels, against the measured BF16 sustained peak."""
    peaks, src = load_peaks()
    gemm_ms = sum(i["gemm_ms"] for i in infos)
    if gemm_ms <= 0:
        return None
    fp64 = peaks_prec == "fp64"
    work = sum(i["gemm_flops"] for i in infos) if fp64 else sum(i["tensor_flops"] for i in infos)
    achieved = work / (gemm_ms * 1e-3) / 1e12
    peak, note = dominant_peak("fp64" if fp64 else "fp32", peaks)
    return {"bound": "tensor", "kernel": "gemm_f64_kernel" if fp64 else "tc_gemm_kernel",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "fp64_equivalent_tflops": sum(i["gemm_flops"] for i in infos) / (gemm_ms * 1e-3) / 1e12,
            "traffic": None, "peak_source": f"{src}: {note}",
            "gemm_share_of_step": None}


def run_drazin(args):
    """Drazin inverse of a 2048 x 2048 index-2 matrix (C 1536 x 1536, 256 2x2
    Jordan blocks), X0 = A^2 / Tr(A^3), order-18 stop (step < 1e-2), finish
    A^2 X^5 A^2 + one order-2 step.  The line's value is the refinement form
    (FP32-class loops, X A X, FP64-class order-2 steps, the finish); the loop
    schedule (FP32-class growth loops, then FP64-class loops), every product
    FP64-class on the tensor cores (fp64_tc) and native FP64 (fp64_gpu) are
    timed beside it."""
    import torch
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    d = W.drazin_index2(2048, 512, seed=2)
    B = np.zeros((2048, 2048))
    B[:1536, :1536] = np.linalg.inv(d.C)
    Pinv = np.linalg.inv(d.P)
    rows = np.random.default_rng(0).choice(2048, 32, replace=False)
    ref_rows = d.P[rows] @ B @ Pinv
    A = torch.from_numpy(d.A).cuda()
    X = torch.empty_like(A)
    h = Handle(0)
    st = torch.cuda.current_stream()
    res = {}
    roof = None
    total_ms = None
    for prec in ("fp32_refine", "fp32", "fp64_tc", "fp64"):
        kw = dict(kind="drazin", drazin_index=2, alpha=0.0, tol=1e-2, stop="order18", prec=prec, finish="clean")
        for _ in range(args.warmup if prec != "fp64" else 1):
            h.solve(A, X, **kw)
        times, infos = [], []
        for _ in range(args.steps if prec != "fp64" else 1):
            e0, e1 = _events(st)
            e0.record(st)
            _, info = h.solve(A, X, profile=(prec == "fp32_refine"), **kw)
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        _, cinfo = h.solve(A, X, check=True, **kw)
        err = float(np.linalg.norm(X.cpu().numpy()[rows] - ref_rows) / np.linalg.norm(ref_rows))
        res[prec] = {"value": 1e3 / statistics.mean(times), "ms_per_solve": statistics.mean(times),
                     "loops": info["iters"], "drazin_residuals": cinfo["drazin"], "sampled_rows_rel_err": err,
                     "meets_1e-9": bool(err <= 1e-9 and max(cinfo["drazin"]) <= 1e-9),
                     "loop_classes": ["fp64" if p == 0 else {1: "bf16", 3: "fp32-class", 4: "fp64-class", 5: "fp32-class order-2", 6: "fp64-class order-2"}[p]
                                      for p in info["precision"]],
                     "step_measures": info["history"]}
        if prec == "fp32_refine":
            roof = _roofline(infos)
            total_ms = sum(times)
            if roof:
                roof["gemm_share_of_step"] = sum(i["gemm_ms"] for i in infos) / total_ms
    # the literal spectrum (eigenvalues all around the annulus): X0 = A^2/Tr(A^3)
    # cannot converge there; G = A^l (A^{2l+1})^T A^l does
    dl = W.drazin_index2(2048, 512, seed=2, sector=math.pi)
    Bl = np.zeros((2048, 2048))
    Bl[:1536, :1536] = np.linalg.inv(dl.C)
    ref_l = dl.P[rows] @ Bl @ np.linalg.inv(dl.P)
    Al_ = torch.from_numpy(dl.A).cuda()
    kwl = dict(kind="drazin_normal", drazin_index=2, alpha=0.0, tol=1e-2, stop="order18", prec="fp64_tc",
               finish="clean")
    h.solve(Al_, X, **kwl)
    e0, e1 = _events(st)
    e0.record(st)
    _, il = h.solve(Al_, X, **kwl)
    e1.record(st)
    torch.cuda.synchronize()
    _, cl = h.solve(Al_, X, check=True, **kwl)
    res["annulus_literal"] = {"value": 1e3 / e0.elapsed_time(e1), "ms_per_solve": e0.elapsed_time(e1),
                              "loops": il["iters"], "drazin_residuals": cl["drazin"],
                              "sampled_rows_rel_err": float(np.linalg.norm(X.cpu().numpy()[rows] - ref_l) /
                                                            np.linalg.norm(ref_l)),
                              "x0": "G = A^2 (A^5)^T A^2, alpha = 1/sqrt(||GA||_1 ||GA||_inf)"}
    t0 = time.perf_counter()
    H.hyperpower_step(d.A, H.x0_drazin(d.A, 2), side="right")
    t_loop = time.perf_counter() - t0
    loops = res["fp32"]["loops"] + 2
    _emit({"metric": "Drazin inverses/s at 1e-9 (2048x2048, index 2)",
           "value": res["fp32_refine"]["value"] if res["fp32_refine"]["meets_1e-9"] else 0.0,
           "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "dtype": "bf16 slices (fp32-class loops, fp64-class refinement)",
           "config": {"workload": "drazin_2048_index2", "n_nilpotent": 512, "spectrum": "sector |arg| <= pi/8",
                      "prec": "fp32_refine", "schedule": SCHEDULES["fp32_refine"], "stop": "order18", "tol": 1e-2,
                      "steps": args.steps, "warmup": args.warmup},
           "mixed": res["fp32_refine"], "fp32_loops": res["fp32"], "roofline": roof,
           "fp64_tc": res["fp64_tc"], "fp64_gpu": res["fp64"], "full_annulus_spectrum": res["annulus_literal"],
           "cpu_baseline": {"value": 1.0 / (t_loop * loops), "unit": "solves/s", "kind": "oracle",
                            "cores": len(os.sched_getaffinity(0)),
                            "sample": f"one naive loop ({t_loop:.2f} s) x {loops} loops"}})
    h.close()


def run_batched(args):
    """4096 independent problems, m ~ U{32..512}, n ~ U{16..m}, rank n,
    singular values log-uniform in [1e-3, 1] (Householder-product factors),
    alpha = 1/s_1^2: one pinv_solve_batched call (BF16 bulk loops, FP32-class
    loops, FP32-class projection and last loop: FP32-finished to 1e-4) against
    the FP64 batched path and a sample of per-matrix FP64 solves."""
    import ctypes as C
    import torch
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    from paper_1604_07893_gb300._lib import Desc, Info
    count = args.count
    ws = W.uneven_batch_fast(count, seed=3)
    As = [torch.from_numpy(w.A).cuda() for w in ws]
    Xs = [torch.empty(w.A.shape[1], w.A.shape[0], dtype=torch.float64, device="cuda") for w in ws]
    h = Handle(0)
    st = torch.cuda.current_stream()

    # order-18 stop (R12): the loop whose step is below delta has reached the
    # final class's rounding floor, and its result is kept; delta^18 below the
    # final class's unit roundoff: 0.25 for FP32 class (0.25^18 = 1.5e-11 <
    # 2^-31), 1e-2 for FP64
    def run(prec, tol):
        descs = (Desc * count)(*[h.make_desc(A, X, alpha=1.0 / w.s[0] ** 2, tol=tol, stop="order18", prec=prec,
                                             finish="clean")
                                 for A, X, w in zip(As, Xs, ws)])
        infos = (Info * count)()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = h._lib.pinv_solve_batched(h._h, count, descs, C.c_void_p(st.cuda_stream), infos)
        torch.cuda.synchronize()
        return rc, time.perf_counter() - t0, infos

    run("bf16_fp32", 0.25)     # warm-up (allocations, tensor maps)
    times = []
    for _ in range(args.steps):
        rc, t, infos = run("bf16_fp32", 0.25)
        times.append(t)
    sample = np.random.default_rng(0).choice(count, 64, replace=False)
    errs = [float(np.linalg.norm(Xs[i].cpu().numpy() - (ws[i].V / ws[i].s) @ ws[i].U.T) /
                  np.linalg.norm((ws[i].V / ws[i].s) @ ws[i].U.T)) for i in sample]
    loops = [infos[i].iters for i in range(count)]
    rc64, t64, _ = run("fp64", 1e-2)
    # per-matrix FP64 solves on a sample, extrapolated
    t0 = time.perf_counter()
    for i in sample[:32]:
        h.solve(As[i], Xs[i], alpha=1.0 / ws[i].s[0] ** 2, tol=1e-2, stop="order18", prec="fp64")
    torch.cuda.synchronize()
    per_matrix = (time.perf_counter() - t0) / 32
    t0 = time.perf_counter()
    for i in sample[:8]:
        w = ws[i]
        H.solve(w.A, H.x0_moore_penrose(w.A, 1.0 / w.s[0] ** 2), tol=1e-2, stop=H.STOP_ORDER18,
                alpha=1.0 / w.s[0] ** 2)
    t_cpu = (time.perf_counter() - t0) / 8
    t = statistics.median(times)
    # roofline of the batch: the tensor-core work every instance's products
    # executed (its share of its padded group's launches) over the batch time
    peaks, src = load_peaks()
    tensor = sum(infos[i].tensor_flops for i in range(count))
    fp64eq = sum(infos[i].gemm_flops for i in range(count))
    roof = {"bound": "tensor", "kernel": "tc_gemm_kernel (every product of the batch, padded groups)",
            "achieved": tensor / t / 1e12, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
            "frac": tensor / t / 1e12 / peaks["bf16_tflops_sustained"],
            "fp64_equivalent_tflops": fp64eq / t / 1e12,
            "algorithmic_fp64_equivalent_tflops": sum(
                (4.0 * min(w.A.shape) ** 2 * max(w.A.shape) + 10.0 * min(w.A.shape) ** 3) * infos[i].iters
                for i, w in enumerate(ws)) / t / 1e12,
            "traffic": None, "peak_source": f"{src}: bf16 sustained"}
    _emit({"metric": "pseudoinverses/s, 4096 uneven problems", "value": count / t, "unit": "solves/s",
           "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "bf16 + bf16 slices",
           "config": {"workload": f"uneven_batch_{count}", "m": [32, 512], "n": [16, "m"],
                      "prec": "bf16_fp32 (BF16 growth loops, FP32-class loops, FP32-class projection + order-18 loop)",
                      "stop": "order18", "tol": 0.25,
                      "finish": "clean",
                      "steps": args.steps},
           "ms_per_batch": t * 1e3, "status_ok": sum(1 for i in range(count) if infos[i].status == 0),
           "roofline": roof,
           "loops": {"min": min(loops), "max": max(loops)},
           "accuracy": {"sampled": 64, "max_rel_err_vs_closed_form": max(errs), "meets_1e-4": max(errs) <= 1e-4},
           "fp64_gpu_batched": {"value": count / t64, "s_per_batch": t64, "status": rc64},
           "fp64_gpu_per_matrix_loop": {"value": 1.0 / per_matrix, "sample": "32 single solves"},
           "cpu_baseline": {"value": 1.0 / t_cpu, "unit": "solves/s", "kind": "oracle",
                            "cores": len(os.sched_getaffinity(0)), "sample": "8 sampled problems, full solves"}})
    h.close()


def _serving_stream(h, mats, rate, duration, seed, kw, warm=False):
    """Run a Poisson stream of `rate` requests/s for `duration` seconds through
    pinv_submit / pinv_poll.  Requests pick their size from the workload's mix
    and a pooled matrix of that size; each in-flight request owns an output
    buffer (pooled per size).  Returns per-request records and a backlog trace."""
    import torch
    from paper_1604_07893_gb300 import PinvError, workloads as W
    count = max(1, int(rate * duration))
    sizes = W.serving_sizes(count, seed=seed)
    arrivals = W.poisson_arrivals(rate, count, seed=seed)
    free = {n: [] for n in mats}
    def take(n):
        return free[n].pop() if free[n] else torch.empty(n, n, dtype=torch.float64, device="cuda")
    inflight, done, rejected, trace = {}, [], [], []
    t0 = time.perf_counter()
    nxt, last_trace = 0, -1.0
    while True:
        now = time.perf_counter() - t0
        while nxt < count and arrivals[nxt] <= now:
            n = int(sizes[nxt])
            A, G = mats[n][nxt % len(mats[n])]
            X = take(n)
            try:
                rid = h.submit(A, X, G=G, **kw)
                inflight[rid] = (nxt, n, X, arrivals[nxt])
            except PinvError as e:
                if e.code != -9:
                    raise
                rejected.append(nxt)
                free[n].append(X)
            nxt += 1
        if nxt >= count and not inflight:
            break
        for rid in list(inflight):
            r = h.poll(rid)
            if r is not None:
                i, n, X, ta = inflight.pop(rid)
                done.append({"i": i, "n": n, "t_done": time.perf_counter() - t0, "t_arrive": ta,
                             "status": r[0], "ms": r[1]["ms"], "iters": r[1]["iters"],
                             "tensor_flops": r[1]["tensor_flops"], "gemm_flops": r[1]["gemm_flops"]})
                free[n].append(X)
        if now - last_trace >= 0.1:
            st = h.serving_stats()
            trace.append((now, st["queued"], st["running"]))
            last_trace = now
        if not inflight:
            time.sleep(0.0002)
    return {"count": count, "done": done, "rejected": rejected, "trace": trace,
            "elapsed": time.perf_counter() - t0}


def _serving_summary(res, duration, peak):
    lo, hi = 0.2 * duration, duration        # steady window: after the ramp, before the drain
    win = [d for d in res["done"] if lo <= d["t_done"] <= hi and d["status"] == 0]
    lat = [d["ms"] for d in win]
    by_size = {}
    for d in win:
        by_size.setdefault(d["n"], []).append(d["ms"])
    tensor = sum(d["tensor_flops"] for d in win)
    fp64 = sum(d["gemm_flops"] for d in win)
    span = hi - lo
    trace = [t for t in res["trace"] if lo <= t[0] <= hi]
    return {
        "offered": res["count"], "completed": len(res["done"]), "rejected": len(res["rejected"]),
        "failed": sum(1 for d in res["done"] if d["status"] != 0),
        "steady_window_s": [lo, hi], "completed_in_window": len(win),
        "solves_per_s": len(win) / span,
        "latency_ms": {"p50": statistics.median(lat) if lat else None, "p99": _pct(lat, 0.99) if lat else None,
                       "by_size": {str(n): {"count": len(v), "p50_ms": statistics.median(v),
                                            "p99_ms": _pct(v, 0.99)} for n, v in sorted(by_size.items())}},
        "backlog": {"queued_mean": statistics.mean([t[1] for t in trace]) if trace else None,
                    "queued_max": max([t[1] for t in trace]) if trace else None,
                    "queued_end": res["trace"][-1][1] if res["trace"] else None,
                    "running_mean": statistics.mean([t[2] for t in trace]) if trace else None},
        "roofline": {"bound": "tensor", "kernel": "tc_gemm_kernel (all products of the window)",
                     "achieved": tensor / span / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": tensor / span / 1e12 / peak, "fp64_equivalent_tflops": fp64 / span / 1e12,
                     "traffic": None},
        "drain_s": res["elapsed"] - duration,
    }


def run_serving(args):
    """Steady-state serving of approximate-inverse preconditioner requests for
    SPD A = Q diag(lambda) Q^T (lambda log-spaced in [1e-3, 1]), n in {256 ...
    8192} with weights 40/25/15/10/7/3 %, G = I, alpha = 1/lambda_max, BF16
    growth loops then FP32-class (FP32-finished to 1e-4), under a 120 GB HBM
    budget and an admission queue of at most 32 waiting requests.

    Phase 1: a Poisson stream at the offered 2000 requests/s for --duration
    seconds (default 10): the offered load exceeds what one GPU serves, the
    library rejects what does not fit the admission queue (PINV_ERR_BUSY), and
    the line reports completions/s over the steady window (the last 80 % of the
    arrival period), p50/p99 latency (submit to result) of those requests,
    rejections and the backlog.  Phase 2: a stream at 80 % of the measured
    service rate for the same duration (sustainable: the backlog stays
    bounded).  Matrices: one pooled matrix per size (two for n <= 1024); each
    in-flight request has its own output buffer."""
    import torch
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    duration = args.duration
    h = Handle(0, hbm_budget_bytes=120 << 30, max_queued=32)
    mats, spd = {}, {}
    for n in (256, 512, 1024, 2048, 4096, 8192):
        mats[n] = []
        for k in range(2 if n <= 1024 else 1):
            Q, lam = W.spd_fast(n, seed=100 + 7 * n + k)
            Qd = torch.from_numpy(Q).cuda()
            A = h.gemm(Qd * torch.from_numpy(lam).cuda(), Qd, trans_b=True, prec="fp64_tc")
            A = (0.5 * (A + A.T)).contiguous()
            mats[n].append((A, torch.eye(n, dtype=torch.float64, device="cuda")))
            if k == 0:
                spd[n] = (Q, lam)
    torch.cuda.synchronize()
    kw = dict(kind="outer_g", alpha=1.0, tol=1e-6, prec="bf16_fp32", symmetric=True)
    # warm-up (untimed): every size alone, then a short stream, so the
    # stream-ordered pool has grown to what the timed streams need
    for n in mats:
        h.solve(mats[n][0][0], G=mats[n][0][1], **kw)
    _serving_stream(h, mats, 200.0, 1.0, seed=4, kw=kw)
    peaks, src = load_peaks()
    peak = peaks["bf16_tflops_sustained"]
    res1 = _serving_stream(h, mats, 2000.0, duration, seed=5, kw=kw)
    s1 = _serving_summary(res1, duration, peak)
    rate2 = max(1.0, 0.8 * s1["solves_per_s"])
    res2 = _serving_stream(h, mats, rate2, duration, seed=6, kw=kw)
    s2 = _serving_summary(res2, duration, peak)
    # accuracy: one request of each size against A^-1 (the last results in the pooled buffers are
    # overwritten, so solve one of each size again)
    errs = {}
    for n, (Q, lam) in spd.items():
        X, info = h.solve(mats[n][0][0], G=mats[n][0][1], **kw)
        inv = (Q / lam) @ Q.T
        errs[str(n)] = float(np.linalg.norm(X.cpu().numpy() - inv) / np.linalg.norm(inv))
    # CPU baseline: the oracle as it stands on a stratified sample -- full
    # solves at n = 256 and 512, one naive loop at n = 1024 scaled by n^3 to
    # the larger sizes -- weighted by the size mix and the loop counts the GPU ran
    loops = {}
    for d in res1["done"] + res2["done"]:
        loops.setdefault(d["n"], []).append(d["iters"])
    mean_loops = {n: statistics.mean(v) for n, v in loops.items()}
    cpu_s = {}
    for n in (256, 512):
        A = mats[n][0][0].cpu().numpy()
        t0 = time.perf_counter()
        H.solve(A, np.eye(n), tol=1e-6, alpha=1.0)
        cpu_s[n] = time.perf_counter() - t0
    A = mats[1024][0][0].cpu().numpy()
    t0 = time.perf_counter()
    H.hyperpower_step(A, np.eye(1024))
    t_loop = time.perf_counter() - t0
    weights = {256: 0.40, 512: 0.25, 1024: 0.15, 2048: 0.10, 4096: 0.07, 8192: 0.03}
    per_req = sum(w * (cpu_s[n] if n in cpu_s else t_loop * (n / 1024) ** 3 * mean_loops.get(n, 4.0))
                  for n, w in weights.items())
    _emit({"metric": "preconditioner solves/s under continuous batching (steady state), p50/p99 latency",
           "value": s1["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
           "data": "synthetic", "dtype": "bf16 + bf16 slices (fp32-class)",
           "config": {"workload": "serving_spd_poisson2000", "sizes": [256, 512, 1024, 2048, 4096, 8192],
                      "weights": [0.40, 0.25, 0.15, 0.10, 0.07, 0.03], "hbm_budget_gb": 120, "max_queued": 32,
                      "tol": 1e-6, "prec": "bf16_fp32 (BF16 growth loops, FP32-class to the end)",
                      "symmetric": True, "duration_s": duration},
           "offered_2000_per_s": s1, "sustainable": {"rate": rate2, **s2},
           "latency_ms": s1["latency_ms"], "roofline": s1["roofline"],
           "accuracy": {"max_rel_err_vs_inverse_by_size": errs, "meets_1e-4": max(errs.values()) <= 1e-4},
           "cpu_baseline": {"value": 1.0 / per_req, "unit": "solves/s", "kind": "oracle",
                            "cores": len(os.sched_getaffinity(0)),
                            "sample": (f"full oracle solves at n=256 ({cpu_s[256]:.2f} s) and n=512 "
                                       f"({cpu_s[512]:.2f} s), one naive loop at n=1024 ({t_loop:.2f} s) scaled "
                                       f"by n^3 and the GPU's loop counts to 2048..8192, weighted by the size mix")}})
    h.close()


def run_complex(args):
    """Moore-Penrose inverse of a complex rank-deficient 2048 x 1536 matrix
    (A = U diag(s) V^*, Haar unitary U, V of rank 1152, s log-spaced in
    [1e-4, 1]) with the headline settings (the refinement schedule, alpha =
    1/s_1^2); the library solves the 4096 x 3072 real embedding with half-width
    (four real products per complex product) tensor-core products.  The
    FP64-class schedule (every product FP64 class, alpha = 2/(s_1^2 + s_r^2))
    is timed beside it."""
    import torch
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    m, n, r = 2048, 1536, 1152
    w = W.rectangular_complex(m, n, r, 1.0, 1e-4, seed=SEED)
    alpha = 1.0 / w.s[0] ** 2
    A = torch.from_numpy(w.A).cuda()
    X = torch.empty((n, m), dtype=torch.complex128, device="cuda")
    h = Handle(0)
    st = torch.cuda.current_stream()
    kw = solve_kwargs("fp32_refine", alpha)
    for _ in range(args.warmup):
        h.solve_complex(A, X, **kw)
    torch.cuda.synchronize()
    infos = []
    with ClockSampler(0) as clk:
        e0, e1 = _events(st)
        e0.record(st)
        for _ in range(args.steps):
            _, info = h.solve_complex(A, X, profile=True, **kw)
            infos.append(info)
        e1.record(st)
        torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    rows = np.random.default_rng(0).choice(n, 32, replace=False)
    ref_rows = (w.V[rows] / w.s) @ w.U.conj().T
    row_err = float(np.linalg.norm(X.cpu().numpy()[rows] - ref_rows) / np.linalg.norm(ref_rows))
    _, cinfo = h.solve_complex(A, X, check=True, **kw)
    ok = max(cinfo["penrose"]) <= 1e-9 and row_err <= 1e-9
    A_pin = torch.from_numpy(w.A).pin_memory()
    X_pin = torch.empty((n, m), dtype=torch.complex128).pin_memory()
    h.solve_complex(A_pin.numpy(), X_pin.numpy(), host=True, **kw)
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        h.solve_complex(A_pin.numpy(), X_pin.numpy(), host=True, **kw)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    # the FP64-class schedule beside it
    kw64 = solve_kwargs("fp64_tc", 2.0 / (w.s[0] ** 2 + w.s[-1] ** 2))
    kw64["switch_tol"] = 0.5
    h.solve_complex(A, X, **kw64)
    torch.cuda.synchronize()
    f0, f1 = _events(st)
    f0.record(st)
    for _ in range(3):
        _, i64 = h.solve_complex(A, X, **kw64)
    f1.record(st)
    torch.cuda.synchronize()
    _, c64 = h.solve_complex(A, X, check=True, **kw64)
    ms64 = f0.elapsed_time(f1) / 3
    fp64_arm = {"value": 1e3 / ms64, "unit": UNIT, "ms_per_solve": ms64, "loops": i64["iters"],
                "stabilized_loops": i64["stabilized_loops"], "penrose_max": max(c64["penrose"]),
                "alpha": "2/(s_1^2 + s_r^2)", "switch_tol": 0.5}
    peaks, peak_src = load_peaks()
    peak, peak_note = dominant_peak("fp32_refine", peaks)
    gemm_ms = sum(i["gemm_ms"] for i in infos)
    achieved = sum(i["tensor_flops"] for i in infos) / (gemm_ms * 1e-3) / 1e12
    complex_flops = sum(i["gemm_flops"] for i in infos)   # 8 mnk real flops per complex product
    cpu = None
    if not args.no_cpu:
        t0 = time.perf_counter()
        H.hyperpower_step(w.A, H.x0_moore_penrose(w.A, alpha), side="left")
        t_loop = time.perf_counter() - t0
        loops = i64["iters"] + 1
        cpu = {"value": 1.0 / (t_loop * loops), "unit": UNIT, "kind": "oracle",
               "cores": len(os.sched_getaffinity(0)),
               "sample": f"one naive complex loop of the full problem ({t_loop:.2f} s) x {loops} "
                         "(the oracle's loops + the cleanup)"}
    _emit({"metric": "complex pseudoinverses/s at 1e-9 Penrose residual", "value": args.steps / (total_ms * 1e-3) if ok else 0.0,
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": total_ms / args.steps, "higher_is_better": True, "vs_baseline": None,
           "dtype": "bf16 slices (fp32-class loops, fp64-class refinement), complex as real embedding",
           "data": "synthetic",
           "config": {"workload": "moore_penrose_complex_rank_deficient_2048x1536_r1152", "m": m, "n": n,
                      "rank": r, "s_range": [1e-4, 1.0], "alpha": "1/s_1^2", "prec": "fp32_refine",
                      "schedule": SCHEDULES["fp32_refine"], "variant": "stabilized",
                      "switch_tol": SWITCH_TOL, "stop": "order18", "tol": 1e-2, "finish": "clean",
                      "l2": "inputs larger than L2 (A 50 MB complex, embedding 100 MB)"},
           "accuracy": {"penrose_max": max(cinfo["penrose"]), "sampled_rows_rel_err": row_err, "meets_1e-9": ok,
                        "loops": infos[-1]["iters"], "stabilized_loops": infos[-1]["stabilized_loops"],
                        "loop_classes": [{3: "fp32-class", 4: "fp64-class", 5: "fp32-class order-2",
                                          6: "fp64-class order-2"}.get(p, str(p)) for p in infos[-1]["precision"]]},
           "e2e": {"value": 1.0 / e2e_s if ok else 0.0, "unit": UNIT, "h2d_bytes_per_step": m * n * 16,
                   "d2h_bytes_per_step": n * m * 16},
           "gpu_launches": sum(i["kernels"] for i in infos),
           "roofline": {"bound": "tensor", "kernel": "tc_gemm_kernel", "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                        "complex_equivalent_fp64_tflops": complex_flops / (gemm_ms * 1e-3) / 1e12,
                        "peak_source": f"{peak_src}: {peak_note}",
                        "gemm_share_of_step": gemm_ms / total_ms},
           "clocks": clk.summary(), "cpu_baseline": cpu, "fp64_tc": fp64_arm})
    h.close()


def run_precond(args):
    """Approximate-inverse preconditioners (Section 8, Example 3): one loop of
    Eq. PM from the Jacobi X0 = diag(1/a_ii), chop 1e-5, for complex shifted
    five-point grid operators -- n = 841 (a 29 x 29 grid, the size of the
    paper's example; latency-bound) and n = 4096 (a 64 x 64 grid)."""
    import torch
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    h = Handle(0)
    st = torch.cuda.current_stream()
    crossover = h.autotune()
    out = {}
    for k, precs in ((29, ("fp64_tc",)), (64, ("fp64_tc", "fp32"))):
        A_np = W.grid_operator(k, seed=7)
        n = k * k
        A = torch.from_numpy(A_np).cuda()
        X = torch.empty_like(A)
        I = torch.eye(n, dtype=A.dtype, device=A.device)
        for prec in precs:
            kw = dict(loops=1, chop=1e-5, prec=prec)
            for _ in range(args.warmup):
                h.preconditioner(A, X, **kw)
            torch.cuda.synchronize()
            lat, infos = [], []
            for _ in range(max(args.steps, 20 if n < 1000 else 3)):
                e0, e1 = _events(st)
                e0.record(st)
                _, info = h.preconditioner(A, X, profile=True, **kw)
                e1.record(st)
                torch.cuda.synchronize()
                lat.append(e0.elapsed_time(e1))
                infos.append(info)
            resid = float(torch.linalg.matrix_norm(I - X @ A).item()) / math.sqrt(n)
            gemm_ms = sum(i["gemm_ms"] for i in infos)
            peaks, _ = load_peaks()
            peak, _ = dominant_peak(prec, peaks)
            tflops = sum(i["tensor_flops"] for i in infos) / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
            out[f"n{n}_{prec}"] = {"value": 1e3 / statistics.mean(lat), "p50_ms": statistics.median(lat),
                                   "p99_ms": _pct(lat, 0.99), "kernels": infos[-1]["kernels"],
                                   "fro_I_minus_XA_over_sqrt_n": resid,
                                   "nonzero_fraction": float((torch.view_as_real(X) != 0).double().mean().item()),
                                   "tc_tflops": tflops, "tc_frac": (tflops / peak) if tflops else None}
    A841 = W.grid_operator(29, seed=7)
    t0 = time.perf_counter()
    H.preconditioner(A841, loops=1, chop_eps=1e-5)
    t841 = time.perf_counter() - t0
    _emit({"metric": "preconditioners/s (one PM loop from Jacobi, chop 1e-5)", "value": out["n841_fp64_tc"]["value"],
           "unit": "preconditioners/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "dtype": "bf16 slices (fp64-/fp32-class), complex as real embedding",
           "config": {"workload": "jacobi_pm1_preconditioner_complex_grid", "sizes": [841, 4096], "loops": 1,
                      "chop": 1e-5, "operator": "shifted five-point grid, complex, 5% jitter",
                      "steps": args.steps, "warmup": args.warmup},
           "engine_crossover": crossover, "results": out,
           "cpu_baseline": {"value": 1.0 / t841, "unit": "preconditioners/s", "kind": "oracle",
                            "cores": len(os.sched_getaffinity(0)), "sample": "full n = 841 preconditioner"}})
    h.close()


def run_weighted(args):
    """Weighted Moore-Penrose inverse A^+_{MN} of a rank-deficient 2048 x 1536
    matrix (rank 1152, s log-spaced in [1e-4, 1]) through G = N^{-1} A^T M,
    M, N positive definite (eigenvalues log-spaced in [0.2, 5] and [0.5, 2]):
    the general-G alpha recipe, FP64-class products, stabilised after a step
    below 0.5, order-18 stop, X A X finish."""
    import torch
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    m, n, r = 2048, 1536, 1152
    w = W.rectangular(m, n, r, 1.0, 1e-4, seed=SEED)
    Ms, Ns = W.spd(m, 0.2, 5.0, seed=SEED + 1), W.spd(n, 0.5, 2.0, seed=SEED + 2)
    G_np = np.ascontiguousarray((Ns.Q / Ns.lam) @ Ns.Q.T @ w.A.T @ Ms.A)
    A = torch.from_numpy(w.A).cuda()
    G = torch.from_numpy(G_np).cuda()
    X = torch.empty((n, m), dtype=torch.float64, device="cuda")
    h = Handle(0)
    st = torch.cuda.current_stream()
    kw = dict(kind="outer_g", G=G, alpha=0.0, tol=1e-2, stop="order18", prec="fp64_tc", variant="stabilized",
              switch_tol=0.5, finish="clean")
    for _ in range(args.warmup):
        h.solve(A, X, **kw)
    torch.cuda.synchronize()
    infos = []
    with ClockSampler(0) as clk:
        e0, e1 = _events(st)
        e0.record(st)
        for _ in range(args.steps):
            _, info = h.solve(A, X, profile=True, **kw)
            infos.append(info)
        e1.record(st)
        torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    # accuracy: sampled rows against N^{-1/2} (M^{1/2} A N^{-1/2})^+ M^{1/2}, from its
    # SVD (rank r), and the two weighted symmetry conditions on the device result
    Mh = (Ms.Q * np.sqrt(Ms.lam)) @ Ms.Q.T
    Nmh = (Ns.Q / np.sqrt(Ns.lam)) @ Ns.Q.T
    U, sv, Vt = np.linalg.svd(Mh @ w.A @ Nmh, full_matrices=False)
    rows = np.random.default_rng(0).choice(n, 32, replace=False)
    ref_rows = ((Nmh[rows] @ Vt[:r].T) / sv[:r]) @ (U[:, :r].T @ Mh)
    Xh = X.cpu().numpy()
    row_err = float(np.linalg.norm(Xh[rows] - ref_rows) / np.linalg.norm(ref_rows))
    ok = row_err <= 1e-9
    peaks, peak_src = load_peaks()
    peak, peak_note = dominant_peak("fp64_tc", peaks)
    gemm_ms = sum(i["gemm_ms"] for i in infos)
    achieved = sum(i["tensor_flops"] for i in infos) / (gemm_ms * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu:
        a = H.alpha_general(w.A, G_np)
        t0 = time.perf_counter()
        H.hyperpower_step(w.A, H.x0_general(G_np, a), side="left")
        t_loop = time.perf_counter() - t0
        loops = infos[-1]["iters"] + 1
        cpu = {"value": 1.0 / (t_loop * loops), "unit": UNIT, "kind": "oracle",
               "cores": len(os.sched_getaffinity(0)),
               "sample": f"one naive loop of the full problem ({t_loop:.2f} s) x {loops}"}
    _emit({"metric": "weighted pseudoinverses/s at 1e-9", "value": args.steps / (total_ms * 1e-3) if ok else 0.0,
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": total_ms / args.steps, "higher_is_better": True, "vs_baseline": None,
           "dtype": "bf16 slices (fp64-class)", "data": "synthetic",
           "config": {"workload": "weighted_moore_penrose_2048x1536_r1152", "M_eigs": [0.2, 5.0],
                      "N_eigs": [0.5, 2.0], "alpha": "general-G recipe", "prec": "fp64_tc",
                      "variant": "stabilized", "stop": "order18", "tol": 1e-2, "finish": "clean (X A X)"},
           "accuracy": {"sampled_rows_rel_err": row_err, "meets_1e-9": ok, "loops": infos[-1]["iters"],
                        "alpha": infos[-1]["alpha"]},
           "gpu_launches": sum(i["kernels"] for i in infos),
           "roofline": {"bound": "tensor", "kernel": "tc_gemm_kernel", "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                        "peak_source": f"{peak_src}: {peak_note}", "gemm_share_of_step": gemm_ms / total_ms},
           "clocks": clk.summary(), "cpu_baseline": cpu})
    h.close()


# Section 8, Example 2 (Tables 2-4): PM wall time in seconds on the paper's
# machine (Mathematica, Core i5-2430M) for H_{m x (m-10)}, m = 100 ... 1000.
PAPER_HILBERT_S = {
    1e-5: [0.047003, 0.211012, 0.388023, 0.941054, 1.611092, 2.505143, 3.645208, 5.113292, 6.872393, 9.012523],
    1e-6: [0.045003, 0.190011, 0.337019, 0.794045, 1.318075, 2.067118, 3.057175, 4.269244, 5.784331, 7.553432],
    1e-7: [0.051003, 0.227013, 0.406023, 0.942054, 1.599092, 2.471141, 3.651209, 5.044289, 6.890394, 9.177525],
}


def run_hilbert(args):
    """Section 8, Example 2: Moore-Penrose inverses of the Hilbert matrices
    H_{m x (m-10)}, m = 100 ... 1000, X0 = 2/(s_1^2 + s_r^2) H^T (s_r the smallest
    singular value above 1e-15 s_1), stop rule of Eq. stopreliable with the
    Frobenius norm at eps = 1e-5, 1e-6, 1e-7 -- the paper's own timing
    workload (Tables 2-4), timed per solve with CUDA events (autotuned engine:
    small products on DMMA, the rest FP64-class on the tensor cores)."""
    import torch
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    h = Handle(0)
    st = torch.cuda.current_stream()
    crossover = h.autotune()
    table = {}
    checks = {}
    for eps in (1e-5, 1e-6, 1e-7):
        rows = []
        for i, m in enumerate(range(100, 1001, 100)):
            Hm = W.hilbert(m, m - 10)
            s = np.linalg.svd(Hm, compute_uv=False)
            s_r = s[s > 1e-15 * s[0]][-1]
            alpha = 2.0 / (s[0] ** 2 + s_r ** 2)
            A = torch.from_numpy(Hm).cuda()
            X = torch.empty((m - 10, m), dtype=torch.float64, device="cuda")
            kw = dict(alpha=alpha, tol=eps, stop="paper", prec="fp64_tc")
            for _ in range(max(1, args.warmup)):
                h.solve(A, X, **kw)
            lat = []
            for _ in range(max(3, args.steps)):
                e0, e1 = _events(st)
                e0.record(st)
                _, info = h.solve(A, X, **kw)
                e1.record(st)
                torch.cuda.synchronize()
                lat.append(e0.elapsed_time(e1))
            ms = statistics.median(lat)
            paper_s = PAPER_HILBERT_S[eps][i]
            rows.append({"m": m, "n": m - 10, "ms": ms, "loops": info["iters"], "paper_s": paper_s,
                         "speedup_vs_paper": paper_s * 1e3 / ms})
            if eps == 1e-5 and m in (100, 500):   # the oracle's loop count and iterate
                ref, oinfo = H.solve(Hm, H.x0_moore_penrose(Hm, alpha), tol=eps, stop=H.STOP_PAPER, alpha=alpha)
                checks[f"H{m}x{m - 10}"] = {"loops": info["iters"], "oracle_loops": oinfo.iters,
                                            "rel_diff_vs_oracle": float(np.linalg.norm(X.cpu().numpy() - ref) /
                                                                        np.linalg.norm(ref))}
        table[f"{eps:g}"] = rows
    last = table["1e-05"][-1]
    _emit({"metric": "ms per Moore-Penrose solve of H_{1000x990} (Example 2, eps = 1e-5)", "value": last["ms"],
           "unit": "ms", "n_gpus": 1, "higher_is_better": False,
           "vs_baseline": last["ms"] / (last["paper_s"] * 1e3),
           "baseline_note": "the paper's Table 2 time on its own machine (Mathematica, Core i5-2430M): context",
           "dtype": "bf16 slices (fp64-class) / f64", "data": "synthetic (Hilbert matrices, as printed)",
           "config": {"workload": "hilbert_example2", "sizes": "H_{m x (m-10)}, m = 100..1000",
                      "x0": "2/(s1^2 + sr^2) H^T", "stop": "paper (Eq. stopreliable, Frobenius)",
                      "eps": [1e-5, 1e-6, 1e-7], "engine_crossover": crossover},
           "tables": table, "oracle_checks": checks})
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32_refine", choices=["fp32_refine", "fp32", "fp64_tc", "fp64", "mixed_bf16"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--workload", default="mp4096x3072",
                    choices=["mp4096x3072", "mp64x48", "drazin2048", "batched4096", "serving", "complex2048x1536",
                             "precond", "weighted", "hilbert"])
    ap.add_argument("--count", type=int, default=None, help="instances (batched)")
    ap.add_argument("--duration", type=float, default=10.0, help="seconds of arrivals per serving phase")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mp64x48":
        return run_mp64(args)
    if args.workload == "drazin2048":
        return run_drazin(args)
    if args.workload == "complex2048x1536":
        return run_complex(args)
    if args.workload == "precond":
        return run_precond(args)
    if args.workload == "weighted":
        return run_weighted(args)
    if args.workload == "hilbert":
        return run_hilbert(args)
    if args.workload == "batched4096":
        args.count = args.count or 4096
        return run_batched(args)
    if args.workload == "serving":
        args.count = args.count or 64
        return run_serving(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
