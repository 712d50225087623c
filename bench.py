#!/usr/bin/env python
"""Benchmark of the batched Walk-on-Spheres hot path on one GB300 (or N replicas).

Workload (one "step"): the batched uneven configuration -- 256 independent problems with
d in {3..12}, 16-4096 ball obstacles (radii log-uniform 0.01-0.2) in [-1,1]^d, sigma in [0,50],
256-16384 walks per query and 64 queries per problem; u and grad u at every query; one
persistent launch replayed from a CUDA graph with autotuned launch shape; FP32 walkers, FP64
per-query sums. Inputs are resident in HBM before timing; L2 (129 MB) is flushed between steps.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on a bounded sample
of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("WoS walk-steps/s and ∇u queries/s at stated RMSE vs FP64 oracle; "
          "mixed vs plain FP32")
WORKLOAD = ("batched uneven: 256 problems, d U{3..12}, 16-4096 balls (r log-U[0.01,0.2]) in [-1,1]^d, "
            "sigma U[0,50], 256-16384 walks/query, 64 queries/problem, eps 1e-3, u + grad u")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-secondary", action="store_true")
    p.add_argument("--no-cv", action="store_true",
                   help="the paper's first-sphere gradient without the control variate")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target CPU-baseline sample time (0 skips it: profiling runs only)")
    p.add_argument("--problems", type=int, default=256,
                   help="leading problems of the workload (fewer: the small profiling case)")
    p.add_argument("--scale-walks", type=float, default=1.0,
                   help="scale of the walk counts (below 1: the small profiling case)")
    p.add_argument("--launch", default=None,
                   help="explicit launch shape threads,ctas_per_sm,item_work[,sphere_ctas_per_sm,sphere_item_walks] "
                        "(skips the autotuner)")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base_seed, rank):
    """Walk seed of a replica: ranks draw disjoint random streams (independent estimates)."""
    return base_seed + 1000003 * rank


def aggregate_over_ranks(seconds, units, world, device="cpu"):
    """Replica aggregation: the job takes as long as its slowest rank and processes the units of
    all ranks. Returns (max seconds over ranks, total units, value = total units / max seconds).
    With world == 1 no process group is used."""
    if world <= 1:
        return seconds, units, units / seconds
    import torch
    import torch.distributed as dist

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0]), float(u[0]) / float(t[0])


def sphere_queue_class(d, tiles):
    """The batch's queue class of a tensor-core sphere set (its launches are one per dimension and
    class): 2 for 32-column sets (128 or more tiles of 64 spheres in d <= 8), 1 for 24 or more
    tiles, 0 below."""
    return 2 if (d <= 8 and tiles >= 128) else (1 if tiles >= 24 else 0)


KERNEL_SOURCES = ["paper_2406_01713_gb300/csrc/walk_mixed.cuh", "paper_2406_01713_gb300/csrc/wos_device.cuh",
                  "paper_2406_01713_gb300/csrc/wos_launch.h"]
TRAFFIC_PROFILE = "profiles/walk_mixed_batched_traffic.txt"
SPHERE_SOURCES = ["paper_2406_01713_gb300/csrc/sphere_kernel.cuh", "paper_2406_01713_gb300/csrc/pointcloud.cu"] + KERNEL_SOURCES
SPHERE_TRAFFIC_PROFILE = "profiles/sphere_kernel_batched_traffic.txt"


def measured_traffic(profile=TRAFFIC_PROFILE, sources=KERNEL_SOURCES):
    """DRAM bytes (read + write) from a committed ncu summary, or None when the kernel sources
    changed since that capture."""
    import hashlib

    try:
        h = hashlib.sha256()
        for f in sources:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        vals = {}
        for line in open(os.path.join(ROOT, profile)):
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            vals[k] = v
        if vals.get("kernel_sources_sha256") != h.hexdigest():
            return None
        return int(vals["dram_bytes_read"]) + int(vals["dram_bytes_write"])
    except (OSError, ValueError, KeyError):
        return None


def alg_flops_per_step(d, n_balls, n_points=0):
    """Algorithmic FP32 flops of one walk step (one distance evaluation): the ball screen
    costs 2d+3 flops per ball (d FMAs of x.m, the b-term FMA and the threshold add), a point
    2d+1 (d FMAs and the compare), the box faces and sampling about 4d."""
    return n_balls * (2 * d + 3) + n_points * (2 * d + 1) + 4 * d


def contraction_k(d):
    """Columns of the tensor-core walker's BF16-split contraction (3d + 2, padded to 32 or 48)."""
    return 32 if 3 * d + 2 <= 32 else 48


def domain_sizes(dom):
    return (dom["ball_r"].size if "ball_r" in dom else 0), (dom["points"].shape[0] if "points" in dom else 0)


FP32_LANES_PER_SM = 128


def fp32_peak_tflops(sms, sm_mhz):
    """FP32 FMA pipe: SMs x 128 lanes x 2 flops x SM clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (nominal: the measured-peaks file holds no FP64 figure)


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [t.strip() for t in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s, p in zip(sm, power) if p is not None and power and p > 0.3 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------------------ oracle sample
def oracle_sample(problems, seed, target_seconds, cv=True, threads=None):
    """The FP64 oracle on a bounded sample of the batched workload: the first `nq` queries of
    each problem (problems in a seeded shuffled order), min(N, 64) gradient walks per query,
    until about target_seconds. The oracle threads over queries, so nq = host cores keeps every
    core busy (threads = 1: the same queries on one core). Returns (walk_steps, seconds, threads
    used, description)."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    nq = min(cores, 64)
    threads = threads or cores
    order = np.random.default_rng(7).permutation(len(problems))
    steps = 0
    used = 0
    t0 = time.perf_counter()
    for i in order:
        p = problems[i]
        n = min(p["n_walks"], 64)
        r = oracle.solve(p["domain"], p["X"][:nq], n, p["eps"], p["sigma"], seed, grad=True, threads=threads,
                         control_variate=cv)
        steps += int(r["walk_steps"].sum())
        used += 1
        if time.perf_counter() - t0 > target_seconds:
            break
    dt = time.perf_counter() - t0
    desc = ("FP64 oracle (plain C, pthreads over queries), %d queries x min(N,64) gradient walks of each of %d "
            "of the 256 problems (seeded order)" % (nq, used))
    return steps, dt, min(threads, nq), desc


def run_reference(args, rank, world):
    from paper_2406_01713_gb300 import synth

    if rank != 0:
        return
    w = synth.c4()
    per_step = max(2.0, args.cpu_seconds / 3.0)
    for _ in range(args.warmup):
        oracle_sample(w["problems"], w["seed"], per_step / 4, not args.no_cv)
    tot_steps, tot_t, threads, desc = 0, 0.0, 1, ""
    for _ in range(args.steps):
        s, t, threads, desc = oracle_sample(w["problems"], w["seed"], per_step, not args.no_cv)
        tot_steps += s
        tot_t += t
    v = tot_steps / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "walk-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": v, "unit": "walk-steps/s", "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": "walk-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ ours
def log(*a):
    print("[bench %.1fs]" % (time.perf_counter() - T0), *a, file=sys.stderr, flush=True)


T0 = time.perf_counter()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import paper_2406_01713_gb300 as pkg
    from paper_2406_01713_gb300 import synth
    from paper_2406_01713_gb300 import wos as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    pkg.build()
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    w = synth.c4(n_problems=args.problems, scale_walks=args.scale_walks)
    probs = w["problems"]
    doms = [W.Domain(p["domain"]) for p in probs]
    workload = WORKLOAD if (args.problems == 256 and args.scale_walks == 1.0) else (
        "SMALL CASE (profiling): first %d problems of [%s], walks x %g" % (args.problems, WORKLOAD, args.scale_walks))
    launch = None
    if args.launch:
        v = [int(t) for t in args.launch.split(",")]
        launch = {"threads": v[0], "ctas_per_sm": v[1], "item_work": v[2]}
        if len(v) == 5:
            launch.update({"sphere_ctas_per_sm": v[3], "sphere_item_walks": v[4]})
        args.no_autotune = True
    batch = W.Batch([{"domain": d, "x": p["X"], "n_walks": p["n_walks"], "eps": p["eps"], "sigma": p["sigma"],
                      "grad": True} for d, p in zip(doms, probs)], seed=replica_seed(w["seed"], rank),
                    config=launch, control_variate=not args.no_cv)
    cache = os.environ.get("WOS_AUTOTUNE_CACHE",
                           os.path.join(ROOT, "paper_2406_01713_gb300", "csrc", "_build", "autotune_cache.txt"))
    log("workload ready: %d problems" % len(probs))
    tuned = batch.autotune(cache) if not args.no_autotune else batch.config()
    log("launch shape", tuned)
    if not args.no_autotune and os.path.exists(cache):
        log("autotune candidates:\n" + "".join(l for l in open(cache) if l.startswith("#"))[-2000:])
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    # per-problem algorithmic flops per launch (walk steps are deterministic for a seed)
    steps_pq = [int(o["walk_steps"].sum()) for o in batch.out]
    total_steps = int(W.stats_dict(batch.stats)["walk_steps"])
    assert total_steps == sum(steps_pq)
    flops = sum(s * alg_flops_per_step(p["domain"]["d"], p["domain"]["ball_r"].size) for s, p in zip(steps_pq, probs))
    total_q = sum(p["X"].shape[0] for p in probs)

    sampler = ClockSampler(dev)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # L2 flush between steps (512 MB > 129 MB L2)
        ev[i][0].record(stream)
        batch.run()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    log("timed steps (ms)", [round(x, 2) for x in step_ms])
    dev_s, _, value = aggregate_over_ranks(sum(step_ms) / 1e3, total_steps * args.steps, world, device="cuda")
    ms_per_step = 1e3 * dev_s / args.steps

    # run-to-run spread of the FP64 sums (atomics land in a different order each run)
    u_a = batch.u_buf.clone()
    batch.run()
    torch.cuda.synchronize()
    run_to_run = {"max_abs_du": float((batch.u_buf - u_a).abs().max()),
                  "max_rel_du": float(((batch.u_buf - u_a).abs() / u_a.abs().clamp_min(1e-300)).max())}
    # accuracy: exact solution u = exp(a.x), grad u = a u on the exponential-data problems
    rmse_u, rmse_g, rmse_gn = exact_rmse(probs, batch.out)
    calib = se_calibration(probs, batch.out)

    # end to end through the public API: pinned host queries in, u and grad u out, each step
    x_host = batch.x_buf.cpu().pin_memory()
    u_host = torch.empty(batch.u_buf.numel(), dtype=torch.float64).pin_memory()
    g_host = torch.empty(batch.grad_buf.numel(), dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        batch.x_buf.copy_(x_host, non_blocking=True)
        batch.run()
        u_host.copy_(batch.u_buf, non_blocking=True)
        g_host.copy_(batch.grad_buf, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e = {"value": total_steps * args.steps * world / e2e_s, "unit": "walk-steps/s",
           "h2d_bytes_per_step": int(x_host.numel() * 8),
           "d2h_bytes_per_step": int((u_host.numel() + g_host.numel()) * 8)}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0
    kernels = kernel_rooflines(W, doms, probs, replica_seed(w["seed"], rank), tuned, not args.no_cv, peaks,
                               props.multi_processor_count, sm_max, flush)
    roofline = dict(max(kernels.values(), key=lambda r: r["ms"]))
    roofline["all_kernels"] = {k: {kk: v for kk, v in r.items() if kk in ("bound", "achieved", "peak", "unit",
                                                                           "frac", "ms", "share", "kernel",
                                                                           "mma_achieved", "mma_frac")}
                               for k, r in kernels.items()}
    # kernels of one batch run: one sphere-set launch per queue, the CUDA-core walker, the
    # per-query reduction, its segment combine (queries of more than 4096 walks) and finalize
    n_sphere_queues = len({(p["domain"]["d"], sphere_queue_class(p["domain"]["d"], d.info()["sphere_tiles"]))
                           for d, p in zip(doms, probs) if d.info()["tensor_sphere_set"]})
    any_segments = any(p["n_walks"] > 4096 for p in probs)
    launches_per_step = (n_sphere_queues + (1 if "cuda_core" in kernels else 0) + 1 + (1 if any_segments else 0)
                         + 1)

    line = {"metric": METRIC, "value": value, "unit": "walk-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "parallelism": "replicas" if world > 1 else "1 GPU",
                       "l2": "flushed between steps (512 MB write)", "launch": tuned,
                       "walk_steps_per_step": total_steps, "queries_per_step": total_q,
                       "algorithmic_flops_per_step": flops},
            "queries_per_s": total_q * args.steps * world / dev_s,
            "grad_evals_per_s": total_q * args.steps * world / dev_s,
            "rmse": {"u_rel": rmse_u, "grad_rel": rmse_g, "grad_rel_aggregate": rmse_gn,
                     "against": "exact solution exp(a.x) on the 128 exponential-data problems",
                     "rmse_over_rms_se": calib, "run_to_run": run_to_run,
                     "grad_estimator": "first sphere" + ("" if args.no_cv else " with control variate")},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
            "wall_s": wall}

    log("e2e done")
    if rank == 0 and not args.no_secondary:
        if not args.no_cv:
            line["without_control_variate"] = paper_estimator(W, doms, probs, replica_seed(w["seed"], rank),
                                                              tuned, ms_per_step)
        try:
            line["error_vs_fp64_same_stream"] = fp64_same_stream(W, doms, probs, batch.out,
                                                                 replica_seed(w["seed"], rank), not args.no_cv)
        except Exception as e:
            line["error_vs_fp64_same_stream"] = {"error": "%s: %s" % (type(e).__name__, e)}
        try:
            line["variance_reduction"] = variance_reduction(W, synth, doms, probs, replica_seed(w["seed"], rank))
        except Exception as e:
            line["variance_reduction"] = {"error": "%s: %s" % (type(e).__name__, e)}
        line["vs_plain_fp32"] = plain_comparison(W, doms, probs, w["seed"], total_steps, dev_s / args.steps,
                                                 rmse_u, not args.no_cv)
        try:
            line["secondary"] = secondary(W, synth, peaks, props.multi_processor_count, sm_max)
        except Exception as e:  # a side measurement must not cost the headline line
            line["secondary"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank == 0:
        if args.cpu_seconds > 0:
            steps_cpu, t_cpu, cores, desc = oracle_sample(probs, w["seed"], args.cpu_seconds, not args.no_cv)
            s1, t1, _, _ = oracle_sample(probs, w["seed"], args.cpu_seconds / 4, not args.no_cv, threads=1)
            line["cpu_baseline"] = {"value": steps_cpu / t_cpu, "unit": "walk-steps/s", "cores": cores,
                                    "kind": "oracle", "sample": desc, "single_thread_value": s1 / t1,
                                    "single_thread_note": "the same sample on one core, about a quarter of the time"}
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def kernel_rooflines(W, doms, probs, seed, config, cv, peaks, sms, sm_max, flush):
    """Roofline of each walker family, each timed alone with CUDA events (two launches after a
    warm-up, L2 flushed before each) on the problems the batch gives it. Both count the
    method's algorithmic flops per walk-step, B(2d+3) + 4d:
      * CUDA-core persistent walker: FP32 ALU bound, against 152 SMs x 128 lanes x 2 flops x the
        maximum SM clock;
      * tensor-core sphere-set walker: bound by the tensor pipe, against the measured sustained
        dense BF16 peak (the launch runs for half a second or more); the BF16-split contraction
        it issues (2K flops per sphere) is reported beside it as mma_*."""
    import torch

    tens = [i for i, d in enumerate(doms) if d.info()["tensor_sphere_set"]]
    groups = {"cuda_core": [i for i in range(len(doms)) if i not in set(tens)], "tensor": tens}
    out = {}
    for name, idx in groups.items():
        if not idx:
            continue
        b = W.Batch([{"domain": doms[i], "x": probs[i]["X"], "n_walks": probs[i]["n_walks"], "eps": probs[i]["eps"],
                      "sigma": probs[i]["sigma"], "grad": True} for i in idx], seed=seed, config=config,
                    control_variate=cv)
        b.run()
        torch.cuda.synchronize()
        times = []
        for _ in range(2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.run()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        steps = [int(o["walk_steps"].sum()) for o in b.out]
        b.close()
        ms = min(times)
        if name == "cuda_core":
            fl = sum(s_ * alg_flops_per_step(probs[i]["domain"]["d"], probs[i]["domain"]["ball_r"].size)
                     for s_, i in zip(steps, idx))
            peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
            r = {"bound": "alu", "peak": peak, "peak_note": "FP32 FMA pipe: %d SMs x 128 lanes x 2 flop x %.0f MHz "
                 "(max SM clock)" % (sms, sm_max), "kernel": "walk_mixed_kernel<true> (CUDA-core persistent walker)",
                 "traffic": measured_traffic(),
                 "traffic_note": "ncu dram__bytes_read+write per launch (profiles/walk_mixed_batched_traffic.txt); "
                                 "balls, queries and sums are L2-resident"}
        else:
            fl, mma = 0, 0
            for s_, i in zip(steps, idx):
                dd = probs[i]["domain"]
                nb, npnt = domain_sizes(dd)
                fl += s_ * alg_flops_per_step(dd["d"], nb, npnt)
                m = nb + npnt
                mma += s_ * (-(-m // 64) * 64) * 2 * contraction_k(dd["d"])
            peak = peaks.get("bf16_tflops_sustained") or 1700.0
            r = {"bound": "tensor", "peak": peak, "peak_note": "measured sustained dense BF16 (cuBLAS), "
                 "MEASURED_PEAKS.json", "kernel": "sphere_kernel<d, true, false, 16|32> (tensor-core sphere-set "
                 "walker, one launch per queue: dimension x set class)", "traffic": measured_traffic(SPHERE_TRAFFIC_PROFILE, SPHERE_SOURCES),
                 "traffic_note": "ncu dram__bytes_read+write summed over the sphere-set launches of one "
                                 "batch run (profiles/sphere_kernel_batched_traffic.txt); tiles and sums are "
                                 "L2-resident",
                 "flops_note": "achieved counts the method's work, B(2d+3)+4d flops per walk-step (the same "
                               "count as the CUDA-core walker); mma_* count the BF16-split contraction the "
                               "tensor cores execute, 2K per sphere per walk-step (K = 3d+2 padded to 32/48, "
                               "spheres padded to 64-column tiles)",
                 "mma_flops_per_launch": mma, "mma_achieved": mma / (ms / 1e3) / 1e12,
                 "mma_frac": mma / (ms / 1e3) / 1e12 / peak}
        achieved = fl / (ms / 1e3) / 1e12
        r.update({"achieved": achieved, "unit": "TFLOP/s", "frac": achieved / r["peak"], "ms": ms,
                  "flops_per_launch": fl, "problems": len(idx)})
        out[name] = r
    tot = sum(r["ms"] for r in out.values())
    for r in out.values():
        r["share"] = r["ms"] / tot
    return out


def exact_rmse(probs, outs):
    """Relative RMSE of u and grad u against the exact solution u = exp(a.x), grad u = a u, on
    the exponential-data problems: per query (|err| / |exact|, then RMS over queries) and in
    aggregate (sqrt(sum |err|^2 / sum |exact|^2) over all queries) for the gradient."""
    rel_u, rel_g, e2, x2 = [], [], 0.0, 0.0
    for p, o in zip(probs, outs):
        if "exp_a" in p["domain"]:
            a = p["domain"]["exp_a"][0]
            us = np.exp(p["X"] @ a)
            u = o["u"].cpu().numpy()
            g = o["grad"].cpu().numpy()
            err = np.linalg.norm(g - a[None, :] * us[:, None], axis=1)
            rel_u.append((u - us) / us)
            rel_g.append(err / (np.linalg.norm(a) * us + 1e-300))
            e2 += float(np.sum(err ** 2))
            x2 += float(np.sum((np.linalg.norm(a) * us) ** 2))
    if not rel_u:
        return None, None, None
    return (float(np.sqrt(np.mean(np.concatenate(rel_u) ** 2))), float(np.sqrt(np.mean(np.concatenate(rel_g) ** 2))),
            float(np.sqrt(e2 / x2)))


def paper_estimator(W, doms, probs, seed, config, cv_ms):
    """One untimed-shape run of the same batch with the paper's first-sphere gradient (no
    control variate): its gradient RMSE and its device time, against the headline run."""
    import torch

    b = W.Batch([{"domain": d, "x": p["X"], "n_walks": p["n_walks"], "eps": p["eps"], "sigma": p["sigma"],
                  "grad": True} for d, p in zip(doms, probs)], seed=seed, config=config)
    b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ru, rg, rgn = exact_rmse(probs, b.out)
    b.close()
    return {"ms_per_step": ms, "control_variate_cost": cv_ms / ms - 1.0, "rmse_u_rel": ru, "rmse_grad_rel": rg,
            "rmse_grad_rel_aggregate": rgn, "note": "same walks (seed), same launch shape, L2 not flushed"}


def plain_comparison(W, doms, probs, seed, mixed_steps, mixed_s, mixed_rmse, cv=False):
    """The plain FP32 walker (one thread per walk, global-memory obstacles, FP32 Bessel series,
    FP32 sums) on the same 256 problems, same seeds and walk counts (equal N: both estimators
    are unbiased, so their RMSE agree up to noise, which is reported)."""
    import torch

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    outs = []
    e0.record()
    base = 0
    steps = torch.zeros(7, dtype=torch.int64, device="cuda")
    total = 0
    for d, p in zip(doms, probs):
        r = d.grad(p["X"], p["n_walks"], p["eps"], p["sigma"], precision="fp32", seed=seed, walk_offset=base,
                   with_stats=True, control_variate=cv)
        base += p["X"].shape[0] * p["n_walks"]
        outs.append((r["u"], r["stats"]))
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    total = sum(int(s[1]) for _, s in outs)
    rel = []
    for (u, _), p in zip(outs, probs):
        if "exp_a" in p["domain"]:
            us = np.exp(p["X"] @ p["domain"]["exp_a"][0])
            rel.append((u.cpu().numpy() - us) / us)
    rmse = float(np.sqrt(np.mean(np.concatenate(rel) ** 2)))
    plain_rate = total / t
    mixed_rate = mixed_steps / mixed_s
    return {"plain_walk_steps_per_s": plain_rate, "mixed_walk_steps_per_s": mixed_rate,
            "speedup": mixed_rate / plain_rate, "plain_rmse_u_rel": rmse, "mixed_rmse_u_rel": mixed_rmse,
            "note": "same walk counts; plain launched per problem (256 launches)"}


def _path_length(path, flags):
    """Length of a planner path up to the goal (or to its end) and the step that reached it."""
    p, f = path.cpu().numpy(), flags.cpu().numpy()
    hit = int(np.argmax(f == 1)) if (f == 1).any() else None
    q = p[: (hit + 1 if hit is not None else len(p))]
    return float(np.linalg.norm(np.diff(q, axis=0), axis=1).sum()), hit


def paper_sweeps(W, synth):
    """The paper's evaluation studies (Sec. VI) in its two-disc environment with the unit
    impulse at the goal, eps = 0.01, start (-8, 0, ...):
      * dimensionality (Fig. 10): angle error of grad u against a 2^26-walk reference at
        (2, -6, 0, ...), a point with a direct line to the goal (the paper's point is shown only in
        a figure; behind the obstacle the gradient is ~1e-10 and rare walks dominate it),
        d = 2..5 (extruded), N = 10^3..10^6 walks, and the device time per estimate;
      * screening (Fig. 6): planner paths for c in {10, 1, 0.1} at k_r = 0.4 (10^4 walks);
      * visibility (Fig. 7): planner paths for k_r in {0.3, 0.45, 0.6} at c = 1 (10^5 walks);
      * multistart (Fig. 5): paths at k_r = 0.2, c = 1 (10^4 walks) from six starts at radius 8
        (angles 90..315 degrees; the paper's starts are shown only in a figure).
    Paths: s_ub = 0.1, at most 400 steps; the length is measured up to the goal."""
    import torch

    eps = 0.01
    dims = {}
    for d in (2, 3, 4, 5):
        dom = W.Domain(synth.paper_environment(d))
        x = np.zeros((1, d))
        x[0, :2] = (2.0, -6.0)
        ref = dom.grad(x, 1 << 26, eps, 1.0, seed=1, control_variate=True)["grad"].cpu().numpy()[0]
        row = {}
        for n in (10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6):
            reps = 16 if n < 10 ** 6 else 4
            errs, ts = [], []
            for r in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g = dom.grad(x, n, eps, 1.0, seed=1000 + r, control_variate=True)["grad"]
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
                g = g.cpu().numpy()[0]
                c = float(np.dot(g, ref) / (np.linalg.norm(g) * np.linalg.norm(ref)))
                errs.append(math.degrees(math.acos(max(-1.0, min(1.0, c)))))
            row[str(n)] = {"angle_error_deg": float(np.mean(errs)), "ms_per_estimate": float(np.median(ts))}
        dims[str(d)] = row
    start = np.array([-8.0, 0.0])
    screening = {}
    for c in (10.0, 1.0, 0.1):
        dom = W.Domain(synth.paper_environment(2, k_r=0.4))
        path, flags, _ = dom.plan_path(start, 400, 10 ** 4, eps, c, 0.1, seed=3, control_variate=True)
        length, hit = _path_length(path, flags)
        screening[str(c)] = {"path_length": length, "reached_goal_at_step": hit}
    visibility = {}
    for k_r in (0.3, 0.45, 0.6):
        dom = W.Domain(synth.paper_environment(2, k_r=k_r))
        path, flags, _ = dom.plan_path(start, 400, 10 ** 5, eps, 1.0, 0.1, seed=3, control_variate=True)
        length, hit = _path_length(path, flags)
        visibility[str(k_r)] = {"path_length": length, "reached_goal_at_step": hit}
    multistart = {}
    try:
        # the six paths as one batched graph (wos_plan_paths), and one at a time for comparison
        dom = W.Domain(synth.paper_environment(2, k_r=0.2))
        degs = (90, 135, 180, 225, 270, 315)
        items = [{"domain": dom, "x0": 8.0 * np.array([math.cos(math.radians(g)), math.sin(math.radians(g))]),
                  "n_walks": 10 ** 4, "eps": eps, "sigma": 1.0, "s_ub": 0.1} for g in degs]
        ms_batch, res = _timed(lambda: W.plan_paths(items, 400, seed=5, control_variate=True))
        same = True

        def singles():
            return [dom.plan_path(it["x0"], 400, 10 ** 4, eps, 1.0, 0.1, seed=5, control_variate=True) for it in items]

        ms_single, one = _timed(singles)
        for g, (path, flags, _), (p1, f1, _) in zip(degs, res, one):
            length, hit = _path_length(path, flags)
            multistart[str(g)] = {"path_length": length, "reached_goal_at_step": hit}
            same &= bool(torch.equal(path, p1)) and bool(torch.equal(flags, f1))
        multistart["batched_ms"] = ms_batch
        multistart["one_at_a_time_ms"] = ms_single
        multistart["batched_equals_one_at_a_time"] = same
    except Exception as e:  # recorded; the studies above are kept
        multistart = {"error": "%s: %s" % (type(e).__name__, e)}
    return {"dimensionality_angle_error": dims, "screening_k_r_0.4": screening, "visibility_c_1": visibility,
            "multistart_k_r_0.2": multistart,
            "note": "angle error in degrees, mean over 16 estimates (4 at 10^6 walks); goal (8, 0) and "
                    "angle point (2, -6) assumed; paths from (-8, 0)"}


def _timed(fn):
    """Device time (ms) of fn() with CUDA events on the current stream, synchronised on both sides."""
    import torch

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), r


def roofline_of(flops, ms, peak, bound, note):
    achieved = flops / (ms / 1e3) / 1e12
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flops": flops, "ms": ms, "note": note}


def path_walk_steps(W, dom, path, flags, n_walks, eps, sigma, seed, cv=False):
    """Walk-steps of a planner path: every step that ran walks (flag 0 or 2) is re-run at its
    path point with its own walk offset (the same walks, so the same counts)."""
    p, f = path.cpu().numpy(), flags.cpu().numpy()
    total = 0
    for i in range(len(f)):
        if f[i] in (0, 2):
            r = dom.grad(p[i][None, :], n_walks, eps, sigma, seed=seed, walk_offset=i * n_walks, with_stats=True,
                         control_variate=cv)
            total += int(r["stats"][1])
    return total


def fp64_same_stream(W, doms, probs, outs, seed, cv, n_pick=24):
    """Error of the mixed-precision batch against the FP64 GPU walker on the same walks (same
    Philox streams, walk indices and control variate): one query from each of n_pick problems,
    half of them on the tensor-core sphere-set walker, including the problems with the most balls
    and the most walks. Returns the largest |mixed - FP64| of u and of grad u, and the largest
    ratio to the combined standard error; for du/dsigma and du/dw (which the batch does not
    return) the mixed single-query call on the same walks against FP64, as the largest absolute
    difference and the largest difference relative to the FP64 value."""
    bases = np.cumsum([0] + [p["X"].shape[0] * p["n_walks"] for p in probs])
    rng = np.random.default_rng(13)
    tens = [i for i, d in enumerate(doms) if d.info()["tensor_sphere_set"]]
    core = [i for i in range(len(doms)) if i not in set(tens)]
    heavy = [max(tens, key=lambda i: probs[i]["domain"]["ball_r"].size * probs[i]["domain"]["d"]),
             max(tens, key=lambda i: probs[i]["n_walks"])] if tens else []
    pick = list(dict.fromkeys(heavy + list(rng.permutation(tens)[: n_pick // 2 - len(heavy)]) +
                              list(rng.permutation(core)[: n_pick // 2])))
    du, dg, ru, rg = 0.0, 0.0, 0.0, 0.0
    ds_abs, ds_rel, dw_abs, dw_rel = 0.0, 0.0, 0.0, 0.0
    for i in pick:
        p, o = probs[i], outs[i]
        q = int(rng.integers(p["X"].shape[0]))
        kw = dict(seed=seed, walk_offset=int(bases[i]) + q * p["n_walks"], control_variate=cv)
        r = doms[i].grad(p["X"][q:q + 1], p["n_walks"], p["eps"], p["sigma"], precision="fp64", **kw)
        m = doms[i].grad(p["X"][q:q + 1], p["n_walks"], p["eps"], p["sigma"], precision="mixed", **kw)
        s64, sm = float(r["du_dsigma"][0]), float(m["du_dsigma"][0])
        ds_abs = max(ds_abs, abs(sm - s64))
        ds_rel = max(ds_rel, abs(sm - s64) / max(abs(s64), 1e-300))
        if r["du_dw"] is not None:
            w64, wm = r["du_dw"][0].cpu().numpy(), m["du_dw"][0].cpu().numpy()
            dw_abs = max(dw_abs, float(np.max(np.abs(wm - w64))))
            dw_rel = max(dw_rel, float(np.max(np.abs(wm - w64) / np.maximum(np.abs(w64), 1e-300))))
        u64, g64 = float(r["u"][0]), r["grad"][0].cpu().numpy()
        se_u, se_g = float(r["u_se"][0]), r["grad_se"][0].cpu().numpy()
        um, gm = float(o["u"][q]), o["grad"][q].cpu().numpy()
        du = max(du, abs(um - u64))
        dg = max(dg, float(np.max(np.abs(gm - g64))))
        ru = max(ru, abs(um - u64) / max(se_u, 1e-300))
        rg = max(rg, float(np.max(np.abs(gm - g64) / np.maximum(se_g, 1e-300))))
    return {"problems": len(pick), "tensor_core_problems": sum(1 for i in pick if i in set(tens)),
            "max_abs_u": du, "max_abs_grad": dg, "max_u_over_se": ru, "max_grad_over_se": rg,
            "max_abs_du_dsigma": ds_abs, "max_rel_du_dsigma": ds_rel, "max_abs_du_dw": dw_abs,
            "max_rel_du_dw": dw_rel,
            "note": "one query from each problem: u and grad u of the mixed batch output, du/dsigma and du/dw "
                    "of the mixed single-query call, against the FP64 GPU walker on the same walks"}


def se_calibration(probs, outs):
    """RMSE over the reported standard error on the exponential-data problems (exact solution
    exp(a.x)): sqrt(mean err^2) / sqrt(mean se^2), pooled over queries (u) and components (grad u).
    About 1 when the errors are the sampling noise the standard errors state."""
    eu, su, eg, sg = [], [], [], []
    for p, o in zip(probs, outs):
        if "exp_a" in p["domain"]:
            a = p["domain"]["exp_a"][0]
            us = np.exp(p["X"] @ a)
            eu.append(o["u"].cpu().numpy() - us)
            su.append(o["u_se"].cpu().numpy())
            eg.append((o["grad"].cpu().numpy() - a[None, :] * us[:, None]).ravel())
            sg.append(o["grad_se"].cpu().numpy().ravel())
    rms = lambda v: float(np.sqrt(np.mean(np.concatenate(v) ** 2)))
    return {"u": rms(eu) / rms(su), "grad": rms(eg) / rms(sg)}


def variance_reduction(W, synth, doms, probs, seed):
    """RMSE per walk-step of the gradient estimators on the batched workload (same walks, same
    launch shape) and on the d = 2 check workload: the paper's first-sphere estimator, the control
    variate, antithetic first directions, Russian roulette below weight 0.1, and roulette with
    antithetic pairs. RMSE against the exact solution (exp data); work = walk-steps; efficiency =
    (RMSE^2 x walk-steps) of the plain estimator over that of the option (higher is better)."""
    import torch

    variants = {"plain": {}, "control_variate": {"control_variate": True}, "antithetic": {"antithetic": True},
                "roulette_0.1": {"roulette": 0.1}, "roulette_0.1_antithetic": {"roulette": 0.1, "antithetic": True}}
    out = {}
    # batched workload
    rows = {}
    for name, kw in variants.items():
        b = W.Batch([{"domain": d, "x": p["X"], "n_walks": p["n_walks"] + (p["n_walks"] & 1), "eps": p["eps"],
                      "sigma": p["sigma"], "grad": True} for d, p in zip(doms, probs)], seed=seed, **kw)
        ms, _ = _timed(b.run)
        st = W.stats_dict(b.stats)
        ru, rg, rgn = exact_rmse(probs, b.out)
        rows[name] = {"rmse_u_rel": ru, "rmse_grad_rel_aggregate": rgn, "walk_steps": st["walk_steps"],
                      "killed": st["killed"], "ms": ms}
        b.close()
    for name, r in rows.items():
        p0 = rows["plain"]
        r["efficiency_u"] = (p0["rmse_u_rel"] ** 2 * p0["walk_steps"]) / (r["rmse_u_rel"] ** 2 * r["walk_steps"])
        r["efficiency_grad"] = ((p0["rmse_grad_rel_aggregate"] ** 2 * p0["walk_steps"]) /
                                (r["rmse_grad_rel_aggregate"] ** 2 * r["walk_steps"]))
    out["batched_uneven"] = rows
    # d = 2 check workload (mixed precision, 64 queries x 10^4 walks)
    w = synth.c1()
    dom = W.Domain(w["domain"])
    a = w["domain"]["exp_a"][0]
    ex = np.exp(w["X"] @ a)
    rows = {}
    for name, kw in variants.items():
        r = dom.grad(w["X"], w["n_walks"], w["eps"], w["sigma"], seed=w["seed"], with_stats=True, **kw)
        u, g = r["u"].cpu().numpy(), r["grad"].cpu().numpy()
        st = W.stats_dict(r["stats"])
        eg = np.linalg.norm(g - a[None, :] * ex[:, None], axis=1)
        rows[name] = {"rmse_u_rel": float(np.sqrt(np.mean(((u - ex) / ex) ** 2))),
                      "rmse_grad_rel_aggregate": float(np.sqrt(np.sum(eg ** 2) / np.sum((np.linalg.norm(a) * ex) ** 2))),
                      "walk_steps": st["walk_steps"], "killed": st["killed"]}
    for name, r in rows.items():
        p0 = rows["plain"]
        r["efficiency_u"] = (p0["rmse_u_rel"] ** 2 * p0["walk_steps"]) / (r["rmse_u_rel"] ** 2 * r["walk_steps"])
        r["efficiency_grad"] = ((p0["rmse_grad_rel_aggregate"] ** 2 * p0["walk_steps"]) /
                                (r["rmse_grad_rel_aggregate"] ** 2 * r["walk_steps"]))
    out["check_2d"] = rows
    out["note"] = ("efficiency = plain RMSE^2 x walk-steps / option's (higher is better); batched workload with "
                   "odd walk counts rounded up to even for the antithetic pairs (all variants)")
    return out


def rr_validation(W, synth):
    """The RR validation (Sec. VII, Table I): paths from q_start toward the unit impulse at q_goal
    with 10^5 walks per step, s = min(0.1, d_bound/2), eps = 0.02, for c = 0 and 5, with the
    Lipschitz arm distance (Sec. V-A; CUDA-core walker) and with the 200 closed-form IK collision
    configurations (a point set: tensor-core walker), mixed precision. Path lengths in joint
    space (the paper's 4.5 for c = 0 and 3.8 for c = 5 come from its own link lengths and joint
    limits, shown only in figures)."""
    out = {}
    for method, precision in (("lipschitz", "mixed"), ("ik", "mixed")):
        for c in synth.RR_TABLE_I["c"]:
            w = synth.rr_arm(c, method=method)
            dom = W.Domain(w["domain"])
            ms, (path, flags, _) = _timed(lambda: dom.plan_path(w["start"], 300, w["n_walks"], w["eps"], w["sigma"],
                                                                w["s_ub"], precision=precision, seed=w["seed"]))
            length, hit = _path_length(path, flags)
            f = flags.cpu().numpy()
            out["%s_c%g" % (method, c)] = {"path_length": length, "reached_goal_at_step": hit, "ms": ms,
                                           "precision": precision, "no_signal_steps": int((f == 2).sum())}
    out["note"] = "joint-space path lengths; link lengths 1, 1 and joint limits [0, -pi]..[3pi/2, pi] read from the figures"
    return out


def secondary(W, synth, peaks, sms, sm_max):
    """Measurements of the other workloads (not the headline), each with the roofline of its
    dominant kernel: algorithmic flops per walk-step from the method (B(2d+3) + 4d for balls,
    M(2d+1) + 4d for points) over the device time of the call (CUDA events)."""
    import torch

    out = {}
    fp32 = fp32_peak_tflops(sms, sm_max)
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    # 2D planning field: 200-step graph-replayed path, 1024 walks per grad u
    w = synth.c2()
    dom = W.Domain(w["domain"])
    dom.plan_path(w["start"], 5, w["n_walks"], w["eps"], w["sigma"], w["s_ub"], seed=w["seed"])
    ms, (path, flags, _) = _timed(lambda: dom.plan_path(w["start"], w["n_steps"], w["n_walks"], w["eps"],
                                                        w["sigma"], w["s_ub"], seed=w["seed"]))
    f = flags.cpu().numpy()
    ran = int(np.sum((f == 0) | (f == 2)))
    steps = path_walk_steps(W, dom, path, flags, w["n_walks"], w["eps"], w["sigma"], w["seed"])
    out["planning_2d"] = {"path_ms": ms, "ms_per_planner_step": ms / max(ran, 1), "planner_steps_with_walks": ran,
                          "reached_goal_at_step": int(np.argmax(f == 1)) if (f == 1).any() else None,
                          "grad_evals_per_s": ran / (ms / 1e3), "walk_steps_per_s": steps / (ms / 1e3),
                          "roofline": roofline_of(steps * alg_flops_per_step(2, 33), ms, fp32, "alu",
                                                  "latency-bound: 1024 walks per dependent step; FP32 FMA peak")}
    # the paper's two-disc environment with a unit impulse at the goal (Sec. VI): r_o = 10,
    # k_r = 0.3, c = sigma = 1, eps = 0.01, start (-8, 0); the goal (8, 0) is this benchmark's
    # choice (the paper shows it only in a figure). 1024 walks per planner step.
    env = synth.paper_environment(2)
    dom = W.Domain(env)
    dom.plan_path(np.array([-8.0, 0.0]), 5, 1024, 0.01, 1.0, 0.1, seed=1, control_variate=True)
    ms, (path, flags, _) = _timed(lambda: dom.plan_path(np.array([-8.0, 0.0]), 400, 1024, 0.01, 1.0, 0.1, seed=1,
                                                        control_variate=True))
    f = flags.cpu().numpy()
    p_end = path.cpu().numpy()[-1]
    out["paper_environment_2d"] = {"path_ms": ms, "ms_per_planner_step": ms / 400,
                                   "reached_goal_at_step": int(np.argmax(f == 1)) if (f == 1).any() else None,
                                   "final_distance_to_goal": float(np.linalg.norm(p_end - env["source_z"]))}
    try:
        out["paper_sweeps"] = paper_sweeps(W, synth)
    except Exception as e:  # recorded, so that the other side measurements are kept
        out["paper_sweeps"] = {"error": "%s: %s" % (type(e).__name__, e)}
    try:
        out["rr_validation"] = rr_validation(W, synth)
    except Exception as e:
        out["rr_validation"] = {"error": "%s: %s" % (type(e).__name__, e)}
    # differentiable d=6: forward + backward, 4096 queries x 2048 walks
    w = synth.c5()
    dom = W.Domain(w["domain"])
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda", requires_grad=True)
    wt = torch.tensor(w["domain"]["exp_w"], dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(w["sigma"], dtype=torch.float64, requires_grad=True)
    u = W.WoSFunction.apply(X, sig, wt, dom, w["n_walks"], w["eps"], w["seed"])
    u.sum().backward()
    torch.cuda.synchronize()
    fwd, fb = [], []

    def fwd_bwd():
        X.grad = None
        u = W.WoSFunction.apply(X, sig, wt, dom, w["n_walks"], w["eps"], w["seed"])
        u.sum().backward()

    for _ in range(3):  # best of three: the first backward pass can include one-time host work
        ms_f, r = _timed(lambda: dom.grad(X.detach(), w["n_walks"], w["eps"], w["sigma"], seed=w["seed"],
                                          with_stats=True))
        ms_fb, _ = _timed(fwd_bwd)
        fwd.append(ms_f)
        fb.append(ms_fb)
    steps = int(r["stats"][1])
    sub = w["X"][:256]
    mix = dom.grad(sub, w["n_walks"], w["eps"], w["sigma"], seed=w["seed"])
    f64 = dom.grad(sub, w["n_walks"], w["eps"], w["sigma"], seed=w["seed"], precision="fp64")
    err = {k: float(torch.max(torch.abs(mix[k] - f64[k]))) for k in ("u", "grad", "du_dsigma", "du_dw")}
    err["note"] = "max |mixed - FP64| on the same walks, 256 of the 4096 queries"
    out["differentiable_6d"] = {"forward_ms": min(fwd), "forward_backward_ms": min(fb),
                                "walk_steps_per_s": steps / (min(fwd) / 1e3),
                                "queries_per_s": w["X"].shape[0] / (min(fwd) / 1e3),
                                "error_vs_fp64_same_stream": err,
                                "roofline": roofline_of(steps * alg_flops_per_step(6, 64), min(fwd), fp32, "alu",
                                                        "CUDA-core walker (64 balls); FP32 FMA peak")}
    # point-cloud C-space, d = 7: 65536 points, tensor-core distance, all 8192 queries x 4096 walks
    w = synth.c3()
    dom = W.Domain(w["domain"])
    M = w["domain"]["points"].shape[0]
    dom.solve(w["X"][:128], 256, w["eps"], w["sigma"], seed=w["seed"])
    ms, r = _timed(lambda: dom.solve(w["X"], w["n_walks"], w["eps"], w["sigma"], seed=w["seed"], with_stats=True))
    st = W.stats_dict(r["stats"])
    rl = roofline_of(st["walk_steps"] * alg_flops_per_step(7, 0, M), ms, bf16, "tensor",
                     "tensor-core sphere-set walker; measured sustained BF16 peak")
    mma = st["walk_steps"] * M * 2 * contraction_k(7)
    rl.update({"mma_achieved": mma / (ms / 1e3) / 1e12, "mma_frac": mma / (ms / 1e3) / 1e12 / bf16})
    out["pointcloud_7d"] = {"queries": int(w["X"].shape[0]), "walks_per_query": w["n_walks"], "ms": ms,
                            "walk_steps_per_s": st["walk_steps"] / (ms / 1e3),
                            "queries_per_s": w["X"].shape[0] / (ms / 1e3),
                            "point_distance_evals_per_s": st["walk_steps"] * M / (ms / 1e3),
                            "bound_shrinks": st["shrinks"], "roofline": rl}
    # plain FP64 d=2 check workload
    w = synth.c1()
    dom = W.Domain(w["domain"])
    for prec in ["fp64", "mixed"]:
        dom.grad(w["X"], w["n_walks"], w["eps"], w["sigma"], precision=prec, seed=w["seed"])
        ms, r = _timed(lambda: dom.grad(w["X"], w["n_walks"], w["eps"], w["sigma"], precision=prec, seed=w["seed"],
                                        with_stats=True))
        steps = int(r["stats"][1])
        fl = steps * alg_flops_per_step(2, 4)
        rl = (roofline_of(fl, ms, FP64_NOMINAL_TFLOPS, "alu", "FP64 walker; nominal GB300 FP64 rate (not measured)")
              if prec == "fp64" else roofline_of(fl, ms, fp32, "alu", "mixed CUDA-core walker; FP32 FMA peak"))
        out["fp64_check_2d_" + prec] = {"ms": ms, "walk_steps_per_s": steps / (ms / 1e3),
                                        "queries_per_s": w["X"].shape[0] / (ms / 1e3), "roofline": rl}
    return out


if __name__ == "__main__":
    main()
