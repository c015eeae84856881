#!/usr/bin/env python3
"""Benchmark: dense affinity propagation on one GB300 through the C ABI.

A step is one pass of the hot path over one synthetic problem: the similarity
build (ap_similarity: centred GEMM + exact median preference), the damped
sweep to convergence (ap_iterate) and the outputs (ap_exemplars).  Workload:
N=20000 points in 64-D from a seeded mixture of 50 Gaussians (centres
N(0,25 I), sigma 1, Dirichlet(2) weights), damping 0.9, at most 1000
iterations, stop after 15 unchanged exemplar sets.

value = algorithmic sweep bytes (20 B per matrix element per iteration: S, R,
A read once, R, A written once) over the whole step's device time, in GB/s.
Inputs stay resident in HBM; S, R, A are 1.6 GB each (> L2), so no L2 flush
is needed between steps.  ``e2e`` repeats the step through the same C ABI
with the features in pinned host memory and the labels copied back.

--impl reference times the float64 CPU oracle on a bounded sample of the same
workload (the oracle is the only reference: the paper ships no code).

Multi-GPU: independent replicas (the method's sweep is not sharded here), one
process per GPU under torchrun; value = all ranks' bytes / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_POINTS, DIM = 20000, 64
REFINE_ROUNDS = 8                 # Algorithm 3 Step 4's refinement rounds
DAMPING, MAX_ITER, CONV_ITER = 0.9, 1000, 15
METRIC = "AP sweep HBM GB/s vs peak; time-to-converge vs plain GPU AP at equal net sim"
WORKLOAD = ("plain dense AP, N=20000, d=64, 50-Gaussian mixture (centres N(0,25I), sigma 1, "
            "Dirichlet(2) weights); S via BF16 tcgen05 GEMM + FP32 norms (or FP32 SIMT GEMM); "
            "preference = off-diagonal median; damping 0.9, max 1000 iters, 15 unchanged sweeps")


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(elapsed_s, bytes_done, world, device):
    """Whole-job figures over the replicas: the slowest rank's time (max) and
    every rank's bytes (sum), by all-reduce when world > 1.  Returns
    (elapsed_max_s, total_bytes, value_gbs)."""
    import torch
    import torch.distributed as dist

    times = torch.tensor([float(elapsed_s)], device=device, dtype=torch.float64)
    tot = torch.tensor([float(bytes_done)], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(times, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    t = max(float(times.item()), 1e-12)
    return t, float(tot.item()), float(tot.item()) / t / 1e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _kernel_source_hash():
    """Hash of the sweep kernel's own source: the text of sweep.cu from its
    device-side structs (state, problem table, work list) through the end of
    sweep_kernel, plus the two device headers it uses (host-side edits leave
    the counters valid)."""
    csrc = os.path.join(ROOT, "paper_0910_1650_gb300", "csrc")
    with open(os.path.join(csrc, "sweep.cu")) as f:
        text = f.read()
    lo = text.index("struct SweepState")
    hi = text.index("// Column sums in a fixed order")
    h = hashlib.sha256(text[lo:hi].encode())
    for name in ("common.cuh", "ptx.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(n):
    """ncu DRAM bytes per sweep launch, if the committed capture matches the
    current kernel source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "sweep_traffic.json")) as f:
            t = json.load(f)
    except OSError:
        return None
    if t.get("source_hash") != _kernel_source_hash():
        return None
    per_elem = t["dram_bytes_per_launch"] / float(t["n"]) ** 2
    return per_elem * n * n


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_0910_1650_gb300 import capi, synth

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    capi.lib()

    X, _ = synth.workload(1, scale=args.n / N_POINTS)
    n, d = X.shape
    Xd = torch.from_numpy(X).to(dev)
    Xh = torch.from_numpy(X).pin_memory()
    S = capi.empty_square(n, dev)
    R = capi.empty_square(n, dev)
    A = capi.empty_square(n, dev)
    stream = torch.cuda.current_stream()

    phase_ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    phase_ms = {"similarity": 0.0, "iterate": 0.0, "exemplars": 0.0}

    def step(X_in, timed=False):
        if timed:
            phase_ev[0].record(stream)
        capi.ap_similarity(X_in, S, precision=args.precision)
        if timed:
            phase_ev[1].record(stream)
        # a cold start (R = A = 0) without clearing R and A: the library reads zeros
        _, _, res, _ = capi.ap_iterate(S, R, A, damping=DAMPING, max_iter=MAX_ITER,
                                       conv_iter=CONV_ITER, time_sweep=True, decisions=False,
                                       cold=True)
        if timed:
            phase_ev[2].record(stream)
        idx, ex = capi.ap_exemplars(S, R, A)
        if timed:
            phase_ev[3].record(stream)
            phase_ev[3].synchronize()
            for k, (a, b) in zip(("similarity", "iterate", "exemplars"), ((0, 1), (1, 2), (2, 3))):
                phase_ms[k] += phase_ev[a].elapsed_time(phase_ev[b])
        return res, ex, idx

    for _ in range(args.warmup):
        step(Xd)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region ------------------------------------------
    launches0 = capi.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, sweep_ms, sweep_launches, results = 0, 0.0, 0, []
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            res, ex, _ = step(Xd, timed=True)
            iters += res["iters"]
            sweep_ms += res["sweep_ms"]
            sweep_launches += res["sweep_launches"]
            results.append((res, ex))
        ev1.record(stream)
        barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = capi.kernel_launches() - launches0
    bytes_done = 20.0 * n * n * iters
    elapsed_max, _, value = aggregate(elapsed, bytes_done, world, dev)

    # ---- end to end through the C ABI: host features in, labels out ------------
    if args.no_e2e:
        args_steps_e2e = 0
    else:
        args_steps_e2e = args.steps
    barrier()
    e0 = time.perf_counter()
    ev0.record(stream)
    e_iters = 0
    for _ in range(args_steps_e2e):
        Xs = Xh.to(dev, non_blocking=True)
        res, ex, idx = step(Xs)
        lab = idx.to("cpu")
        e_iters += res["iters"]
    ev1.record(stream)
    barrier()
    e_elapsed = ev0.elapsed_time(ev1) / 1e3
    e_wall = time.perf_counter() - e0
    _, _, e_value = aggregate(max(e_elapsed, 1e-9), 20.0 * n * n * e_iters, world, dev)

    if rank == 0:
        peaks, src = _peaks()
        sweep_bytes_per_iter = 20.0 * n * n
        # launch 1 has no availability half (16 B per element: S, A, R read,
        # R written) and the last launch no responsibility half (12 B: R, A
        # read, A written); the others move 20 B
        alg_bytes = n * n * (20.0 * max(sweep_launches - 2 * args.steps, 0) + 28.0 * args.steps)
        achieved = alg_bytes / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None
        traffic = _traffic(n)
        last_res, last_ex = results[-1]
        line = {
            "metric": METRIC,
            "value": round(value, 2),
            "unit": "GB/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(elapsed_max / args.steps * 1e3, 3),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic (seeded generator; paper datasets unavailable)",
            "config": {"workload": WORKLOAD, "n": n, "d": d, "precision": args.precision,
                       "damping": DAMPING, "max_iter": MAX_ITER, "conv_iter": CONV_ITER,
                       "iters_per_step": last_res["iters"],
                       "n_exemplars": last_ex["n_exemplars"], "netsim": last_ex["netsim"],
                       "l2": "inputs larger than L2 (S, R, A 1.6 GB each); no flush",
                       "phase_ms_per_step": {k: round(v / args.steps, 3) for k, v in phase_ms.items()},
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"kernel": "sweep_kernel", "bound": "hbm",
                         "achieved": round(achieved, 1) if achieved else None,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / peaks["hbm_gbs"], 4) if achieved else None,
                         "traffic": traffic, "peak_source": src,
                         "alg_bytes_per_launch": sweep_bytes_per_iter,
                         "launch_ms": round(sweep_ms / max(sweep_launches, 1), 4)},
            "e2e": {"value": round(e_value, 2), "unit": "GB/s",
                    "h2d_bytes_per_step": int(n * d * 4), "d2h_bytes_per_step": int(n * 4 + 56),
                    "wall_s": round(e_wall, 3)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        if not args.no_ttc and world == 1:
            del S, R, A, Xd
            torch.cuda.empty_cache()
            line["time_to_converge"] = time_to_converge(dev)
            line["autotune"] = autotune(dev)
            line["pap_table2"] = pap_table2(dev)
            line["small_problem"] = small_problem(dev)
            line["batch_learned"] = batch_learned(dev)
            line["paper_2d"] = paper_2d(dev)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sharded(args):
    """--sharded: the step's sweep (Algorithm 1 from zero messages to
    convergence) on the same workload with the rows of S, R and A split over
    the ranks, one GPU each, and one NCCL all-reduce of 2n + 2 floats per
    iteration (sharded.iterate).  Total work is fixed as ranks are added
    (strong scaling); with one rank it is the single-GPU sweep.  value =
    20 B x N^2 x iterations over the slowest rank's device time."""
    import torch
    import torch.distributed as dist

    from paper_0910_1650_gb300 import capi, sharded, synth

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    X, _ = synth.workload(1, scale=args.n / N_POINTS)
    n = X.shape[0]
    r0, r1 = sharded.row_range(n, world, rank)
    S, _ = capi.ap_similarity(torch.from_numpy(X).to(dev), precision=args.precision)
    ld = capi.padded_ld(n)
    Sr = torch.zeros(r1 - r0, ld, dtype=torch.float32, device=dev)
    Sr[:, :n] = S[r0:r1]
    del S
    torch.cuda.empty_cache()
    R = torch.zeros_like(Sr)
    A = torch.zeros_like(Sr)
    sh = sharded.LibraryShard(Sr, R, A, n, r0, r1, damping=DAMPING, max_iter=MAX_ITER, conv_iter=CONV_ITER)
    allreduce = sharded.torch_allreduce() if world > 1 else (lambda t: None)

    def step():
        R.zero_()
        A.zero_()
        return sharded.iterate(sh, allreduce)

    for _ in range(args.warmup):
        step()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    iters = 0
    ev0.record()
    for _ in range(args.steps):
        iters += step()["iters"]
    ev1.record()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    t = torch.tensor([elapsed], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        value = 20.0 * n * n * iters / float(t.item()) / 1e9
        print(json.dumps({
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(float(t.item()) / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator; paper datasets unavailable)",
            "config": {"workload": WORKLOAD, "n": n, "d": X.shape[1], "phase": "iterate to convergence",
                       "iters_per_step": iters // max(args.steps, 1),
                       "parallelism": f"rows of S, R, A split over {world} GPU(s), one all-reduce of "
                                      f"2n+2 floats per iteration"}}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def pap_table2(dev, reps=5):
    """Table 2's shape on a seeded stand-in: 2021 points in 62-D from 86
    Gaussian classes (the faces' size, dimension and class count; centres
    N(0, 4I), sigma 1), plain AP against PAP with k = 2, 4, 8, 16 equal
    blocks, at the paper's damping 0.5 and at the workloads' 0.9; max 1000,
    15 unchanged sweeps.  Iterations and device time of whole calls, means
    over ``reps`` seeded sets."""
    import torch

    from paper_0910_1650_gb300 import capi, synth

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ev[0].record()
        r = fn()
        ev[1].record()
        ev[1].synchronize()
        return r, ev[0].elapsed_time(ev[1])

    out = {}
    # untimed: the process's first calls at these shapes pay one-time set-up
    # (launch configuration probes, graph capture), about 0.25 s
    X, _ = synth.gaussian_mixture(2021, 62, 86, synth.SEED_BASE + 899, 2.0, 1.0)
    S, _ = capi.ap_similarity(torch.from_numpy(X).to(dev), precision="fp32")
    capi.ap_iterate(S, damping=0.5, max_iter=MAX_ITER, conv_iter=CONV_ITER)
    for k in (2, 4, 8, 16):
        capi.pap_run(S, k, None, damping=0.5, max_iter=MAX_ITER, conv_iter=CONV_ITER)
    torch.cuda.synchronize()
    for lam in (0.5, 0.9):
        kw = dict(damping=lam, max_iter=MAX_ITER, conv_iter=CONV_ITER)
        rows = {"plain": [], **{k: [] for k in (2, 4, 8, 16)}}
        for r in range(reps):
            X, _ = synth.gaussian_mixture(2021, 62, 86, synth.SEED_BASE + 900 + r, 2.0, 1.0)
            S, _ = capi.ap_similarity(torch.from_numpy(X).to(dev), precision="fp32")
            (R, A, ra, _), t = timed(lambda: capi.ap_iterate(S, **kw))
            _, ea = capi.ap_exemplars(S, R, A)
            rows["plain"].append((ra["iters"], t, ea["netsim"], ea["n_exemplars"], ra["converged"]))
            for k in (2, 4, 8, 16):
                (_, _, _, pr), tp = timed(lambda: capi.pap_run(S, k, None, **kw))
                f = pr["final"]
                rows[k].append((f["iters"], tp, f["netsim"], f["n_exemplars"], f["converged"],
                                pr["sub_iters_max"], ea["netsim"]))
        plain = rows["plain"]
        res = {"plain": {"iters": round(float(np.mean([x[0] for x in plain])), 1),
                         "ms": round(float(np.mean([x[1] for x in plain])), 2),
                         "converged": int(sum(x[4] for x in plain)),
                         "n_exemplars": round(float(np.mean([x[3] for x in plain])), 1)}}
        for k in (2, 4, 8, 16):
            v = rows[k]
            res[f"pap_k{k}"] = {
                "step4_iters": round(float(np.mean([x[0] for x in v])), 1),
                "step4_iters_over_plain": round(float(np.mean([x[0] for x in v])) / max(res["plain"]["iters"], 1), 3),
                "sub_iters_max": round(float(np.mean([x[5] for x in v])), 1),
                "ms": round(float(np.mean([x[1] for x in v])), 2),
                "converged": int(sum(x[4] for x in v)),
                "netsim_rel_diff_mean": float(np.mean([(x[2] - x[6]) / abs(x[6]) for x in v]))}
        out[f"damping_{lam}"] = res
    out["workload"] = ("2021 points, 62-D, 86 Gaussian classes (centres N(0,4I), sigma 1); equal "
                       "contiguous blocks; %d seeded sets" % reps)
    return out


def autotune(dev, iters=30):
    """The sweep autotuner on the step's workload (N = 20000): every admissible
    (cluster, float4 per thread, stages) configuration timed over 10
    iterations, the fastest pinned; reported against the built-in rule's
    choice, each timed over ``iters`` iterations with per-launch CUDA events.
    The pin is removed afterwards (the headline numbers use the rule)."""
    import torch

    from paper_0910_1650_gb300 import capi, synth

    X, _ = synth.workload(1)
    n = X.shape[0]
    S, _ = capi.ap_similarity(torch.from_numpy(X).to(dev), precision="bf16")
    R = capi.empty_square(n, dev, 0.0)
    A = capi.empty_square(n, dev, 0.0)

    def per_iter():
        R.zero_()
        A.zero_()
        _, _, r, _ = capi.ap_iterate(S, R, A, damping=DAMPING, max_iter=iters, conv_iter=0,
                                     time_sweep=True, decisions=False)
        return r["sweep_ms"] / r["sweep_launches"]

    capi.ap_sweep_set_config(n)
    rule = capi.ap_sweep_get_config(n)
    per_iter()
    t_rule = per_iter()
    t0 = time.perf_counter()
    best = capi.ap_sweep_autotune(S, R, A, damping=DAMPING, iters=10)
    tune_s = time.perf_counter() - t0
    t_best = per_iter()
    capi.ap_sweep_set_config(n)
    del S, R, A
    torch.cuda.empty_cache()
    cfg = lambda c: f"cluster {c['cluster']}, {c['ept']} float4/thread, {c['stages']} stages"
    return {"n": n, "rule": cfg(rule), "rule_ms_per_iter": round(t_rule, 4),
            "tuned": cfg(best), "tuned_ms_per_iter": round(t_best, 4), "tuning_s": round(tune_s, 2),
            "rule_frac_of_tuned": round(t_best / t_rule, 4)}


def small_problem(dev, reps=20):
    """The 500-point 2-D mixture (damping 0.5, max 200, 15 unchanged sweeps):
    S, R and A (1 MB each) stay in L2, so a run is bound by launch latency,
    not HBM.  Device time of whole ap_iterate calls (CUDA events) with the
    iterations enqueued as CUDA graphs and as separate launches."""
    import torch

    from paper_0910_1650_gb300 import capi, synth

    X, _ = synth.workload(0)
    S, _ = capi.ap_similarity(torch.from_numpy(X).to(dev), precision="fp32")
    R = capi.empty_square(S.shape[0], dev, 0.0)
    A = capi.empty_square(S.shape[0], dev, 0.0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {"workload": "500 points in 2-D, 5 Gaussians (centres U[-10,10]^2, sigma 1); "
                       "p = off-diagonal median; damping 0.5, max 200, 15 unchanged sweeps; "
                       "L2-resident (roofline n/a)", "n": int(S.shape[0])}
    for graph in (True, False):
        def run():
            R.zero_()
            A.zero_()
            return capi.ap_iterate(S, R, A, damping=0.5, max_iter=200, conv_iter=15,
                                   graph=graph)[2]
        r = run()                       # capture (graph) / warm-up
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            r = run()
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / reps
        key = "graph" if graph else "stream"
        out[key] = {"iters": r["iters"], "ms_to_converge": round(ms, 4),
                    "us_per_iter": round(ms * 1e3 / max(r["iters"], 1), 3)}
    return out


def _agreement(ref, got):
    """Fraction of points whose cluster under ``got``, mapped to the ``ref``
    cluster holding most of its points, equals their ``ref`` cluster (the
    reading of Table 1's undefined "accuracy")."""
    ref = np.asarray(ref)
    got = np.asarray(got)
    ok = 0
    for g in np.unique(got):
        members = ref[got == g]
        ok += np.bincount(np.unique(members, return_inverse=True)[1]).max()
    return ok / ref.size


def paper_2d(dev, reps=10):
    """Table 1's landmark-count sweep on a seeded stand-in (5-Gaussian 2-D
    mixtures of 1000 points, damping 0.5): AP against landmark AP with
    100-500 landmarks, averaged over ``reps`` seeded sets.  Device time of
    whole calls (CUDA events)."""
    import torch

    from paper_0910_1650_gb300 import capi, synth

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ev[0].record()
        r = fn()
        ev[1].record()
        ev[1].synchronize()
        return r, ev[0].elapsed_time(ev[1])

    kw = dict(damping=0.5, max_iter=1000, conv_iter=15)
    table1 = []
    base = []
    for r in range(reps):
        X, _ = synth.gaussian_mixture_2d(seed=synth.SEED_BASE + 600 + r, per_cluster=200)
        Xd = torch.from_numpy(X).to(dev)
        S, _ = capi.ap_similarity(Xd, precision="fp32")
        (R, A, _, _), t = timed(lambda: capi.ap_iterate(S, **kw))
        idx, _ = capi.ap_exemplars(S, R, A)
        base.append((Xd, idx.cpu().numpy(), t))
    for L in (500, 400, 300, 200, 100):
        ms, acc = [], []
        for r, (Xd, ref, _) in enumerate(base):
            (idx, _, _), t = timed(lambda: capi.lap_run(Xd, L, "uniform", seed=synth.SEED_BASE + 700 + r,
                                                        precision="fp32", **kw))
            ms.append(t)
            acc.append(_agreement(ref, idx.cpu().numpy()))
        table1.append({"landmarks": L, "ms": round(float(np.mean(ms)), 2),
                       "agreement_with_ap": round(float(np.mean(acc)), 4)})
    return {"workload": "5-Gaussian 2-D mixtures (centres U[-10,10]^2, sigma 1), damping 0.5, max 1000, "
                        "15 unchanged sweeps; %d seeded sets per point" % reps,
            "table1": {"n": 1000, "ap_ms": round(float(np.mean([b[2] for b in base])), 2),
                       "lap": table1,
                       "agreement": "fraction of points whose LAP cluster, mapped to its majority AP "
                                    "cluster, is their AP cluster"}}


def batch_learned(dev, count=256, n_train=32):
    """The batch workload: 256 independent problems of image-like vectors
    (N uniform in [200, 4000], d = 4096).  S of every problem by the batched
    tensor-core similarity; Algorithm 1 on all problems at once (one batched
    sweep per iteration) from a cold start, and from the learned warm start
    (network trained here on 32 further problems of the same generator),
    each warm result judged against the cold one (net similarity within
    0.5 %, else the cold result is kept).  Device times by CUDA events."""
    import torch

    from paper_0910_1650_gb300 import batched, capi, learned, synth

    # start from an empty allocator cache: after the 160 GB runs of the
    # time-to-converge section, arenas carved from torch's cached blocks ran
    # the batch about 1.5x slower than freshly allocated ones
    torch.cuda.empty_cache()
    sizes, _ = synth.batch_problem_sizes(count)
    # the features are drawn first (a pool of host processes): drawing them
    # while the timed similarity calls run starved those calls' host-side set-up
    # and left the GPU waiting (20-46 ms for the same work)
    problems = list(batched.image_batch(count))
    B = batched.Batch(problems, sizes[:count])
    del problems
    peaks, src = _peaks()
    tflops = B.gemm_flops / (B.sim_ms / 1e3) / 1e12
    R = torch.zeros_like(B.S)
    A = torch.zeros_like(B.S)
    ws = capi.ap_iterate_batched_workspace(B.n, B.ld, B.S.device)
    R, A, rc, ms_c = batched.run(B, R, A, ws=ws)
    cold = batched.netsims(B, R, A)
    F, T, _ = learned.make_dataset(list(batched.image_batch(n_train, offset=count)))
    P, P16, losses = learned.train(F, T, epochs=60, batch=4096, lr=2e-3)
    R, A, ms_ws = batched.warm_start(B, P, P16, R=R, A=A)
    R, A, rw, ms_w = batched.run(B, R, A, ws=ws)
    warm = batched.netsims(B, R, A)
    keep = batched.judge(cold, warm)
    del R, A, ws
    torch.cuda.empty_cache()
    it_c = [r["iters"] for r in rc]
    it_w = [r["iters"] for r in rw]
    rel = [abs(w[0] - c[0]) / abs(c[0]) for c, w in zip(cold, warm)]
    return {
        "workload": "256 problems, N ~ U{200..4000}, d = 4096 image-like vectors (rank-20 "
                    "nonnegative templates, 5-40 clusters, + U[0,0.05] noise); damping 0.9, "
                    "max 1000, 15 unchanged sweeps",
        "sum_n2": float(sum(float(m) * m for m in B.n)),
        "similarity": {"ms": round(B.sim_ms, 2), "tflops": round(tflops, 1),
                       "frac_of_bf16_peak": round(tflops / peaks["bf16_tflops"], 4),
                       "peak_source": src,
                       "note": "whole batched similarity (means, centring, Gram product, "
                               "median) over 2 n^2 d flops"},
        "cold": {"ms": round(ms_c, 1), "iters_mean": round(sum(it_c) / count, 1),
                 "iters_max": max(it_c), "converged": sum(r["converged"] for r in rc)},
        "train": {"problems": n_train, "rows": int(F.shape[0]), "epochs": 60,
                  "loss_first": round(losses[0], 4), "loss_last": round(losses[-1], 4)},
        "warm": {"ms_warm_start": round(ms_ws, 1), "ms": round(ms_w, 1),
                 "iters_mean": round(sum(it_w) / count, 1), "iters_max": max(it_w),
                 "judge_keeps": sum(keep), "netsim_rel_diff_median": round(sorted(rel)[count // 2], 5)},
        "time_ratio_cold_over_warm": round(ms_c / (ms_ws + ms_w), 3),
    }


def time_to_converge(dev):
    """Time to converge of partition AP and landmark AP against plain GPU AP
    on the same inputs (device time, CUDA events), with net similarities."""
    import torch

    from paper_0910_1650_gb300 import capi, learned, synth

    out = {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, warm=True):
        if warm:
            fn()                    # untimed first run: allocator misses stay outside
            torch.cuda.synchronize()
        ev[0].record()
        r = fn()
        ev[1].record()
        ev[1].synchronize()
        return r, ev[0].elapsed_time(ev[1])

    # ---- partition AP: 60000 points on 10 subspaces of R^100, 32 uneven subsets
    X, _ = synth.subspaces()
    offs = synth.uneven_partition()
    n = X.shape[0]
    S, _ = capi.ap_similarity(torch.from_numpy(X).to(dev), precision="bf16")
    R = capi.empty_square(n, dev, 0.0)
    A = capi.empty_square(n, dev, 0.0)

    def plain():
        R.zero_()
        A.zero_()
        _, _, r, _ = capi.ap_iterate(S, R, A, damping=DAMPING, max_iter=MAX_ITER,
                                     conv_iter=CONV_ITER, decisions=False)
        _, ex = capi.ap_exemplars(S, R, A)
        return r, ex

    (rp, exp_), t_plain = timed(plain)
    (_, _, _, pr), t_pap = timed(lambda: capi.pap_run(S, len(offs) - 1, list(offs), damping=DAMPING,
                                                      max_iter=MAX_ITER, conv_iter=CONV_ITER,
                                                      R=R, A=A))
    out["pap"] = {
        "workload": "60000 points on 10 random 5-dim subspaces of R^100 + N(0,0.01) noise; "
                    "32 uneven seeded subsets (500-4000)",
        "plain": {"iters": rp["iters"], "ms": round(t_plain, 1), "netsim": exp_["netsim"],
                  "n_exemplars": exp_["n_exemplars"]},
        "pap": {"sub_iters_max": pr["sub_iters_max"], "step4_iters": pr["final"]["iters"],
                "ms": round(t_pap, 1), "sub_ms": round(pr["sub_ms"], 1),
                "merge_ms": round(pr["merge_ms"], 1), "final_ms": round(pr["final_ms"], 1),
                "netsim": pr["final"]["netsim"], "n_exemplars": pr["final"]["n_exemplars"]},
        "time_ratio_plain_over_pap": round(t_plain / t_pap, 3),
        "netsim_rel_diff": (pr["final"]["netsim"] - exp_["netsim"]) / abs(exp_["netsim"]),
    }
    # the same 32 uneven subsets with Step 4 also starting from the subsets' R,
    # and the paper's equal partition at several k (Table 2's k-sensitivity)
    (_, _, _, pc), t_pc = timed(lambda: capi.pap_run(S, len(offs) - 1, list(offs), damping=DAMPING,
                                                     max_iter=MAX_ITER, conv_iter=CONV_ITER,
                                                     R=R, A=A, carry_r=True), warm=False)
    out["pap"]["carry_r"] = {"ms": round(t_pc, 1), "step4_iters": pc["final"]["iters"],
                             "netsim_rel_diff": (pc["final"]["netsim"] - exp_["netsim"]) / abs(exp_["netsim"]),
                             "time_ratio_plain_over_pap": round(t_plain / t_pc, 3)}
    sweep = []
    for k in (8, 16, 32, 64):
        (_, _, _, pk), t_k = timed(lambda: capi.pap_run(S, k, None, damping=DAMPING, max_iter=MAX_ITER,
                                                        conv_iter=CONV_ITER, R=R, A=A), warm=False)
        sweep.append({"k": k, "ms": round(t_k, 1), "sub_iters_max": pk["sub_iters_max"],
                      "step4_iters": pk["final"]["iters"],
                      "netsim_rel_diff": (pk["final"]["netsim"] - exp_["netsim"]) / abs(exp_["netsim"]),
                      "time_ratio_plain_over_pap": round(t_plain / t_k, 3)})
    out["pap"]["k_sweep_equal_partition"] = sweep
    del S, R, A
    torch.cuda.empty_cache()

    # ---- landmark AP: 1e6 points, 1000 Gaussians in R^128, 20000 uniform landmarks;
    # plain AP is compared on the first 100000 points (1e6 points would need 12 TB)
    X, _ = synth.workload(3)
    Xd = torch.from_numpy(X).to(dev)
    (idx, lm, lr), t_lap_full = timed(lambda: capi.lap_run(Xd, 20000, "uniform", seed=synth.config_seed(3),
                                                           precision="bf16", damping=DAMPING,
                                                           max_iter=MAX_ITER, conv_iter=CONV_ITER))
    full = {"n": X.shape[0], "ms": round(t_lap_full, 1), "landmark_iters": lr["landmark"]["iters"],
            "n_exemplars": lr["n_exemplars"], "netsim": lr["netsim"],
            "assign_ms": round(lr["assign_ms"], 2), "landmark_ms": round(lr["landmark_ms"], 1)}
    del idx, lm
    # landmarks by the learned exemplar score (network trained on mixtures of
    # the landmark pool's density), against uniform landmarks
    t0 = time.perf_counter()
    Fl, Tl, _ = learned.make_dataset(learned.landmark_training_problems())
    Pl, P16l, ll = learned.train(Fl, Tl, epochs=60, batch=4096, lr=2e-3)
    train_s = time.perf_counter() - t0

    def lap_learned(Xv):
        score, t_sc = timed(lambda: learned.landmark_scores(Xv, 20000, Pl, P16l))
        (_, _, r), t = timed(lambda: capi.lap_run(Xv, 20000, "score", score=score, precision="bf16",
                                                  damping=DAMPING, max_iter=MAX_ITER,
                                                  conv_iter=CONV_ITER))
        return {"ms": round(t_sc + t, 1), "score_ms": round(t_sc, 1),
                "landmark_iters": r["landmark"]["iters"], "n_exemplars": r["n_exemplars"],
                "netsim": r["netsim"]}

    full["learned_landmarks"] = lap_learned(Xd)
    full["learned_landmarks"]["netsim_rel_vs_uniform"] = (
        (full["learned_landmarks"]["netsim"] - full["netsim"]) / abs(full["netsim"]))
    # Algorithm 3 in full (Steps 1-4, Step 4 refining the merged centres) on all 1e6 points
    (_, _, lf1), t_f1 = timed(lambda: capi.lap_run_full(Xd, 20000, 20000, seed=synth.config_seed(3),
                                                        precision="bf16", damping=DAMPING,
                                                        max_iter=MAX_ITER, conv_iter=CONV_ITER,
                                                        refine_rounds=REFINE_ROUNDS), warm=False)
    full["steps_1_4_refined"] = {"ms": round(t_f1, 1), "levels": lf1["levels"],
                                 "unassigned": lf1["unassigned"], "exemplars_at": lf1["exemplars_at"],
                                 "n_exemplars": lf1["n_exemplars"], "netsim": lf1["netsim"],
                                 "refine": [lf1["refine_rounds"], lf1["refine_removed"],
                                            lf1["refine_moved"]],
                                 "netsim_rel_vs_steps_1_2": (lf1["netsim"] - full["netsim"]) / abs(full["netsim"])}
    del Xd
    m = 100000
    Xs = torch.from_numpy(X[:m]).to(dev)
    S, _ = capi.ap_similarity(Xs, precision="bf16")
    R = capi.empty_square(m, dev, 0.0)
    A = capi.empty_square(m, dev, 0.0)
    (rp, exp_), t_plain = timed(plain)
    del R, A
    torch.cuda.empty_cache()
    (_, _, ls), t_lap = timed(lambda: capi.lap_run(Xs, 20000, "uniform", seed=synth.config_seed(3),
                                                   precision="bf16", damping=DAMPING,
                                                   max_iter=MAX_ITER, conv_iter=CONV_ITER))
    lrn = lap_learned(Xs)
    (_, _, lf0), t_full0 = timed(lambda: capi.lap_run_full(Xs, 20000, 20000, seed=synth.config_seed(3),
                                                           precision="bf16", damping=DAMPING,
                                                           max_iter=MAX_ITER, conv_iter=CONV_ITER))
    (_, _, lf), t_full = timed(lambda: capi.lap_run_full(Xs, 20000, 20000, seed=synth.config_seed(3),
                                                         precision="bf16", damping=DAMPING,
                                                         max_iter=MAX_ITER, conv_iter=CONV_ITER,
                                                         refine_rounds=REFINE_ROUNDS))
    # landmark count against net similarity (Table 1's trend), Steps 1-4 refined:
    # the smallest count within 0.5 % of plain AP is the equal-netsim point
    lsweep = []
    for L in (2000, 5000, 10000, 20000):
        (_, _, lq), t_q = timed(lambda: capi.lap_run_full(Xs, L, L, seed=synth.config_seed(3),
                                                          precision="bf16", damping=DAMPING,
                                                          max_iter=MAX_ITER, conv_iter=CONV_ITER,
                                                          refine_rounds=REFINE_ROUNDS), warm=False)
        lsweep.append({"landmarks": L, "ms": round(t_q, 1), "n_exemplars": lq["n_exemplars"],
                       "levels": lq["levels"],
                       "netsim_rel_diff": (lq["netsim"] - exp_["netsim"]) / abs(exp_["netsim"]),
                       "time_ratio_plain_over_lap": round(t_plain / t_q, 3)})
    equal = [q for q in lsweep if abs(q["netsim_rel_diff"]) <= 0.005]
    out["lap"] = {
        "workload": "1000 Gaussians in R^128 (sigma 0.5, centres N(0,16I)); 20000 uniform landmarks; "
                    "learned: the 20000 best exemplar scores of a 40000-point uniform pool",
        "scorer_training": {"problems": 12, "rows": int(Fl.shape[0]), "loss_first": round(ll[0], 4),
                            "loss_last": round(ll[-1], 4), "wall_s": round(train_s, 1)},
        "lap_steps_1_4": {"ms": round(t_full, 1), "levels": lf["levels"], "base_case": lf["base_case"],
                          "unassigned": lf["unassigned"], "exemplars_at": lf["exemplars_at"],
                          "n_exemplars": lf["n_exemplars"], "netsim": lf["netsim"],
                          "refine": {"rounds": lf["refine_rounds"], "removed": lf["refine_removed"],
                                     "moved": lf["refine_moved"]},
                          "time_ratio_plain_over_lap": round(t_plain / t_full, 3),
                          "netsim_rel_diff": (lf["netsim"] - exp_["netsim"]) / abs(exp_["netsim"]),
                          "without_refinement": {
                              "ms": round(t_full0, 1), "n_exemplars": lf0["n_exemplars"],
                              "netsim_rel_diff": (lf0["netsim"] - exp_["netsim"]) / abs(exp_["netsim"])}},
        "landmark_sweep_steps_1_4": lsweep,
        "equal_netsim": (dict(equal[0], rule="smallest landmark count with |netsim - plain| <= 0.5 %")
                         if equal else None),
        "lap_learned": dict(lrn, time_ratio_plain_over_lap=round(t_plain / lrn["ms"], 3),
                            netsim_rel_diff=(lrn["netsim"] - exp_["netsim"]) / abs(exp_["netsim"])),
        "full_1e6": full,
        "subsample": m,
        "plain": {"iters": rp["iters"], "ms": round(t_plain, 1), "netsim": exp_["netsim"],
                  "n_exemplars": exp_["n_exemplars"]},
        "lap": {"landmark_iters": ls["landmark"]["iters"], "ms": round(t_lap, 1),
                "netsim": ls["netsim"], "n_exemplars": ls["n_exemplars"]},
        "time_ratio_plain_over_lap": round(t_plain / t_lap, 3),
        "netsim_rel_diff": (ls["netsim"] - exp_["netsim"]) / abs(exp_["netsim"]),
    }
    del S, Xs
    torch.cuda.empty_cache()
    return out


def _oracle_sample(n_sample, seconds):
    """The float64 oracle on the first n_sample points of the same workload:
    S build, then iterations until ``seconds`` of iterating have passed."""
    from oracle import ap as oap
    from paper_0910_1650_gb300 import synth

    X, _ = synth.workload(1)
    Xs = X[:n_sample]
    S, _ = oap.build_similarity(Xs)
    R = np.zeros_like(S)
    A = np.zeros_like(S)
    t0 = time.perf_counter()
    its = 0
    while True:
        R, A = oap.iterate_once(S, R, A, DAMPING)
        its += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return its, dt


def _oracle_worker(args):
    n_sample, seconds = args
    return _oracle_sample(n_sample, seconds)


def _oracle_all_cores(n_sample, seconds):
    """The oracle as it stands, one process per host core (spawned, so no
    CUDA state is inherited), each iterating its own copy of the sample for
    ``seconds``.  Returns (total iterations, wall seconds, processes)."""
    import multiprocessing as mp

    procs = len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(n_sample, seconds)] * procs)
    wall = time.perf_counter() - t0
    # each worker's own iterating time bounds the rate; the pool start-up is excluded
    its = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return its, dt, procs, wall


def cpu_baseline(seconds):
    n_sample = 3000
    its, dt = _oracle_sample(n_sample, seconds)
    gbs1 = 20.0 * n_sample * n_sample * its / dt / 1e9
    its_p, dt_p, procs, wall = _oracle_all_cores(n_sample, seconds)
    gbs = 20.0 * n_sample * n_sample * its_p / dt_p / 1e9
    return {"value": round(gbs, 4), "unit": "GB/s", "cores": procs, "kind": "oracle",
            "sample": f"float64 oracle, first {n_sample} points of the N=20000 workload: one process "
                      f"per host core ({procs}), {its_p} iterations in {dt_p:.1f} s "
                      f"(pool wall {wall:.1f} s)",
            "one_thread": {"value": round(gbs1, 4), "unit": "GB/s", "cores": 1,
                           "sample": f"{its} iterations in {dt:.1f} s (numpy, one thread)"}}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    n_sample = 3000
    per_step = max(1.0, 60.0 / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        _oracle_sample(n_sample, per_step / 4)
    tot_its, tot_dt, procs = 0, 0.0, 1
    for _ in range(args.steps):
        its, dt, procs, _ = _oracle_all_cores(n_sample, per_step)
        tot_its += its
        tot_dt += dt
    v = 20.0 * n_sample * n_sample * tot_its / tot_dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_POINTS, "d": DIM,
                       "sample_points": n_sample},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": procs, "kind": "oracle",
                             "sample": f"float64 oracle on the first {n_sample} points, one process "
                                       f"per host core ({procs}), {tot_its} iterations"},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def similarity_only(args):
    """The similarity build alone (bf16 tensor-core Gram product with the
    distance epilogue, plus means, centring and the median) on one image-like
    problem: the tensor-bound case of the batch workload, for profiling."""
    import torch

    from paper_0910_1650_gb300 import capi, synth

    X, _ = synth.image_like(args.n, args.similarity_only, 20, stream=7)
    Xd = torch.from_numpy(X).cuda()
    S = capi.empty_square(args.n, "cuda")
    for _ in range(args.warmup):
        capi.ap_similarity(Xd, S=S, precision="bf16")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(args.steps):
        capi.ap_similarity(Xd, S=S, precision="bf16")
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    fl = 2.0 * args.n * args.n * args.similarity_only
    print(json.dumps({"case": "similarity", "n": args.n, "d": args.similarity_only,
                      "ms": round(ms, 4), "tflops": round(fl / ms / 1e9, 1)}), flush=True)


def batch_similarity(args):
    """The batched similarity build alone on the first COUNT problems of the
    256-problem image batch (features uploaded once, one S arena, workspace
    allocated once): --warmup untimed calls, then --steps timed ones; prints
    one JSON line, for profiling."""
    import numpy as np
    import torch

    from paper_0910_1650_gb300 import batched, capi

    probs = list(batched.image_batch(args.batch_similarity))
    rows = [p.shape[0] for p in probs]
    d = probs[0].shape[1]
    X = torch.from_numpy(np.concatenate(probs)).cuda()
    xoff = np.concatenate([[0], np.cumsum(rows)[:-1]]) * d
    off, n, ld, total = batched.layout(rows)
    S = torch.empty(total, dtype=torch.float32, device="cuda")
    ws = capi.ap_similarity_batched_workspace(n, d, X.device)
    for _ in range(args.warmup):
        capi.ap_similarity_batched(X, xoff, n, S, off, ld, precision="bf16", ws=ws)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(args.steps):
        capi.ap_similarity_batched(X, xoff, n, S, off, ld, precision="bf16", ws=ws)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    fl = sum(2.0 * m * m * d for m in rows)
    print(json.dumps({"case": "batch_similarity", "problems": len(rows), "d": d,
                      "sum_n2": float(sum(float(m) * m for m in rows)), "ms": round(ms, 4),
                      "tflops": round(fl / ms / 1e9, 1)}), flush=True)


def lap_only(args):
    """Landmark AP alone (Steps 1-2 of Algorithm 3: landmark similarity and
    AP, then the tensor-core nearest-exemplar assignment) on the first N
    points of the 1e6-point workload, for profiling the assignment GEMM."""
    import torch

    from paper_0910_1650_gb300 import capi, synth

    X, _ = synth.workload(3, scale=args.lap_only / 1_000_000)
    Xd = torch.from_numpy(X).cuda()
    _, _, r = capi.lap_run(Xd, min(20000, args.lap_only), "uniform", seed=synth.config_seed(3),
                           precision="bf16", damping=DAMPING, max_iter=MAX_ITER, conv_iter=CONV_ITER)
    c = r["n_exemplars"]
    fl = 2.0 * args.lap_only * c * X.shape[1]
    print(json.dumps({"case": "lap", "n": args.lap_only, "exemplars": c, "assign_ms": round(r["assign_ms"], 3),
                      "assign_tflops": round(fl / r["assign_ms"] / 1e9, 1), "ms": round(r["landmark_ms"], 2)}),
          flush=True)


def sweep_configs(args):
    """Every admissible sweep configuration (cluster 1-16 x float4 per thread
    x stages) timed at each N of --sweep-configs on random 16-D points (bf16
    S, damping 0.9, 6 fixed iterations, per-launch CUDA-event time), with the
    default configuration; one JSON line per N."""
    import torch

    from paper_0910_1650_gb300 import capi

    peaks, _ = _peaks()
    for n in args.sweep_configs:
        torch.manual_seed(0)
        X = torch.randn(n, 16, device="cuda")
        S, _ = capi.ap_similarity(X, precision="bf16")
        R = capi.empty_square(n, "cuda", 0.0)
        A = capi.empty_square(n, "cuda", 0.0)
        dflt = capi.ap_sweep_get_config(n)
        rows = []
        for cl in range(1, 17):
            for ept in range(1, 5):
                for ns in (2, 3, 4):
                    try:
                        capi.ap_sweep_set_config(n, cl, ept, ns)
                    except capi.ApgbError:
                        continue
                    cfg = capi.ap_sweep_get_config(n)
                    R.zero_()
                    A.zero_()
                    _, _, r, _ = capi.ap_iterate(S, R, A, damping=0.9, max_iter=6, conv_iter=0,
                                                 time_sweep=True, decisions=False)
                    rows.append((r["sweep_ms"] / max(1, r["sweep_launches"]), cl, ept, ns,
                                 cfg["clusters"] * cl))
        capi.ap_sweep_set_config(n)
        rows.sort()
        frac = lambda ms: round(20.0 * n * n / 1e6 / ms / peaks["hbm_gbs"], 3)
        key = (dflt["cluster"], dflt["ept"], dflt["stages"])
        dms = [m for m, c, e, st, _ in rows if (c, e, st) == key]
        print(json.dumps({"case": "sweep_configs", "n": n,
                          "default": {"cluster": key[0], "ept": key[1], "stages": key[2],
                                      "ctas": dflt["clusters"] * key[0],
                                      "ms": round(dms[0], 3) if dms else None,
                                      "frac": frac(dms[0]) if dms else None},
                          "fastest": [{"cluster": c, "ept": e, "stages": st, "ctas": k, "ms": round(m, 3),
                                       "frac": frac(m)} for m, c, e, st, k in rows[:5]],
                          "fastest_power_of_two": [{"cluster": c, "ept": e, "stages": st, "ctas": k,
                                                    "ms": round(m, 3), "frac": frac(m)}
                                                   for m, c, e, st, k in rows if c & (c - 1) == 0][:1]}),
              flush=True)
        del S, R, A
        torch.cuda.empty_cache()


def lap_full_only(args):
    """Algorithm 3 in full (Steps 1-4, the refinement included) on all 1e6
    points of the 1e6-point workload, once, as the time-to-converge section
    runs it; for the launch list of that call."""
    import torch

    from paper_0910_1650_gb300 import capi, synth

    X, _ = synth.workload(3)
    Xd = torch.from_numpy(X).cuda()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    _, _, r = capi.lap_run_full(Xd, 20000, 20000, seed=synth.config_seed(3), precision="bf16",
                                damping=DAMPING, max_iter=MAX_ITER, conv_iter=CONV_ITER,
                                refine_rounds=REFINE_ROUNDS)
    ev[1].record()
    ev[1].synchronize()
    print(json.dumps({"case": "lap_full", "n": X.shape[0], "ms": round(ev[0].elapsed_time(ev[1]), 1),
                      "levels": r["levels"], "unassigned": r["unassigned"][:r["levels"]],
                      "n_exemplars": r["n_exemplars"], "refine_rounds": r["refine_rounds"]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--pap-table2", action="store_true",
                    help="only the PAP k sweep on Table 2's shape (prints one JSON line)")
    ap.add_argument("--sharded", action="store_true",
                    help="split the rows of S, R, A over the ranks (one all-reduce per iteration) "
                         "and time the sweep to convergence")
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ttc", action="store_true",
                    help="skip the time-to-converge comparisons (partition and landmark AP)")
    ap.add_argument("--n", type=int, default=N_POINTS,
                    help="points (default: the 20000-point workload; smaller for profiling)")
    ap.add_argument("--lap-only", type=int, default=0, metavar="N",
                    help="profiling aid: one landmark AP (Steps 1-2, 20000 landmarks, bf16) on the "
                         "first N points of the 1e6-point workload, print one JSON line")
    ap.add_argument("--sweep-configs", type=int, nargs="+", default=None, metavar="N",
                    help="profiling aid: time every admissible sweep configuration at each N, "
                         "one JSON line per N")
    ap.add_argument("--lap-full-only", action="store_true",
                    help="profiling aid: one call of Algorithm 3 Steps 1-4 (refined) on all 1e6 "
                         "points, print one JSON line")
    ap.add_argument("--similarity-only", type=int, default=0, metavar="D",
                    help="profiling aid: time the bf16 similarity build alone on one image-like "
                         "problem of --n points and D features, print one JSON line")
    ap.add_argument("--batch-similarity", type=int, default=0, metavar="COUNT",
                    help="profiling aid: time the batched bf16 similarity build alone on the first "
                         "COUNT problems of the image batch, print one JSON line")
    args = ap.parse_args()
    if args.batch_similarity:
        batch_similarity(args)
        return
    if args.similarity_only:
        similarity_only(args)
        return
    if args.lap_only:
        lap_only(args)
        return
    if args.lap_full_only:
        lap_full_only(args)
        return
    if args.sweep_configs:
        sweep_configs(args)
        return
    if args.pap_table2:
        import torch
        print(json.dumps(pap_table2(torch.device("cuda", 0))), flush=True)
        return
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.sharded:
        run_sharded(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
