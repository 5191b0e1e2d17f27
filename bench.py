#!/usr/bin/env python3
"""Benchmark of the QED event generator (arXiv:2008.10468) on GB300.

Headline: sub-stepped particle-steps per second (executed sub-steps of
Algorithms 1/2 per second) for one global step of the clumped mixed population:
2^24 particles (25% e-, 25% e+, 50% photons), 1% of them in a contiguous hot
clump with chi log-uniform in [10, 100], the rest chi in [1e-3, 1e-2];
emission + pair production with the in-step cascade.  Every timed step starts
from the same population (restored, then L2 flushed, outside the timed window)
with a new step index, i.e. new random draws.

Also reported: F1/F2 evaluations per second on 2^28 log-uniform arguments in
[1e-4, 50] (array mode, 12 bytes per evaluation, and in-kernel generation
mode), per-kernel times from CUDA events on the library stream, the roofline of
the dominant kernel, the end-to-end rate through host buffers, SM clocks during
the timed region, and the FP64 oracle on the host cores (a bounded sample).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PARTICLES = 1 << 24
SWEEP_N = 1 << 28
SEED_UNIFORM = 20081046 + 1
SEED_CLUMPED = 20081046 + 3
SEED_SWEEP = 20081046 + 2
SEED_CASCADE = 20081046 + 4
CASCADE_CELLS = 4096
CASCADE_CAPACITY = 1 << 26
CASCADE_DRAIN_CHI = 0.05
# DRAM traffic of the hot pass is not reported per run: a capture of its
# counters over whole steps of the full-size workload is larger than the
# profiling rules allow, and at the 2^22 rows that may be captured the
# children's writes stay in the 129 MB L2 (profiles/hot_pass_traffic_clumped_2p22.md).
HOT_TRAFFIC_NOTE = ("null: a capture of the pass's launches at 2^22 rows reads 90 MB per step "
                    "from DRAM while its writes (the children) stay in L2 at that size; a "
                    "full-size capture of these counters is outside the profiling size rule")

METRIC = "particle-steps/sec (sub-stepped)"
UNIT = "substeps/s"
WORKLOAD = ("clumped mixed population 2^24 (25% e-, 25% e+, 50% photons; 1% hot clump "
            "chi 10-100), emission + pairs + in-step cascade, one global step dt = 0.1 T")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() in ("active", "yes", "0x1", "1"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# distributed helpers (one process per GPU; the path shards by particles)
# --------------------------------------------------------------------------
def dist_init(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allreduce_max(pg, v, device="cuda"):
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(pg, v, device="cuda"):
    """Sum over the ranks (work done by the whole job)."""
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def job_rate(pg, units, ms, device="cuda"):
    """Whole-job throughput of independent shards: all ranks' units over the
    slowest rank's time (weak scaling, no data-path collective)."""
    t_max = allreduce_max(pg, ms, device)
    return allreduce_sum(pg, units, device) / (t_max / 1e3), t_max


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores, bounded sample
# --------------------------------------------------------------------------
def population_sample(arr, m, seed):
    """m rows of the population with the same hot fraction (stratified)."""
    n = len(arr["px"])
    n_hot = int(round(n * 0.01))
    h0 = (n - n_hot) // 2
    rng = np.random.default_rng(seed)
    k_hot = max(1, int(round(m * 0.01)))
    hot = rng.choice(np.arange(h0, h0 + n_hot), k_hot, replace=False)
    cold_pool = rng.choice(n - n_hot, m - k_hot, replace=False)
    cold = np.where(cold_pool < h0, cold_pool, cold_pool + n_hot)
    # random order: the oracle's threads take contiguous ranges, and a sorted
    # sample would put the whole clump on one thread
    rows = rng.permutation(np.concatenate([hot, cold]))
    from paper_2008_10468_gb300 import inputs as I
    return I.subset(arr, rows)


def cpu_baseline(arr, seed, budget_s=12.0):
    """The FP64 oracle on the host cores (threads take 32-row chunks from a
    shared counter): once with F1/F2 by quadrature, once with the memoised
    table a production CPU code would use (within 1e-10 of the quadrature).
    Each on a stratified sample sized to about budget_s seconds."""
    import oracle as O
    cores = os.cpu_count() or 1
    cf = O.make_config(seed, process_mask=3, cascade=1, threads=cores)

    def timed(memo):
        m = 2000
        while True:
            sub = population_sample(arr, m, 11)
            t0 = time.perf_counter()
            if memo:
                with O.memoised_F1F2(threads=cores):
                    t0 = time.perf_counter()
                    _, st = O.event_step_mt(cf, sub, 100, capacity=m * 64)
            else:
                _, st = O.event_step_mt(cf, sub, 100, capacity=m * 64)
            dt = time.perf_counter() - t0
            if dt > budget_s / 4 or m >= 1 << 21:
                return m, st, dt
            m = min(1 << 21, int(m * max(2.0, budget_s / 2 / max(dt, 1e-3))))

    m, st, dt = timed(False)
    mm, stm, dtm = timed(True)
    note = ("host threads as the container reports them (os.cpu_count); the host "
            "may hold more cores than this process sees")
    return {"value": st["substeps"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d rows of the same population (1%% hot, stratified), one step, "
                      "%d sub-steps in %.1f s; F1/F2 by quadrature" % (m, st["substeps"], dt),
            "memoised": {"value": stm["substeps"] / dtm, "unit": UNIT, "cores": cores,
                         "kind": "oracle, F1/F2 from a memoised FP64 table (within 1e-10)",
                         "sample": "%d rows, %d sub-steps in %.1f s"
                                   % (mm, stm["substeps"], dtm)},
            "cores_note": note}


def measured_peaks():
    """Rates of the arithmetic the event kernels run on, from the library's
    probes on this GPU (qed_peak_probe), with the SM clock they ran at."""
    from paper_2008_10468_gb300 import qed
    out = {}
    for name, kind in (("mul32_per_s", qed.PROBE_MUL32), ("fma32_flop_per_s", qed.PROBE_FMA32),
                       ("ex2_per_s", qed.PROBE_EX2), ("alu_per_s", qed.PROBE_ALU)):
        rate, ms = qed.peak_probe(kind, 1 << 16)
        out[name] = rate
        out[name.replace("_per_s", "_ms")] = ms
    return out


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_gb300(args):
    import torch
    from paper_2008_10468_gb300 import inputs as I
    from paper_2008_10468_gb300 import qed

    rank, world, local, pg = dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_peak, peak_kind = peaks()

    n = args.particles
    arr = I.clumped_mixed(n, SEED_CLUMPED + 1000 * rank)
    cap = n + 2 * n       # the hot clump cascades: ~35 children per hot particle
    pristine = qed.ParticleStore.from_numpy(arr, capacity=cap, device=dev)
    store = qed.ParticleStore(cap, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2
    ctx = qed.Context(seed=SEED_CLUMPED + rank, process_mask=3, cascade=True)
    if getattr(args, "tail_rows", None) is not None:
        ctx.set_tail(args.tail_rows)
    stream = torch.cuda.current_stream()

    def restore():
        for k in qed.FLOAT_FIELDS + ("id", "type"):
            getattr(store, k)[:n].copy_(getattr(pristine, k)[:n])
        store.type[n:].fill_(qed.REMOVED)
        store.count.fill_(n)
        flush.fill_(1)

    for w in range(args.warmup):
        restore()
        ctx.event_step(store, 1000 + w)
    torch.cuda.synchronize()
    peaks_measured = measured_peaks()

    # headline: each step is the library's one-step graph (generations in a
    # device-side loop), timed with CUDA events on the library stream
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.5)   # the sampler's first record comes before the timed steps
    total_ms = 0.0
    sub_total = 0
    launches_timed = 0
    agg = {"emissions": 0, "pairs": 0, "children": 0, "candidates": 0, "plans": 0,
           "passes": 0, "max_N": 0, "substeps_warp": 0}
    for k in range(args.steps):
        restore()
        torch.cuda.synchronize()
        barrier(pg)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ctx.event_step(store, 2000 + k)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
        total_ms += e0.elapsed_time(e1)
        sub_total += st["substeps"]
        # our kernels per graph step: step index, step init, three per loop
        # generation, and the tail pass's four (launched whether or not it ran;
        # when it ran it counts as one of the passes)
        launches_timed += 2 + 3 * (st["passes"] - st["tail"]) + 4
        for key in agg:
            agg[key] = max(agg[key], st[key]) if key == "max_N" else agg[key] + st[key]
        if st["status"] != 0:
            raise SystemExit("step failed with status %d" % st["status"])
    clk = clocks.stop()

    # per-kernel times: the same steps again, launched kernel by kernel with
    # CUDA events around each launch (the graph cannot be split)
    ctx.profile_read()
    ctx.profile(True)
    kern = {}
    prof_steps = max(3, min(args.steps, 10))
    prof_ms = 0.0
    pagg = {"children": 0, "emissions": 0, "substeps_warp": 0}
    for k in range(prof_steps):
        restore()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pst = ctx.event_step(store, 2000 + k)
        e1.record(stream)
        torch.cuda.synchronize()
        prof_ms += e0.elapsed_time(e1)
        for key in pagg:
            pagg[key] += pst[key]
        for name, (ms, nl) in ctx.profile_read().items():
            a = kern.setdefault(name, [0.0, 0])
            a[0] += ms
            a[1] += nl
    ctx.profile(False)

    value, t_max = job_rate(pg, sub_total, total_ms)

    # dominant kernel and its roofline (event-timed on the library stream)
    dom = max(("cold", "hot"), key=lambda k: kern.get(k, [0])[0])
    steps = prof_steps
    if dom == "cold":
        # algorithmic bytes of the thread-per-particle pass per step: read type of
        # every row (1 B) and p, E, B, id of every active row (44 B); write child
        # rows with their remaining time (57 B) and changed momenta (12 B)
        rows = n + pagg["children"] / steps
        bytes_step = 45.0 * rows + 57.0 * pagg["children"] / steps + 12.0 * pagg["emissions"] / steps
        t_launch = kern["cold"][0] / kern["cold"][1]
        per_launch = bytes_step / (kern["cold"][1] / steps)
        achieved = per_launch / (t_launch / 1e3) / 1e9
        roof = {"kernel": "k_cold", "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                "peak_kind": peak_kind}
    else:
        # hot pass: its work is Philox4x32-10, 4 32-bit multiply results per
        # round, 40 per block, one block per two sub-steps -> 20 multiplies per
        # sub-step.  Peak: the same multiplies as Philox issues them (high and
        # low word of each 32 x 32 -> 64 product, with the xors between),
        # measured on this GPU by the library's probe.
        mul_peak = peaks_measured["mul32_per_s"] / 1e12
        t_launch = kern["hot"][0] / kern["hot"][1] / 1e3
        per_launch = 20.0 * pagg["substeps_warp"] / kern["hot"][1]
        achieved = per_launch / t_launch / 1e12
        roof = {"kernel": "k_hot_lanes + k_step (hot pass)", "bound": "alu", "achieved": achieved,
                "peak": mul_peak, "unit": "T int32-mul/s", "frac": achieved / mul_peak,
                "traffic": None, "traffic_note": HOT_TRAFFIC_NOTE,
                "peak_kind": "measured: qed_peak_probe MUL32 (Philox multiplies) on this GPU"}

    # synchrotron sweep, array mode and generation mode
    sweep = run_sweep(ctx, dev, args, hbm_peak, peak_kind)

    # end to end from pinned host buffers through the public API
    e2e = None if args.no_e2e else run_e2e(ctx, arr, cap, dev, args, pg)

    # cascade batch: many steps of growing pools in one captured graph
    cascade = None if args.no_cascade else run_cascade(dev, args)

    # learned sampler against rejection on the same population
    sampler = None if args.no_sampler else run_sampler(arr, pristine, store, cap, n, dev, args,
                                                        restore, value)

    # the same step with the Boris push before every e+- draw
    push = None if args.no_push else run_push(store, dev, args, restore, value)

    # per-cell planning over the same store (64 rows per cell)
    cells = run_plan_cells(ctx, pristine, n, dev, hbm_peak, peak_kind)

    # the uniform-field electrons (1e5, emission only, one step)
    uniform = run_uniform(dev, args)

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "particles_per_s": world * n * args.steps / (t_max / 1e3),
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N_PARTICLES else WORKLOAD + " (reduced: %d rows)" % n,
                   "particles": n, "capacity": cap,
                   "l2": "inputs (822 MB) larger than L2, and a 256 MB buffer written before "
                         "each timed step", "parallelism": "independent particle shards"
                                                       if world > 1 else "single GPU"},
        "per_step": {k: v / args.steps for k, v in agg.items() if k != "max_N"},
        "max_N": agg["max_N"],
        "kernels_ms_per_step": {k: v[0] / steps for k, v in kern.items() if v[1]},
        "profiled_steps": {"steps": prof_steps, "ms_per_step": prof_ms / prof_steps,
                           "note": "kernel-by-kernel launches with CUDA events around each "
                                   "(the source of kernels_ms_per_step and roofline); the "
                                   "headline steps run as one graph each"},
        "roofline": roof,
        "peaks_measured": peaks_measured,
        "sweep": sweep,
        "uniform_field": uniform,
        "sampler": sampler,
        "push": push,
        "plan_cells": cells,
        "cascade": cascade,
        "e2e": e2e,
        "gpu_launches": launches_timed,
        "clocks": clk,
    }
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = cpu_baseline(arr, SEED_CLUMPED)
        print(json.dumps(res))
    if pg is not None:
        pg.destroy_process_group()


def run_sweep(ctx, dev, args, hbm_peak, peak_kind):
    import torch
    from paper_2008_10468_gb300 import inputs as I
    from paper_2008_10468_gb300 import qed
    SWEEP_N = args.sweep_n
    y = torch.from_numpy(I.sweep_points(SWEEP_N, SEED_SWEEP)).to(dev)
    F1 = torch.empty_like(y)
    F2 = torch.empty_like(y)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        ctx.synchrotron_F1F2(y, F1, F2)
    torch.cuda.synchronize()
    reps = max(3, args.steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.synchrotron_F1F2(y, F1, F2)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    evals = SWEEP_N / (ms / 1e3)
    gbs = 12.0 * SWEEP_N / (ms / 1e3) / 1e9
    # generation mode: no argument or result traffic
    chk = torch.zeros(1, device=dev)
    for _ in range(2):
        ctx.synchrotron_generate(7, SWEEP_N, 1e-4, 50.0, chk)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        ctx.synchrotron_generate(7, SWEEP_N, 1e-4, 50.0, chk)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_gen = e0.elapsed_time(e1) / reps
    del y, F1, F2

    # binary64 functions (the double-precision level of Table 1), same points:
    # 8 B in + 16 B out per evaluation; the arithmetic is two degree-11
    # polynomials (22 multiply-adds, 44 FP64 flops) plus exp for x >= 1/2, on
    # the FP64 pipe (nominal 1.25 TFLOP/s dense on GB300; not in the measured
    # peaks file)
    y64 = torch.from_numpy(I.sweep_points(SWEEP_N, SEED_SWEEP).astype(np.float64)).to(dev)
    G1 = torch.empty_like(y64)
    G2 = torch.empty_like(y64)
    for _ in range(2):
        qed.synchrotron_F1F2_f64(y64, G1, G2, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        qed.synchrotron_F1F2_f64(y64, G1, G2, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / reps
    del y64, G1, G2
    tf64 = 44.0 * SWEEP_N / (ms64 / 1e3) / 1e12
    f64 = {"evals_per_s": SWEEP_N / (ms64 / 1e3), "ms": ms64,
           "hbm_gbs": 24.0 * SWEEP_N / (ms64 / 1e3) / 1e9,
           "fp64": {"achieved": tf64, "peak": 1.25, "unit": "TFLOP/s", "frac": tf64 / 1.25,
                    "peak_kind": "nominal (GB300 dense FP64)", "flops_per_eval": 44}}
    return {"n": SWEEP_N, "evals_per_s": evals, "ms": ms,
            "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "peak_kind": peak_kind, "bytes_per_eval": 12},
            "generate_evals_per_s": SWEEP_N / (ms_gen / 1e3), "generate_ms": ms_gen,
            "binary64": f64}


def run_cascade(dev, args):
    """Independent cells with power-law counts; all global steps in one CUDA
    graph, photons below the drain chi moved to the spectrum at each step's
    compaction.  The pools grow by cascades; a step that would exceed the
    capacity stops the run with QED_ERR_CAPACITY and the later steps do
    nothing, so the record gives the steps completed.  Timed on the second
    launch of the graph (the first warms up), from the same initial pools."""
    import torch
    from paper_2008_10468_gb300 import inputs as I
    from paper_2008_10468_gb300 import qed
    arr, _cell = I.cascade_cells(CASCADE_CELLS, SEED_CASCADE)
    n0 = len(arr["px"])
    cap = CASCADE_CAPACITY
    pristine = qed.ParticleStore.from_numpy(arr, capacity=n0, device=dev)
    store = qed.ParticleStore(cap, device=dev)
    ctx = qed.Context(seed=SEED_CASCADE, process_mask=3, cascade=True, drain_chi=CASCADE_DRAIN_CHI)

    def restore():
        for k in qed.FLOAT_FIELDS + ("id", "type"):
            getattr(store, k)[:n0].copy_(getattr(pristine, k)[:n0])
        store.type[n0:].fill_(qed.REMOVED)
        store.count.fill_(n0)

    # the full run once: which steps complete before the capacity stops it
    restore()
    ctx.graph_capture(store, 0, args.cascade_steps)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.graph_launch()
    e1.record(stream)
    torch.cuda.synchronize()
    full_ms = e0.elapsed_time(e1)
    full = ctx.graph_read_stats()
    k = sum(1 for st in full if st["status"] == 0)
    failed = next((st for st in full if st["status"] != 0), None)
    # then exactly the completed steps, as one graph, timed on its second launch
    ms, sub, done, spec = None, 0, [], None
    if k > 0:
        restore()
        ctx.graph_capture(store, 0, k)
        ctx.graph_launch()
        torch.cuda.synchronize()
        restore()
        ctx.read_spectrum(reset=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        done = ctx.graph_read_stats()
        if any(st["status"] != 0 for st in done):
            raise SystemExit("cascade steps that completed in the full run failed when rerun")
        sub = sum(st["substeps"] for st in done)
        spec = ctx.read_spectrum()
    return {
        "cells": CASCADE_CELLS, "particles0": n0, "capacity": cap, "steps": args.cascade_steps,
        "steps_completed": k,
        "per_step_substeps_per_s": sub / (ms / 1e3) if ms else None,
        "note": "the pools grow about tenfold per step and exceed the capacity (2^26 rows) "
                "at the second step; under the drain rule the run stops there with "
                "QED_ERR_CAPACITY, so the rate is that of the completed step(s), timed as "
                "a graph of exactly those steps, not of 100 steps",
        "status": failed["status"] if failed else 0,
        "required_capacity": failed["required_capacity"] if failed else 0,
        "ms": ms, "substeps": sub, "substeps_per_s": sub / (ms / 1e3) if ms else None,
        "full_run_ms": full_ms,
        "count_after": [st["count"] for st in done],
        "substeps_per_step": [st["substeps"] for st in done],
        "drained_photon_weight": float(spec.sum()) if spec is not None else 0.0,
        "drain_chi": CASCADE_DRAIN_CHI,
    }


def run_uniform(dev, args):
    """1e5 electrons (gamma 1e2..1e4, chi 0.1..10) in their crossed fields,
    emission only, one global step: sub-steps per second over K steps, each
    from the same population with a new step index."""
    import torch
    from paper_2008_10468_gb300 import inputs as I
    from paper_2008_10468_gb300 import qed
    n = 100_000
    arr = I.uniform_field_electrons(n, SEED_UNIFORM)
    cap = 16 * n   # about 9.5 photons per electron and step
    pristine = qed.ParticleStore.from_numpy(arr, capacity=n, device=dev)
    store = qed.ParticleStore(cap, device=dev)
    ctx = qed.Context(seed=SEED_UNIFORM, process_mask=1, cascade=False)
    stream = torch.cuda.current_stream()

    def restore():
        for k in qed.FLOAT_FIELDS + ("id", "type"):
            getattr(store, k)[:n].copy_(getattr(pristine, k)[:n])
        store.type[n:].fill_(qed.REMOVED)
        store.count.fill_(n)

    for w in range(3):
        restore()
        ctx.event_step(store, 500 + w)
    total, subs, st = 0.0, 0, None
    for k in range(args.steps):
        restore()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ctx.event_step(store, 600 + k)
        e1.record(stream)
        torch.cuda.synchronize()
        if st["status"] != 0:
            raise SystemExit("uniform-field step failed with status %d" % st["status"])
        total += e0.elapsed_time(e1)
        subs += st["substeps"]
    return {"workload": "uniform-field electrons: 1e5 e-, gamma log-uniform 1e2..1e4, chi "
                        "log-uniform 0.1..10, crossed fields, emission only, one step",
            "substeps_per_s": subs / (total / 1e3), "ms_per_step": total / args.steps,
            "substeps_per_step": subs / args.steps, "emissions_per_step": st["emissions"],
            "max_N": st["max_N"]}


def run_push(store, dev, args, restore, plain_value):
    """The clumped step with the Boris push of Algorithm 1 before every e+-
    draw (qed_event_step_push): one lane per particle through its sub-steps
    in order, the whole cascade in one persistent launch that takes children
    as they come; beside it the same step generation by generation
    (tail_rows 0) and with one sub-step per cell."""
    import torch
    from paper_2008_10468_gb300 import qed
    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 5))

    def timed(ctx, call):
        for w in range(2):
            restore()
            call(ctx, 4000 + w)
        ms, subs, agg = 0.0, 0, {"emissions": 0, "pairs": 0, "children": 0, "passes": 0}
        for k in range(steps):
            restore()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = call(ctx, 2000 + k)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            subs += st["substeps"]
            for key in agg:
                agg[key] += st[key]
            if st["status"] != 0:
                raise SystemExit("push step failed with status %d" % st["status"])
        return ms, subs, agg

    def plain_push(ctx, step):
        return ctx.event_step(store, step, push=True)

    ctx = qed.Context(seed=SEED_CLUMPED, process_mask=3, cascade=True)
    total_ms, subs, agg = timed(ctx, plain_push)
    value = subs / (total_ms / 1e3)
    # one profiled step: the persistent kernel's share
    restore()
    ctx.profile_read()
    ctx.profile(True)
    plain_push(ctx, 2000)
    kern = ctx.profile_read()
    ctx.profile(False)
    # the generation loop (one launch per cascade generation, the host
    # checking each), for comparison
    gen_ctx = qed.Context(seed=SEED_CLUMPED, process_mask=3, cascade=True)
    gen_ctx.set_tail(0)
    g_ms, g_subs, g_agg = timed(gen_ctx, plain_push)
    # one sub-step per cell (64 consecutive rows per cell), Algorithm 1 as printed
    restore()
    n = int(store.count.item())
    cell = (torch.arange(n, device=store.device, dtype=torch.int64) // 64).to(torch.int32)
    ncells = (n + 63) // 64
    c_ms, c_subs, _ = timed(ctx, lambda c, step: c.event_step_push_cells(store, step, cell,
                                                                           ncells))
    cells = {"rows_per_cell": 64, "ms_per_step": c_ms / steps, "substeps_per_step": c_subs / steps,
             "substeps_per_s": c_subs / (c_ms / 1e3)}
    return {"substeps_per_s": value, "ms_per_step": total_ms / steps, "steps": steps,
            "with_cells": cells,
            "per_step": {k: v / steps for k, v in agg.items()},
            "substeps_per_step": subs / steps,
            "k_push_ms_one_step": kern.get("hot", (0.0, 0))[0],
            "relative_to_step_without_push": value / plain_value,
            "generations": {"ms_per_step": g_ms / steps, "substeps_per_s": g_subs / (g_ms / 1e3),
                            "passes_per_step": g_agg["passes"] / steps},
            "note": "the whole cascade in one persistent launch (children taken as they are "
                    "reserved); 'generations' is the same step one launch per generation"}


def run_plan_cells(ctx, store, n, dev, hbm_peak, peak_kind):
    """qed_plan_cells over the 2^24 store, 64 consecutive rows per cell: rows/s
    and the pass's algorithmic bytes (the fields the planner reads, 37 B: type,
    momentum, E and B; and the row's 4 B cell index; the counts are atomics on
    256K words) against HBM."""
    import torch
    ncells = (n + 63) // 64
    cell = (torch.arange(n, device=dev, dtype=torch.int64) // 64).to(torch.int32)
    N_cell = torch.empty(ncells, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        ctx.plan_cells(store, n, cell, ncells, N_cell)
    reps = 20
    total = 0.0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(reps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.plan_cells(store, n, cell, ncells, N_cell)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    ms = total / reps
    gbs = 41.0 * n / (ms / 1e3) / 1e9
    return {"rows": n, "cells": ncells, "ms": ms, "rows_per_s": n / (ms / 1e3),
            "max_cell_N": int(N_cell.max().item()),
            "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "peak_kind": peak_kind, "bytes_per_row": 41}}


def run_sampler(arr, pristine, store, cap, n, dev, args, restore, plain_value):
    """Train the learned samplers on the GPU (emission: 2^26 exact-CDF samples
    in batches of 2048; pair production: the same), measure their per-bin CDF
    error, and time the clumped step with them against rejection (which is
    kept outside their usable bins): per sub-step (sampler_mode 1: each
    sub-step an event with the tabulated probability, the network per event
    on one warp) and event-driven (sampler_mode 2: the sub-steps to the next
    event drawn at once, one lane per particle, each warp's events through the
    network together on the tensor cores; photons too, with the pair
    network)."""
    import torch
    from paper_2008_10468_gb300 import qed
    ctx = qed.Context(seed=SEED_CLUMPED, process_mask=3, cascade=True, sampler=True,
                      sampler_max_err=1e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = ctx.sampler_train(20081051, 1 << 26, batch=2048, lr=3e-3)
    train_s = time.perf_counter() - t0
    err = ctx.sampler_evaluate()
    usable = err <= 1e-3
    params = ctx.sampler_save()
    ctx.sampler_process(qed.PROC_PAIR)
    t0 = time.perf_counter()
    ploss = ctx.sampler_train(20081052, 1 << 26, batch=2048, lr=3e-3)
    ptrain_s = time.perf_counter() - t0
    perr = ctx.sampler_evaluate()
    pparams = ctx.sampler_save()
    ctx.sampler_process(qed.PROC_EMISSION)
    stream = torch.cuda.current_stream()

    def timed(c):
        for w in range(2):
            restore()
            c.event_step(store, 4000 + w)
        total_ms, agg = 0.0, {}
        for k in range(args.steps):
            restore()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = c.event_step(store, 2000 + k)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            if st["status"] != 0:
                raise SystemExit("sampler step failed with status %d" % st["status"])
            for key in ("substeps", "emissions", "pairs", "sampler_events", "sampler_pairs",
                        "candidates"):
                agg[key] = agg.get(key, 0) + st[key]
        c.profile_read()
        c.profile(True)
        restore()
        torch.cuda.synchronize()
        c.event_step(store, 2000)
        kern = {k: v[0] for k, v in c.profile_read().items() if v[1]}
        c.profile(False)
        value = agg["substeps"] / (total_ms / 1e3)
        return {"substeps_per_s": value, "ms_per_step": total_ms / args.steps,
                "speedup_vs_rejection": value / plain_value,
                "emissions_from_sampler": agg["sampler_events"] / max(agg["emissions"], 1),
                "pairs_from_sampler": agg["sampler_pairs"] / max(agg["pairs"], 1),
                "per_step": {k: v / args.steps for k, v in agg.items()},
                "kernels_ms_one_step": kern}

    per_sub_step = timed(ctx)
    ectx = qed.Context(seed=SEED_CLUMPED, process_mask=3, cascade=True, sampler="event",
                       sampler_max_err=1e-3)
    ectx.sampler_load(params)
    ectx.sampler_evaluate()
    event_emission_only = timed(ectx)
    ectx.sampler_process(qed.PROC_PAIR)
    ectx.sampler_load(pparams)
    ectx.sampler_evaluate()
    ectx.sampler_process(qed.PROC_EMISSION)
    event = timed(ectx)
    uniform = run_sampler_uniform(params, dev)
    lo = int((np.log10(0.3) + 2) * 16)
    return {"train_samples": 1 << 26, "train_s": train_s, "final_mse": loss,
            "bins_usable": int(usable.sum()), "bins": int(len(err)),
            "max_cdf_err_usable": float(err[usable].max()) if usable.any() else None,
            "max_cdf_err_all": float(err.max()), "median_cdf_err": float(np.median(err)),
            "pair": {"train_s": ptrain_s, "final_mse": ploss,
                     "bins_usable": int((perr <= 1e-3).sum()),
                     "max_cdf_err_chi_ge_0.3": float(perr[lo:].max())},
            "speedup_vs_rejection": event["speedup_vs_rejection"],
            "substeps_per_s": event["substeps_per_s"], "ms_per_step": event["ms_per_step"],
            "per_sub_step": per_sub_step,
            "event_driven": event,
            "event_driven_emission_only": event_emission_only,
            "uniform_field_1e6": uniform,
            "note": "event-driven: about 1e9 per-sub-step draws become ~6e6 waiting-time "
                    "draws, but each generation of the cascade ends with its longest chain "
                    "of events (up to ~100 per particle), one network evaluation per event "
                    "on the critical path (a 16-row tensor-core tile, ~4 us on a nearly "
                    "idle warp)"}


def run_sampler_uniform(params, dev, n=1_000_000, steps=10):
    """The event-driven sampler against rejection where the generator is
    throughput-bound: the uniform-field electrons (the plain generator's
    recipe) at 1e6 rows, emission only, one step, no cascade."""
    import torch
    from paper_2008_10468_gb300 import inputs as I
    from paper_2008_10468_gb300 import qed
    arr = I.uniform_field_electrons(n, SEED_UNIFORM)
    pristine = qed.ParticleStore.from_numpy(arr, capacity=n, device=dev)
    store = qed.ParticleStore(40 * n, device=dev)

    def restore():
        for k in qed.FLOAT_FIELDS + ("id", "type"):
            getattr(store, k)[:n].copy_(getattr(pristine, k)[:n])
        store.type[n:].fill_(qed.REMOVED)
        store.count.fill_(n)

    out = {"workload": "uniform-field electrons, 1e6 rows (the plain generator's recipe), "
                       "emission only, one step"}
    stream = torch.cuda.current_stream()
    for mode, name in ((False, "rejection"), ("event", "event_driven")):
        ctx = qed.Context(seed=SEED_UNIFORM, process_mask=1, cascade=False, sampler=mode,
                          sampler_max_err=1e-3)
        if mode:
            ctx.sampler_load(params)
            ctx.sampler_evaluate()
        for w in range(3):
            restore()
            ctx.event_step(store, 100 + w)
        ms, subs, em, se = 0.0, 0, 0, 0
        for k in range(steps):
            restore()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = ctx.event_step(store, 200 + k)
            e1.record(stream)
            torch.cuda.synchronize()
            if st["status"] != 0:
                raise SystemExit("uniform-field sampler step failed with status %d" % st["status"])
            ms += e0.elapsed_time(e1)
            subs += st["substeps"]
            em += st["emissions"]
            se += st["sampler_events"]
        out[name] = {"ms_per_step": ms / steps, "substeps_per_s": subs / (ms / 1e3),
                     "emissions_per_step": em / steps,
                     "emissions_from_sampler": se / max(em, 1)}
    out["speedup_vs_rejection"] = (out["rejection"]["ms_per_step"]
                                   / out["event_driven"]["ms_per_step"])
    return out


def run_e2e(ctx, arr, cap, dev, args, pg=None):
    """Same metric through the API with host buffers: qed_event_step_host on a
    page-locked host store, which copies the population to the device, steps
    it and copies back what the step changed (momenta and types of the
    original rows, every field of the appended children), so that the host
    holds the whole updated store.  Timed with CUDA events around the call;
    the host store is restored between steps outside the timed region."""
    import torch
    from paper_2008_10468_gb300 import qed
    n = len(arr["px"])
    h = qed.HostStore.from_numpy(arr, capacity=cap)
    keep = {k: getattr(h, k)[:n].clone() for k in ("px", "py", "pz", "type")}
    stream = torch.cuda.current_stream()
    steps = max(2, min(args.steps, 5))
    total = 0.0
    subs = 0
    h2d = d2h = 0
    parts = []
    for k in range(steps + 2):
        for key, v in keep.items():
            getattr(h, key)[:n].copy_(v)
        h.count = n
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st = ctx.event_step_host(h, 3000 + k)
        e1.record(stream)
        torch.cuda.synchronize()
        if st["status"] != 0:
            raise SystemExit("host-store step failed with status %d" % st["status"])
        if k < 2:
            continue  # the first calls allocate the device copy and warm the host link
        m = st["count"]
        total += e0.elapsed_time(e1)
        subs += st["substeps"]
        h2d += 49 * n
        d2h += 13 * m + 36 * (m - n)
    # the whole job: every rank's sub-steps and bytes over the slowest rank's time
    value, t_max = job_rate(pg, subs, total, dev)
    h2d = allreduce_sum(pg, h2d, dev)
    d2h = allreduce_sum(pg, d2h, dev)
    return {"value": value, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d) // steps, "d2h_bytes_per_step": int(d2h) // steps,
            "ms_per_step": t_max / steps, "api": "qed_event_step_host (page-locked host store)"}


# --------------------------------------------------------------------------
# reference arm: the FP64 oracle, as it stands, on the host cores
# --------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2008_10468_gb300 import inputs as I
    arr = I.clumped_mixed(N_PARTICLES, SEED_CLUMPED)
    cores = os.cpu_count() or 1
    cf = O.make_config(SEED_CLUMPED, process_mask=3, cascade=1, threads=cores)
    m = int(os.environ.get("QED_REFERENCE_SAMPLE", "65536"))
    sub = population_sample(arr, m, 11)
    for w in range(args.warmup):
        O.event_step_mt(cf, sub, 1000 + w, capacity=m * 64)
    t = 0.0
    subs = 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        _, st = O.event_step_mt(cf, sub, 2000 + k, capacity=m * 64)
        t += time.perf_counter() - t0
        subs += st["substeps"]
    value = subs / t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles": N_PARTICLES},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d rows of the population (1%% hot, stratified) per step" % m},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sampler", action="store_true")
    ap.add_argument("--no-cascade", action="store_true")
    ap.add_argument("--no-push", action="store_true")
    ap.add_argument("--cascade-steps", type=int, default=100)
    ap.add_argument("--tail-rows", type=int, default=None,
                    help="generations below this many rows go to the tail pass (0: off; "
                         "default: the library's)")
    ap.add_argument("--particles", type=int, default=N_PARTICLES,
                    help="population size (smaller values only for profiling runs)")
    ap.add_argument("--sweep-n", type=int, default=SWEEP_N,
                    help="synchrotron sweep length (smaller values only for profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
