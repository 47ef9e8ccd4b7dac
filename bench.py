#!/usr/bin/env python
"""Throughput of the fully adaptive MR-LBM time step on GB300.

Workload: the D2Q4^4 compressible-Euler four-quadrant Riemann problem on
[0, 1]^2 (gamma = 1.4, lambda = 5, s^q = 1.9/1.75, s^xy = 1, copy
boundaries), min level 2, max level 10 (1024^2 finest cells), epsilon = 1e-3,
mu_bar = 0, seeded quadrant states.  One step = one pass of Algorithm 1's
loop (encode, T/H/G adaptation, compaction, data transfer, ghost
prediction, transport, collision) through the C-ABI.  Metric: leaf updates
per second (sum over timed steps of the leaves of the new mesh, divided by
the event-timed duration of those steps).

The headline is the chosen form of this workload, FP32 arithmetic with FP16
storage (FP64 mesh decisions); the plain FP64 form is timed beside it
("forms"), and "batched" times many independent instances (D2Q9 vortices
and D2Q4^4 Riemann problems) stepped by shared launches against the same
instances stepped one at a time in the plain form.

The timed window starts at step 200 of the run from the initial condition
(``--start-step``, untimed), where the Riemann problem's leaf count has
grown; the warm-up follows, then the K timed steps.  Every form (FP64, FP32,
FP16 and BF16 storage) is timed on the same window, and its relative L1
distance to the FP64 run at the end of the window is reported against its
bound.

Also on the line: the exact collision, the prediction of half-width s = 2
and 3 ("prediction_s") and the 3D ball (D3Q6) legs; the
other configurations ("configs": D1Q2 advection at J = 9 in microseconds
per step, D1Q2 Burgers and D1Q3 dam break at J = 12 per form with their L1
distance at T = 0.4, the D2Q9 obstacle flow at J = 10 and the time of its
adjoint per forward step); the roofline of the transport + collision kernel
(algorithmic bytes or flops over its live launch time, and the DRAM bytes of
an ncu capture of it scaled to the timed launches); the CPU oracle on one
core and on every host core (one process per core); and the end-to-end rate
through the C-ABI with host buffers.

Runs on N GPUs as N independent replicas (the single-instance step does not
shard).  ``--impl reference`` times the CPU oracle on a bounded sample of
the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "adaptive leaf updates/s per MR-LBM step"
UNIT = "leaf updates/s"
WORKLOAD = "d2q4x4_euler_riemann_J10"

# Algorithmic work of the transport + collision kernel per leaf (FP64 form,
# D2Q4^4): reads and writes the 16 populations of the leaf and reads its key
# and level (2 * 16 * 8 + 4 + 1 bytes); 320 FP64 flops (16 populations x 11
# for the flattened row weights and update, 141 for the collision: moments,
# fluxes with one division, relaxation, back to populations).  Window values
# of neighbours are L2 reuse, not algorithmic.  The other forms store b bytes
# per value: 2 * 16 * b + 5 bytes.
ALG_BYTES_PER_LEAF = 2 * 16 * 8 + 5
ALG_FLOPS_PER_LEAF = 320.0
FORM_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
# DRAM bytes (read + write) of one launch of the transport + collision kernel
# per leaf, from ncu captures of this workload: FP16 storage, the first timed
# launch after the 200-step advance (about 105.2k leaves: 6.20 MB read, 1.8 kB
# written); FP64, the 7th launch from the initial condition (about 45.7k
# leaves: 8.97 MB read, nothing written).  `traffic` scales them by the
# leaves of the timed launches.  They hold for the kernel as captured and
# must be retaken when it changes.
CAPTURED_DRAM_BYTES_PER_LEAF = {"fp16": (6.201088e6 + 1.792e3) / 105187.0, "fp64": 8.9728e6 / 45729.25}
CAPTURED_DRAM_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one cold launch, per leaf, scaled "
                      "by the leaves of the timed launches")
FORM_DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f32 (f16 storage)", "bf16": "f32 (bf16 storage)"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--max-level", type=int, default=10)
    p.add_argument("--e2e-steps", type=int, default=30)
    p.add_argument("--exact-only", action="store_true",
                   help="run only the exact-collision leg (for profiler runs)")
    p.add_argument("--d3-only", action="store_true", help="run only the 3D leg (for profiler runs)")
    p.add_argument("--d3-steps", type=int, default=100,
                   help="steps timed on the 3D ball advection (D3Q6, 256^3 finest cells); 0 skips the leg")
    p.add_argument("--exact-steps", type=int, default=200,
                   help="steps timed with the original adaptive collision (FP64); 0 skips the leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--cpu-all-cores", type=int, default=1,
                   help="also time the oracle sample on every host core at once (1) or not (0)")
    p.add_argument("--profile-groups", action="store_true",
                   help="also time every kernel group once (extra steps, not part of value)")
    p.add_argument("--form", default="fp16", choices=["fp64", "fp32", "fp16", "bf16"],
                   help="storage / arithmetic form of the timed run")
    p.add_argument("--serving-n", type=int, default=256,
                   help="instances of the batched serving measurement (0: skip it)")
    p.add_argument("--serving-steps", type=int, default=30)
    p.add_argument("--autotune-steps", type=int, default=3,
                   help="steps per candidate of the batch autotuner before the batched timing; 0 skips it")
    p.add_argument("--serving-loop", type=int, default=1,
                   help="also step every instance alone in the plain form (one-at-a-time baseline)")
    p.add_argument("--minimal", action="store_true",
                   help="time the chosen form only and print a short line (for profiler runs)")
    p.add_argument("--batched-only", action="store_true",
                   help="run only the batched serving measurement (for profiler runs)")
    p.add_argument("--start-step", type=int, default=200,
                   help="untimed steps from the initial condition before the warm-up: the Euler workload's "
                        "throughput window starts at step 200, where its leaf count has grown")
    p.add_argument("--config-legs", type=int, default=1,
                   help="also measure the other configurations: D1Q2 advection J=9, D1Q2 Burgers and D1Q3 "
                        "dam break J=12 per form, D2Q9 obstacle J=10 with its adjoint (1) or not (0)")
    p.add_argument("--ns-steps", type=int, default=50, help="timed steps of the D2Q9 obstacle leg")
    p.add_argument("--adjoint-steps", type=int, default=4000,
                   help="forward steps of the timed adjoint run (D2Q9 obstacle, J=10); 0 skips it")
    p.add_argument("--adjoint-every", type=int, default=100, help="checkpoint interval of the adjoint run")
    p.add_argument("--legs-only", action="store_true", help="run only the configuration legs")
    p.add_argument("--pred-s", type=int, default=1,
                   help="half-width of the prediction for the --minimal run (for profiler runs)")
    p.add_argument("--wide-leg", type=int, default=1,
                   help="also time the headline workload with the prediction of half-width s = 2 and 3 (1) or not")
    return p.parse_args()


def _line_config(cfg, args):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": WORKLOAD, "scheme": "D2Q4^4 Euler", "max_level": cfg["max_level"],
            "min_level": cfg["min_level"], "eps": cfg["eps"], "mu_bar": cfg["mu_bar"], "seed": args.seed,
            "finest_cells": (cfg["roots"][0] << cfg["max_level"]) * (cfg["roots"][1] << cfg["max_level"]),
            "l2": "GPU arm: 256 MiB write between timed steps, outside the step events",
            "parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "single"}


def _workload(args):
    from paper_2103_02903_gb300 import workloads
    return workloads.euler_2d(seed=args.seed, max_level=args.max_level)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        exe = shutil.which("nvidia-smi")
        if exe:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen([exe, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _l2_copy_gbs(torch):
    """Copy bandwidth of buffers that stay in L2 (2 x 32 MiB of the 129 MB
    L2): read + write bytes of 20 back-to-back copies replayed from a CUDA
    graph (no host launch gaps), over their event time, best of 5: the
    ceiling of a kernel whose data live in L2."""
    n = 32 << 20
    a = torch.zeros(n, dtype=torch.uint8, device="cuda")
    b = torch.zeros(n, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.copy_(a)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(20):
                b.copy_(a)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3 / 20)
    del g, a, b
    return 2.0 * n / best / 1e9


def _fp64_peak_tflops(torch):
    """FP64 throughput measured with a cuBLAS DGEMM (2 N^3 flops), best of 3."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


# --------------------------------------------------------------------------- CPU oracle
def _oracle_sample(cfg, u, seconds, max_steps=None):
    """Time oracle steps of the workload from its initial condition until
    `seconds` of CPU time have elapsed (single thread)."""
    from oracle import Oracle
    o = Oracle(cfg)
    o.init(u)
    leaves, steps, t = 0, 0, 0.0
    while t < seconds and (max_steps is None or steps < max_steps):
        t0 = time.perf_counter()
        o.step(1)
        t += time.perf_counter() - t0
        leaves += o.num_leaves()
        steps += 1
    return leaves, steps, t


def _oracle_replica(job):
    cfg, u, seconds = job
    return _oracle_sample(cfg, u, seconds)


def _oracle_sample_all_cores(cfg, u, seconds, nproc):
    """The same sample on every host core: one process per core (spawned, so
    none inherits the GPU context), each stepping its own copy of the workload
    from its initial condition.  Returns the summed leaf updates, the time of
    the slowest process and the steps of each."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(_oracle_replica, [(cfg, u, seconds)] * nproc)
    return sum(r[0] for r in res), max(r[2] for r in res), [r[1] for r in res]


def run_reference(args):
    """The oracle (FP64, single thread) on the same workload: W untimed steps
    from the initial condition, then K timed ones, each phase capped in CPU
    time so that the run ends within a few minutes (the oracle's dense step
    costs about two seconds at J = 10)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    cfg, u = _workload(args)
    from oracle import Oracle
    o = Oracle(cfg)
    o.init(u)
    warm_budget, budget = 60.0, 150.0
    warm, tw = 0, 0.0
    while warm < args.warmup and tw < warm_budget:
        t0 = time.perf_counter()
        o.step(1)
        tw += time.perf_counter() - t0
        warm += 1
    leaves, steps, t = 0, 0, 0.0
    while steps < args.steps and t < budget:
        t0 = time.perf_counter()
        o.step(1)
        t += time.perf_counter() - t0
        leaves += o.num_leaves()
        steps += 1
    value = leaves / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * t / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _line_config(cfg, args),
        "window": "oracle steps %d..%d from the initial condition (warm-up capped at %.0f s, timed steps at "
                  "%.0f s of CPU time); the GPU arm times steps S+W+1..S+W+K after an untimed advance of S "
                  "steps, which the oracle cannot reach in minutes" % (warm + 1, warm + steps, warm_budget, budget),
        "leaves_per_step_avg": leaves / steps,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "oracle (one thread) steps %d..%d of the workload from its initial condition"
                                   % (warm + 1, warm + steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU
def run_serving(args, stream, flush, local):
    """Batched serving form: many independent instances (D2Q9 vortex flows and
    D2Q4^4 Riemann problems, uneven levels and thresholds) stepped by shared
    launches in FP32 with FP16 storage; against the same instances stepped one
    at a time in the plain FP64 form."""
    import numpy as np
    import torch
    from paper_2103_02903_gb300 import workloads
    from paper_2103_02903_gb300.binding import Batch, Solver

    cases = workloads.serving_batch(seed=args.seed, n=args.serving_n, precision="fp16")
    t0 = time.perf_counter()
    b = Batch([c for c, _ in cases], stream=stream.cuda_stream)
    for s, (c, u) in zip(b.instances, cases):
        s.init(u)
    b.step(args.warmup)
    b.synchronize()
    setup_s = time.perf_counter() - t0
    tune = None
    if args.autotune_steps > 0:
        # schedules picked by the library's autotuner from the warmed-up state
        # (the batch is put back as it was); the timed steps below use them
        t1 = time.perf_counter()
        default = b.schedule()
        ms_fixed, ms_tuned = b.autotune(args.autotune_steps)
        tune = {"trial_steps": args.autotune_steps, "ms_per_step_default_schedule": ms_fixed,
                "ms_per_step_tuned_schedule": ms_tuned, "gain": ms_fixed / ms_tuned,
                "default_schedule": default[0], "chosen_schedule_per_part": b.schedule(),
                "phases": ["projection", "details", "mesh flags and grading", "compaction", "data transfer",
                           "prediction", "transport + collision"],
                "unit": "blocks per SM of each phase's grid", "tuning_s": time.perf_counter() - t1}
    K = args.serving_steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    per0 = [s.counters()[0] for s in b.instances]
    l0 = b.launch_count()
    b.profile_enable(1)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    for k in range(K):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        b.step(1)
        ev[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    kms, kn = b.profile_read()
    b.profile_enable(0)
    launches = b.launch_count() - l0
    per1 = [s.counters()[0] for s in b.instances]
    step_ms = np.array([a.elapsed_time(c) for a, c in ev])
    upd = [y - x for x, y in zip(per0, per1)]
    total = float(sum(upd))
    # algorithmic bytes of the transport + collision kernels: read and write
    # every leaf's populations (2 bytes each) plus its index entry and level
    alg_bytes = sum(u_ * (2 * 2 * (9 if c["scheme"] == "d2q9_ns" else 16) + 5) for u_, (c, _) in zip(upd, cases))
    peaks, peak_kind = _peaks()
    ksec = kms / 1e3
    gbs = alg_bytes / ksec / 1e9 if ksec > 0 else None
    out = {
        "workload": "%d instances: D2Q9 periodic vortices and D2Q4^4 Riemann quadrants, J in {6..10}, "
                    "eps in {1e-3, 1e-4}, FP32 arithmetic with FP16 storage" % len(cases),
        "value": total / (step_ms.sum() / 1e3), "unit": UNIT, "steps": K,
        "ms_per_step": float(step_ms.mean()), "latency_ms_p50": float(np.percentile(step_ms, 50)),
        "latency_ms_p99": float(np.percentile(step_ms, 99)),
        "leaves_per_step_avg": total / K, "gpu_launches": launches, "autotune": tune,
        "launches_per_step": launches / K, "setup_s": setup_s,
        "roofline": {"kernel": "k_stream_collide (transport + collision), both schemes", "bound": "hbm",
                     "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": (gbs / peaks["hbm_gbs"]) if gbs else None, "peak_kind": peak_kind,
                     "traffic": None, "kernel_ms_per_step": kms / max(K, 1),
                     "note": "kernel time summed over the scheme branches (concurrent), so frac is a lower bound"},
    }
    b.close()
    if args.serving_loop:
        # one instance at a time, plain FP64, each with its own CUDA graph
        lat, leaves = [], 0.0
        for c, u in cases:
            c = dict(c, precision="fp64")
            s = Solver(c, stream=stream.cuda_stream)
            s.init(u)
            s.step(args.warmup)
            s.synchronize()
            a0 = s.counters()[0]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n_it = 5
            e0.record(stream)
            s.step(n_it)
            e1.record(stream)
            torch.cuda.synchronize()
            lat.append(e0.elapsed_time(e1) / n_it)
            leaves += (s.counters()[0] - a0) / n_it
            s.close()
        lat = np.array(lat)
        out["one_at_a_time_plain"] = {
            "value": leaves / (lat.sum() / 1e3), "unit": UNIT, "ms_per_round": float(lat.sum()),
            "instance_step_ms_p50": float(np.percentile(lat, 50)),
            "instance_step_ms_p99": float(np.percentile(lat, 99)),
            "note": "each instance stepped alone in FP64 (own CUDA graph), 5 steps after the warm-up; a round "
                    "steps every instance once"}
        out["speedup_vs_one_at_a_time_plain"] = out["value"] / out["one_at_a_time_plain"]["value"]
    return out


def _l1(a, b):
    """Largest relative L1 distance over the conserved moments (rows of a, b)."""
    import numpy as np
    return float((np.abs(a - b).sum(axis=1) / np.abs(b).sum(axis=1)).max())


def _time_steps(s, n, stream, flush):
    """n steps of solver s, each bracketed by CUDA events on `stream`, with
    the L2 flush between them outside the events.  Returns (per-step ms,
    leaf updates)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    c0, _ = s.counters()
    for k in range(n):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        s.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    c1, _ = s.counters()
    return [a.elapsed_time(b) for a, b in ev], c1 - c0


def run_config_legs(args, stream, flush):
    """The other measured configurations: D1Q2 advection at J = 9 (latency,
    us per step), D1Q2 Burgers and D1Q3 dam break at J = 12 per precision
    form with the L1 distance of each form to the FP64 path at T = 0.4, the
    D2Q9 obstacle flow at J = 10 (leaf updates/s) and its adjoint (time per
    forward step)."""
    import numpy as np
    import torch
    from paper_2103_02903_gb300 import workloads as wl
    from paper_2103_02903_gb300.binding import MrError, Solver

    out = {}

    def fresh(cfg, u, warm):
        # a solver whose step graphs are captured (warm-up), then reset to the initial condition
        s = Solver(cfg, stream=stream.cuda_stream)
        s.init(u)
        s.step(warm)
        s.init(u)
        s.synchronize()
        return s

    # config 1: D1Q2 advection, J = 9, the whole run to T = 0.4
    cfg, u = wl.advection_1d(seed=args.seed, max_level=9)
    n = wl.steps_to(cfg, 0.4)
    s = fresh(cfg, u, max(args.warmup, 4))
    ms, upd = _time_steps(s, n, stream, flush)
    out["d1q2_advection_J9"] = {
        "workload": "D1Q2 advection, [-3, 3] periodic, 512 finest cells, eps 1e-4, T = 0.4 (%d steps), FP64" % n,
        "us_per_step": 1e3 * float(np.mean(ms)), "us_per_step_p50": 1e3 * float(np.median(ms)),
        "leaves_per_step_avg": upd / n, "value": upd / (sum(ms) / 1e3), "unit": UNIT}
    s.close()

    # config 2: D1Q2 Burgers and D1Q3 dam break, J = 12, T = 0.4, every form
    for name in ("burgers_1d", "shallow_water_1d"):
        cfg, u = wl.WORKLOADS[name](seed=args.seed, max_level=12)
        n = wl.steps_to(cfg, 0.4)
        leg = {"workload": "%s, [-1, 1] copy faces, 4096 finest cells, eps 1e-4, T = 0.4 (%d steps)"
                           % ("D1Q2 Burgers" if name == "burgers_1d" else "D1Q3 dam break", n), "forms": {}}
        ref = None
        for fm in ("fp64", "fp32", "fp16", "bf16"):
            s = fresh(dict(cfg, precision=fm), u, max(args.warmup, 4))
            ms, upd = _time_steps(s, n, stream, flush)
            p = s.project(12)
            if fm == "fp64":
                ref = p
            e = _l1(p, ref)
            bound = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-3}[fm]
            leg["forms"][fm] = {"us_per_step": 1e3 * float(np.mean(ms)), "leaves_per_step_avg": upd / n,
                                "value": upd / (sum(ms) / 1e3), "l1_vs_fp64_path_at_T": e,
                                "l1_bound": bound, "meets_bound": e <= bound}
            s.close()
        leg["l1_note"] = ("relative L1 distance of the conserved moments on level 12 to the FP64 path at T; the "
                          "FP64 path matches the oracle to 1e-12, and the GPU tests check the FP32 / FP16 forms "
                          "of this configuration against the oracle itself (<= 1e-5 / 1e-3)")
        out[name + "_J12"] = leg

    # config 4: D2Q9 flow past the obstacle, J = 10, and its adjoint
    cfg, u = wl.ns_obstacle_2d(seed=args.seed, max_level=10)
    leg = {"workload": "D2Q9 obstacle flow, [0, 2] x [0, 1], 2048 x 1024 finest cells, Re 1200, eps 1e-4, "
                       "mu_bar 1; steps %d..%d timed after an untimed advance"
                       % (args.start_step + args.warmup + 1, args.start_step + args.warmup + args.ns_steps),
           "forms": {}}
    proj = {}
    for fm in ("fp64", "fp16"):
        s = Solver(dict(cfg, precision=fm), stream=stream.cuda_stream)
        s.init(u)
        s.step(args.start_step + args.warmup)
        s.synchronize()
        ms, upd = _time_steps(s, args.ns_steps, stream, flush)
        proj[fm] = s.project(10)
        leg["forms"][fm] = {"value": upd / (sum(ms) / 1e3), "unit": UNIT, "ms_per_step": float(np.mean(ms)),
                            "leaves_per_step_avg": upd / args.ns_steps}
        s.close()
    e = _l1(proj["fp16"], proj["fp64"])
    leg["forms"]["fp16"].update({"l1_vs_fp64_path": e, "l1_bound": 1e-3, "meets_bound": e <= 1e-3})
    if args.adjoint_steps > 0:
        try:
            s = fresh(cfg, u, max(args.warmup, 4))
            ms, upd = _time_steps(s, args.adjoint_steps, stream, flush)
            s.close()
            s = Solver(cfg, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            J, grad, gs = s.adjoint(u, args.adjoint_steps, checkpoint_every=args.adjoint_every)
            torch.cuda.synchronize()
            t_adj = time.perf_counter() - t0
            s.close()
            fwd = float(np.mean(ms))
            leg["adjoint"] = {
                "forward_steps": args.adjoint_steps, "checkpoint_every": args.adjoint_every,
                "functional": "time-integrated kinetic energy, sum over steps and leaves of |C| |q|^2 / (2 rho)",
                "ms_per_forward_step": 1e3 * t_adj / args.adjoint_steps,
                "forward_only_ms_per_step": fwd, "ratio_to_forward": 1e3 * t_adj / args.adjoint_steps / fwd,
                "J": J, "grad_s_shear": float(gs[1]), "finite": bool(np.isfinite(grad).all()),
                "note": "wall time of mr_lbm_adjoint (forward pass with checkpoints, replay of each segment, "
                        "backward sweep, gradients w.r.t. the initial field and the relaxation rates), FP64"}
        except MrError as e:
            leg["adjoint"] = {"error": str(e)}
    out["ns_obstacle_J10"] = leg
    return out


def run_ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2103_02903_gb300.binding import Solver

    cfg, u = _workload(args)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed_run(form, clocks_too=False, extra=None, steps=None):
        """S untimed steps from the initial condition (the start of the
        throughput window), W untimed warm-up steps, then K steps timed one
        by one with CUDA events (L2 flushed between them, outside the events)."""
        steps = steps or args.steps
        s = Solver(dict(cfg, precision=form, **(extra or {})), stream=stream.cuda_stream)
        s.init(u)
        s.step(args.start_step + args.warmup)
        s.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        upd0, _ = s.counters()
        l0 = s.launch_count()
        s.profile_enable(1)  # events around the transport + collision kernel
        clk = ClockSampler(local) if clocks_too else None
        barrier()
        tw = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            s.step(1)
            ev[k][1].record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        tw = time.perf_counter() - tw
        clocks = clk.stop() if clk else None
        kms, kn = s.profile_read()
        s.profile_enable(0)
        upd1, _ = s.counters()
        tot = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        return s, dict(updates=upd1 - upd0, total_s=tot, wall_s=tw, launches=s.launch_count() - l0,
                       kern_ms=kms, kern_n=kn, clocks=clocks)

    def exact_leg(fp64_ms=None):
        """The original adaptive collision (Sec. 5.3) on the same workload, FP64."""
        s3, r3 = timed_run("fp64", extra={"exact_collision": 1}, steps=args.exact_steps)
        nJ = (cfg["roots"][0] << cfg["max_level"]) * (cfg["roots"][1] << cfg["max_level"])
        ms3 = 1e3 * r3["total_s"] / args.exact_steps
        out = {"value": r3["updates"] / r3["total_s"], "unit": UNIT, "ms_per_step": ms3,
               "steps": args.exact_steps, "leaves_per_step_avg": r3["updates"] / args.exact_steps,
               "launches_per_step": r3["launches"] / args.exact_steps,
               "finest_cells_collided_per_step": nJ, "finest_cells_per_s": nJ / (ms3 / 1e3),
               "dtype": "f64",
               "note": "collision on the dense reconstruction of the post-transport data at level J, "
                       "then averaged onto the leaves (Eq. sourceoferror); timed like the other forms"}
        if fp64_ms is not None:
            out["ms_per_step_over_leaf_collision_fp64"] = ms3 - fp64_ms
        s3.close()
        return out

    def wide_leg():
        """The same workload and window with the prediction of half-width s = 2
        and 3 (Table 1): wider stencils, grading and transport windows."""
        out = {"workload": WORKLOAD + " with pred_s = 2, 3", "unit": UNIT, "steps": args.steps}
        for sw in (2, 3):
            for fm in ("fp64", "fp16"):
                s5, r5 = timed_run(fm, extra={"pred_s": sw})
                out["s%d_%s" % (sw, fm)] = {"value": r5["updates"] / r5["total_s"],
                                            "ms_per_step": 1e3 * r5["total_s"] / args.steps,
                                            "leaves_per_step_avg": r5["updates"] / args.steps,
                                            "launches_per_step": r5["launches"] / args.steps}
                s5.close()
        return out

    def d3_leg():
        """The 3D test of Sec. 7.3: D3Q6 advection of a ball, J = 8 (256^3), eps = 1e-3, mu_bar = 2."""
        from paper_2103_02903_gb300 import workloads
        cfg3, u3 = workloads.advection_3d(seed=args.seed, max_level=8)
        out = {"workload": "d3q6_ball_advection_J8", "finest_cells": 256 ** 3, "eps": cfg3["eps"],
               "mu_bar": cfg3["mu_bar"], "steps": args.d3_steps, "unit": UNIT}
        for fm in ("fp16", "fp64"):
            s3 = Solver(dict(cfg3, precision=fm), stream=stream.cuda_stream)
            s3.init(u3)
            s3.step(args.warmup)
            s3.synchronize()
            e3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.d3_steps)]
            c0, _ = s3.counters()
            torch.cuda.nvtx.range_push("timed")
            for k in range(args.d3_steps):
                flush.fill_(k & 0xFF)
                e3[k][0].record(stream)
                s3.step(1)
                e3[k][1].record(stream)
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            c1, _ = s3.counters()
            ms3 = sum(a.elapsed_time(b) for a, b in e3) / args.d3_steps
            _, mesh_or3, _ = s3.stats()
            out[fm] = {"value": (c1 - c0) / (ms3 * args.d3_steps / 1e3), "ms_per_step": ms3,
                       "leaves_per_step_avg": (c1 - c0) / args.d3_steps, "occupancy_final": mesh_or3}
            s3.close()
        return out

    if args.exact_only:
        print(json.dumps({"exact_collision": exact_leg()}), flush=True)
        return 0
    if args.d3_only:
        print(json.dumps({"d3q6_3d": d3_leg()}), flush=True)
        return 0
    if args.batched_only:
        out = run_serving(args, stream, flush, local)
        print(json.dumps({"batched": out}), flush=True)
        return 0
    if args.legs_only:
        print(json.dumps({"configs": run_config_legs(args, stream, flush)}), flush=True)
        return 0
    solver, r = timed_run(args.form, clocks_too=not args.minimal,
                          extra={"pred_s": args.pred_s} if args.minimal and args.pred_s != 1 else None)
    if args.minimal:
        print(json.dumps({"form": args.form, "value": r["updates"] / r["total_s"],
                          "ms_per_step": 1e3 * r["total_s"] / args.steps,
                          "leaves_per_step_avg": r["updates"] / args.steps,
                          "transport_kernel_ms": r["kern_ms"] / max(r["kern_n"], 1)}), flush=True)
        solver.close()
        return 0
    clocks, launches, kern_ms, kern_n = r["clocks"], r["launches"], r["kern_ms"], r["kern_n"]
    total_s, t_wall, leaf_updates = r["total_s"], r["wall_s"], r["updates"]
    J = cfg["max_level"]
    proj = {args.form: solver.project(J)}  # state at the end of the timed window
    # every form timed on the same window; the plain FP64 form is the reference of the L1 distances
    forms = {}
    fp64_tflops = None
    for fm in ("fp64", "fp32", "fp16", "bf16"):
        if fm == args.form:
            r2 = r
        else:
            s2, r2 = timed_run(fm)
            proj[fm] = s2.project(J)
            s2.close()
        lv = r2["updates"] / args.steps
        ksec = r2["kern_ms"] / 1e3 / max(r2["kern_n"], 1)
        bpl = 2 * 16 * FORM_BYTES[fm] + 5
        forms[fm] = {"value": r2["updates"] / r2["total_s"], "ms_per_step": 1e3 * r2["total_s"] / args.steps,
                     "leaves_per_step_avg": lv, "dtype": FORM_DTYPE[fm], "transport_kernel_ms": 1e3 * ksec,
                     "transport_hbm_gbs_alg": bpl * lv / ksec / 1e9}
        if fm == "fp64":
            fp64_tflops = _fp64_peak_tflops(torch)
            ach = ALG_FLOPS_PER_LEAF * lv / ksec / 1e12
            forms[fm]["transport_roofline"] = {
                "bound": "alu", "achieved": ach, "peak": fp64_tflops, "unit": "TFLOP/s", "frac": ach / fp64_tflops,
                "peak_kind": "FP64 measured with cuBLAS DGEMM in this run"}

    bounds = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-3}
    for fm in forms:
        e = _l1(proj[fm], proj["fp64"])
        forms[fm]["l1_vs_fp64_path"] = e
        forms[fm]["l1_bound"] = bounds[fm]
        forms[fm]["meets_bound"] = e <= bounds[fm]

    exact = exact_leg(forms["fp64"]["ms_per_step"]) if args.exact_steps > 0 else None
    legs = run_config_legs(args, stream, flush) if args.config_legs else None
    d3 = d3_leg() if args.d3_steps > 0 else None
    wide = wide_leg() if args.wide_leg else None

    serving = run_serving(args, stream, flush, local) if args.serving_n > 0 else None

    # whole-job aggregate: updates summed over ranks, time = max over ranks
    from paper_2103_02903_gb300.replicas import aggregate
    leaf_updates_all, total_s_max = aggregate(leaf_updates, total_s, device="cuda")
    value = leaf_updates_all / total_s_max
    per_step_leaves = leaf_updates / args.steps

    # roofline of the transport + collision kernel, timed live above
    peaks, peak_kind = _peaks()
    kern_avg_s = kern_ms / 1e3 / max(kern_n, 1)
    bytes_per_leaf = 2 * 16 * FORM_BYTES[args.form] + 5
    achieved_gbs = bytes_per_leaf * per_step_leaves / kern_avg_s / 1e9
    hbm = {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": achieved_gbs / peaks["hbm_gbs"], "peak_kind": peak_kind}
    if args.form == "fp64":
        achieved_tflops = ALG_FLOPS_PER_LEAF * per_step_leaves / kern_avg_s / 1e12
        roofline = {
            "kernel": "k_stream_collide<3> (transport + collision)",
            "bound": "alu", "achieved": achieved_tflops, "peak": fp64_tflops, "unit": "TFLOP/s",
            "frac": achieved_tflops / fp64_tflops,
            "peak_kind": "FP64 measured with cuBLAS DGEMM in this run",
            "traffic": None, "hbm": hbm,
        }
    else:
        roofline = dict(hbm, kernel="k_stream_collide<3> (transport + collision)", bound="hbm", traffic=None)
    if args.form in CAPTURED_DRAM_BYTES_PER_LEAF:
        roofline["traffic"] = CAPTURED_DRAM_BYTES_PER_LEAF[args.form] * per_step_leaves
        roofline["traffic_unit"] = "B per launch"
        roofline["traffic_kind"] = CAPTURED_DRAM_NOTE
        # the same bytes over the live launch time, against the measured HBM peak
        roofline["traffic_gbs"] = roofline["traffic"] / kern_avg_s / 1e9
        roofline["traffic_frac_of_hbm"] = roofline["traffic_gbs"] / peaks["hbm_gbs"]
    # the state of this single instance stays in L2: the same bytes against the L2 copy bandwidth
    l2_gbs = _l2_copy_gbs(torch)
    roofline["l2"] = {"achieved": achieved_gbs, "peak": l2_gbs, "unit": "GB/s", "frac": achieved_gbs / l2_gbs,
                      "peak_kind": "graph-replayed copies of a 32 MiB buffer (L2-resident) measured in this run"}
    roofline.update({"kernel_ms_avg": 1e3 * kern_avg_s, "kernel_share_of_step": kern_ms / 1e3 / total_s,
                     "alg_flops_per_leaf": ALG_FLOPS_PER_LEAF, "alg_bytes_per_leaf": bytes_per_leaf})

    groups = None
    if args.profile_groups:
        groups = {}
        names = {1: "transport+collision", 2: "details", 3: "projection", 4: "prediction",
                 5: "mesh adaptation+compaction", 6: "data transfer"}
        for gid, name in names.items():
            solver.profile_enable(gid)
            solver.step(20)
            ms, n = solver.profile_read()
            groups[name] = {"ms_per_step": ms / 20.0, "launches_per_step": n / 20.0}
        solver.profile_enable(0)

    # end to end through the C-ABI with host buffers: upload the state,
    # one step, download the state
    e2e = None
    if args.e2e_steps > 0:
        n = solver.num_leaves()
        cap = int(n * 1.5) + 1024
        keys = torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        levs = torch.empty(cap, dtype=torch.int8, pin_memory=True).numpy()
        f = torch.empty(16 * cap, dtype=torch.float64, pin_memory=True).numpy()
        nn = solver.get_leaves_into(keys[:cap], levs[:cap], f[:16 * cap])
        h2d = d2h = 0
        e2e_leaves = 0
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fk = f[:16 * nn]
            solver.set_leaves(keys[:nn], levs[:nn], fk.reshape(16, nn))
            h2d += nn * (8 + 1 + 16 * 8)
            solver.step(1)
            nn = solver.get_leaves_into(keys[:cap], levs[:cap], f[:16 * cap])
            d2h += nn * (8 + 1 + 16 * 8)
            e2e_leaves += nn
        barrier()
        t_e2e = time.perf_counter() - t0
        e2e_all, t_e2e_max = aggregate(e2e_leaves, t_e2e, device="cuda")
        e2e = {"value": e2e_all / t_e2e_max, "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.e2e_steps, "d2h_bytes_per_step": d2h // args.e2e_steps,
               "steps": args.e2e_steps,
               "call": "mr_lbm_set_leaves(host) + mr_lbm_step(1) + mr_lbm_get_leaves(host), pinned buffers"}

    per_level, mesh_or, mem_or = solver.stats()
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        lv, st, t = _oracle_sample(cfg, u, args.cpu_seconds)
        from paper_2103_02903_gb300 import workloads as wl
        dense_cells = st * int(np.prod(wl.finest_shape(cfg)))
        cpu = {"value": lv / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "dense_cell_updates_per_s": dense_cells / t,
               "sample": "oracle (single thread) steps 1..%d of the same workload from its initial "
                         "condition, %.1f s" % (st, t)}
        if args.cpu_all_cores:
            nproc = os.cpu_count() or 1
            lv_all, t_all, st_all = _oracle_sample_all_cores(cfg, u, args.cpu_seconds, nproc)
            cpu_all = {"value": lv_all / t_all, "unit": UNIT, "cores": nproc, "kind": "oracle",
                       "sample": "%d oracle processes at once, one per host core (nproc %d), each stepping "
                                 "its own copy of the same workload from its initial condition for %.0f s "
                                 "(%d..%d steps); leaf updates summed over the processes / time of the "
                                 "slowest" % (nproc, nproc, args.cpu_seconds, min(st_all), max(st_all))}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": FORM_DTYPE[args.form],
            "data": "synthetic",
            "config": _line_config(cfg, args),
            "window": "steps %d..%d from the initial condition: %d untimed steps to the start of the throughput "
                      "window, %d warm-up, %d timed" % (args.start_step + args.warmup + 1,
                                                        args.start_step + args.warmup + args.steps,
                                                        args.start_step, args.warmup, args.steps),
            "leaves_per_step_avg": per_step_leaves, "mesh_or_final": mesh_or, "mem_or_final": mem_or,
            "wall_s_timed_region": t_wall,
            "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "clocks": clocks,
        }
        if groups is not None:
            line["kernel_groups"] = groups
        line["forms"] = forms
        line["chosen_form"] = args.form
        line["speedup_chosen_vs_plain_fp64"] = forms[args.form]["value"] / forms["fp64"]["value"] \
            if args.form in forms else value / forms["fp64"]["value"]
        line["accuracy_of_forms"] = {
            "measured": {fm: forms[fm]["l1_vs_fp64_path"] for fm in forms},
            "bound": {fm: bounds[fm] for fm in forms},
            "meets_bound": {fm: forms[fm]["meets_bound"] for fm in forms},
            "how": "largest relative L1 distance over the conserved moments on level J at the end of the timed "
                   "window, each form's run against the FP64 run of the same steps (the FP64 path matches the "
                   "oracle to 1e-12); BF16 storage does not reach the 1e-3 of 16-bit storage"}
        if exact is not None:
            line["exact_collision"] = exact
        if d3 is not None:
            line["d3q6_3d"] = d3
        if wide is not None:
            line["prediction_s"] = wide
        if serving is not None:
            line["batched"] = serving
        if legs is not None:
            line["configs"] = legs
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
