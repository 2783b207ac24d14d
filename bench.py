#!/usr/bin/env python
"""Benchmark of the DSMC hot path: particle-steps/s of the 5e7-particle VHS workload
(argon, omega = 0.81, Kn = 0.1, 2,000 cells x 25,000 particles per cell) on one GB300,
one JSON line on stdout.

A step is one DSMC time step over every particle: collisions with the symmetric
moment sample, free flight with the body force and the walls, and the stable cell
sort (four kernel launches).  The particle state (1.6 GB with its sort buffer) is
resident in HBM and larger than L2, so no flush is needed between steps.  Besides the
headline, the line carries (one GPU):
  precision   the same run with binary64 moment sums (options.accum) against the
              default binary32 ones: time per step and their difference;
  hs_kn1      the 20,000-particle hard-sphere run (L2-resident, launch-bound): time per
              step under CUDA-graph replay;
  batched     the 256-instance batched workload (one batch handle, tuned partition,
              graph replay) against the same instances stepped as single runs;
  serving     2,000 micro-solve requests arriving at 50/s, each to a 1 % standard
              error of its channel-mean velocity, through the request loop
              (continuous batching), against 8 of them solved one after another;
  cpu_baseline / cpu_all_cores   the oracle on one and on all host cores.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank advances its own independent
instance (seed = rank): replicas with no data-path collective; the barrier and the
max over ranks of the timed region only frame the measurement.

--impl reference times the CPU oracle (the plain C DSMC the GPU path is checked
against) on the host cores, on the same workload; under torchrun only rank 0 runs it.
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

from paper_2311_14140_gb300 import workloads as W  # noqa: E402

WORKLOAD = W.VHS_KN01_50M
METRIC = "particle-steps/s"

# Algorithmic bytes per launch of each kernel, per particle (N) or per histogram
# entry (W x n_cells), as stated in the design notes.
def algorithmic_bytes(kernel: str, N: int, n_cells: int, sort_warps: int) -> float:
    return {
        "collide_move": 32.0 * N,         # y, vx, vy, vz read and written once, in place
        "scatter_spans": 32.0 * N,        # state read once, written once to the other buffer
        "scan_hist": 12.0 * sort_warps * n_cells,
        "cell_offsets": 8.0 * n_cells,
        "index_count": 4.0 * N,
        "index_scatter": 32.0 * N,
        "init": 16.0 * N,
    }.get(kernel, 0.0)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if that summary
    was taken from the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("sources_sha256") != sources_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch_full_size")


# Sources of the step kernels the committed traffic figures were taken from.
STEP_SOURCES = ("dsmc_step.cu", "dsmc_device.cuh", "dsmc_internal.h")


def _code_only(text: str) -> str:
    """The source without its comments and trailing blanks (so a reworded comment does not
    void a traffic record of unchanged kernels)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_14140_gb300", "csrc")
    for fn in STEP_SOURCES:
        with open(os.path.join(csrc, fn), encoding="utf-8") as f:
            h.update(fn.encode() + b"\0" + _code_only(f.read()).encode())
    return h.hexdigest()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline_sample(steps: int = 2) -> dict:
    """The oracle as it stands on one host core: `steps` steps of the full workload after
    its initialisation (not timed)."""
    import oracle
    w = WORKLOAD
    s = oracle.OracleSim(omega=w.omega, Kn=w.Kn, F=w.body_force, n_cells=w.n_cells,
                         ppc=w.ppc, seed=0, sample_start=1, G=w.group_size)
    t0 = time.perf_counter()
    s.step(steps)
    t = time.perf_counter() - t0
    s.close()
    return {"value": w.n_particles * steps / t, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of the full {w.name} workload "
                      f"({w.n_particles * steps:.1e} particle-steps) after initialisation, "
                      "single-threaded C oracle"}


def _oracle_config0(seed: int) -> float:
    """One full hard-sphere Kn = 1 run of the oracle (100 cells x 200 particles, 2,000
    steps, the last 1,000 sampled); returns its seconds."""
    import oracle
    w = W.HS_KN1
    s = oracle.OracleSim(omega=w.omega, Kn=w.Kn, F=w.body_force, n_cells=w.n_cells,
                         ppc=w.ppc, seed=seed, sample_start=w.sample_start)
    t0 = time.perf_counter()
    s.step(w.steps)
    t = time.perf_counter() - t0
    s.close()
    return t


def cpu_all_cores() -> dict:
    """The oracle on every host core at once: one process per core, each the full
    hard-sphere Kn = 1 run with its own seed (processes started with spawn)."""
    import multiprocessing as mp
    P = os.cpu_count() or 1
    w = W.HS_KN1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(P) as pool:
        times = pool.map(_oracle_config0, range(100, 100 + P))
    wall = time.perf_counter() - t0
    work = P * w.n_particles * w.steps
    return {"value": work / wall, "unit": METRIC, "cores": P, "kind": "oracle",
            "sample": f"{P} processes, each the full {w.name} run ({w.steps} steps x "
                      f"{w.n_particles} particles, own seed); wall {wall:.2f} s including "
                      f"process start, slowest run {max(times):.2f} s",
            "per_core_value": w.n_particles * w.steps / (sum(times) / len(times))}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    w = WORKLOAD
    s = oracle.OracleSim(omega=w.omega, Kn=w.Kn, F=w.body_force, n_cells=w.n_cells,
                         ppc=w.ppc, seed=0, sample_start=1, G=w.group_size)
    # One oracle step of the full workload takes seconds on one core: bound the sample
    # so that the whole run stays within a few minutes.
    warm = min(args.warmup, 3)
    timed_steps = min(args.steps, 20)
    s.step(warm)
    t0 = time.perf_counter()
    s.step(timed_steps)
    t = time.perf_counter() - t0
    s.close()
    value = w.n_particles * timed_steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / timed_steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(w, args.gpus),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{timed_steps} timed steps of the full workload after "
                                       f"{warm} untimed (at most 20 and 3 of the requested "
                                       f"{args.steps} and {args.warmup}), single-threaded "
                                       "C oracle"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_dict(w, n_gpus):
    return {"workload": w.name, "gas": "argon VHS omega=0.81", "Kn": w.Kn,
            "n_cells": w.n_cells, "ppc": w.ppc, "n_particles_per_gpu": w.n_particles,
            "body_force": w.body_force, "group_size": w.group_size,
            "dt_factor": w.dt_factor, "parallelism": f"replicas x{n_gpus}",
            "l2": "inputs larger than L2 (1.6 GB resident state vs 129 MB L2)"}


def batch_defs(n: int = 256):
    return [dict(Kn=w.Kn, n_cells=w.n_cells, ppc=w.ppc, omega=w.omega,
                 body_force=w.body_force, seed=w.seeds[0]) for w in W.batch_instances(n)]


def run_batched(steps: int, warmup: int, rank: int, span: int = 0,
                sequential: bool = True) -> dict:
    """The 256-instance batched workload (Kn log-uniform in [0.05, 10], 50-1000 cells,
    50-400 particles per cell, force 0.5-2 x the Kn = 1 force): one batch handle with
    the tuned span partition (or `span` particles per span on 4-warp CTAs), steps
    replayed as CUDA graphs, against the same instances stepped one after another as
    plain single runs (unless `sequential` is false)."""
    import torch
    from paper_2311_14140_gb300 import Dsmc, DsmcBatch
    defs = batch_defs()
    if rank:
        for d in defs:
            d["seed"] += rank << 32
    n_part = sum(d["n_cells"] * d["ppc"] for d in defs)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        if span:
            b = DsmcBatch(defs, sample_start=1, graph=True, stream=side.cuda_stream,
                          span_particles=span, cta_warps=4)
            best = span
        else:
            b = DsmcBatch(defs, sample_start=1, graph=True, stream=side.cuda_stream)
            best, tuned_ms = b.autotune(steps_per_trial=3)
        b.step(max(warmup, 16))
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(side)
        b.step(steps)
        e1.record(side)
        side.synchronize()
        t_batch = e0.elapsed_time(e1) / 1e3
        # kernel shares of the same steps launched directly with timing events
        b.set_options(profile=True, graph=False)
        b.reset_kernel_times()
        b.step(8)
        kt = b.kernel_times()
        info = b.info(0)
        b.close()
        del b
    torch.cuda.synchronize()
    ms_cm, n_cm = kt.get("collide_move", (0.0, 0))
    tot = sum(v[0] for v in kt.values())
    peak, peak_kind = peaks()
    value = n_part * steps / t_batch
    out = {
        "workload": "batch256: Kn log-uniform [0.05,10], 50-1000 cells, 50-400 ppc, HS argon",
        "n_instances": len(defs), "n_particles": n_part, "steps": steps,
        "value": value, "unit": METRIC, "ms_per_step": 1e3 * t_batch / steps,
        "instance_steps_per_s": len(defs) * steps / t_batch,
        "span_particles": best, "graph_replay": True,
        "effective_step": {"bytes_per_particle_step": 32,
                           "gbs": 32.0 * value / 1e9, "frac": 32.0 * value / 1e9 / peak,
                           "peak_kind": peak_kind},
        "collide_move_share": ms_cm / tot if tot else None,
        "collide_move_gbs": (32.0 * n_part / (ms_cm / 1e3 / n_cm) / 1e9) if n_cm else None,
        "cells_per_span_instance0": info["cells_per_span"],
    }
    if not sequential:
        return out
    # The same instances as separate plain runs, stepped one after another.
    runs = [Dsmc(sample_start=1, **d) for d in defs]
    stream = torch.cuda.current_stream()
    for r in runs:
        r.step(warmup)
    torch.cuda.synchronize()
    seq_steps = max(1, min(steps, 20))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in runs:
        r.step(seq_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    for r in runs:
        r.close()
    del runs
    torch.cuda.synchronize()
    out["sequential_single_runs"] = {"value": n_part * seq_steps / t_seq, "unit": METRIC,
                                     "ms_per_step": 1e3 * t_seq / seq_steps,
                                     "steps": seq_steps}
    out["speedup_vs_sequential"] = value / (n_part * seq_steps / t_seq)
    return out


def run_precision(steps: int) -> dict:
    """The benchmark workload with binary64 moment sums against the default binary32
    ones: same seed, hence the same trajectory; `steps` sampled steps each, then the
    time per step of each mode and the largest difference of the sums, relative to
    count x <|v|^2>^(degree / 2) (the size of the sum of |products| up to a factor of
    order one)."""
    import numpy as np
    import torch
    from paper_2311_14140_gb300 import Dsmc
    w = WORKLOAD
    out, ms = {}, {}
    for accum in (0, 1):
        g = Dsmc(w.Kn, w.n_cells, w.ppc, omega=w.omega, body_force=w.body_force, seed=7,
                 sample_start=1, group_size=w.group_size, dt_factor=w.dt_factor,
                 accum=accum)
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[accum] = e0.elapsed_time(e1) / steps
        out[accum] = g.moments()[0]
        g.close()
        torch.cuda.synchronize()
    m32, m64 = out[0], out[1]
    deg = np.array([0, 1, 1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3], np.float64)
    cnt = np.maximum(m64[:, 0], 1.0)
    e = np.maximum((m64[:, 4] + m64[:, 5] + m64[:, 6]) / cnt, 1e-30)
    scale = cnt[:, None] * e[:, None] ** (deg / 2.0)
    rel = np.abs(m32 - m64) / scale
    return {"sampled_steps": steps,
            "fp32": {"ms_per_step": ms[0], "accum": "binary32 per-lane sums (default)"},
            "fp64": {"ms_per_step": ms[1], "accum": "binary64 per-lane sums"},
            "fp32_vs_fp64_max_rel": float(rel.max()),
            "fp32_vs_fp64_max_rel_by_degree": {str(d): float(rel[:, deg == d].max())
                                               for d in (0, 1, 2, 3)}}


def run_hs_kn1(steps: int = 2048) -> dict:
    """The 20,000-particle hard-sphere Kn = 1 run (L2-resident, launch-bound): time per
    step under CUDA-graph replay (16 steps per replay), sampling on."""
    import torch
    from paper_2311_14140_gb300 import Dsmc
    w = W.HS_KN1
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        g = Dsmc(w.Kn, w.n_cells, w.ppc, omega=w.omega, body_force=w.body_force, seed=0,
                 sample_start=1, graph=True, stream=side.cuda_stream)
        g.step(64)
        g.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(side)
        g.step(steps)
        e1.record(side)
        side.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        g.close()
    return {"workload": w.name, "n_particles": w.n_particles, "steps": steps,
            "us_per_step": 1e6 * t / steps, "value": w.n_particles * steps / t,
            "unit": METRIC, "graph_replay": True,
            "l2": "state 0.64 MB with its sort buffer: L2-resident, no HBM roofline"}


def serve_leg(n_requests: int, rate: float, target_se: float, warmup_steps: int,
              pool_particles: int, time_limit: float, sequential: int, rank: int) -> dict:
    """Serving workload: Poisson arrivals of micro-solve requests drawn as the batched
    workload, each run to a relative standard error of its channel-mean velocity
    (capped at 200,000 steps), through the library's request loop on one pool
    (continuous batching, graph replay); beside it, the first `sequential` requests
    solved one after another as plain runs.  Micro-solves/s and latency percentiles
    count requests that met their target only; capped and unfinished ones are reported
    separately."""
    import numpy as np
    import torch
    from paper_2311_14140_gb300 import DsmcPool, solve
    reqs = W.serving_requests(n_requests, rate, target_se, seed=4242 + 1000 * rank)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        pool = DsmcPool(max_particles=pool_particles, max_cells=pool_particles // 50,
                        max_instances=4096, max_cells_per_instance=1000,
                        sample_start=warmup_steps, graph=True, stream=side.cuda_stream)
        t0 = time.perf_counter()
        res = pool.serve(reqs, epoch_steps=32, batches=16, time_limit=time_limit)
        wall = time.perf_counter() - t0
        pool.close()
    conv = [k for k, r in enumerate(res) if r["converged"] == 1 and r["finished"] >= 0]
    capped = sum(1 for r in res if r["converged"] == 0 and r["finished"] >= 0)
    unfinished = sum(1 for r in res if r["finished"] < 0)
    lat = np.array([res[k]["finished"] - reqs[k]["arrival"] for k in conv])
    qwait = np.array([r["admitted"] - q["arrival"] for r, q in zip(res, reqs)
                      if r["admitted"] >= 0])
    psteps = sum(r["steps"] * q["n_cells"] * q["ppc"] for r, q in zip(res, reqs))
    # The same requests one at a time as plain runs (graph replay on their own stream).
    seq = []
    t1 = time.perf_counter()
    with torch.cuda.stream(side):
        for q in reqs[:sequential]:
            seq.append(solve(q, epoch_steps=32, batches=16, sample_start=warmup_steps,
                             graph=True, stream=side.cuda_stream))
    t_seq = time.perf_counter() - t1
    seq_conv = sum(1 for r in seq if r["converged"] == 1)
    seq_psteps = sum(r["steps"] * q["n_cells"] * q["ppc"] for r, q in zip(seq, reqs))

    def pct(a, p):
        return float(np.percentile(a, p)) if a.size else None

    served = len(conv) / wall
    seq_rate = seq_conv / t_seq if t_seq > 0 else None
    return {
        "metric": "micro-solves/s", "value": served, "unit": "micro-solves/s",
        "workload": "serving: Poisson arrivals at 50/s, requests drawn as batch256 (Kn "
                    "log-uniform [0.05, 10], 50-1000 cells, 50-400 ppc, force 0.5-2 x the "
                    "Kn = 1 force), HS argon",
        "requests": n_requests, "rate_per_s": rate, "target_se": target_se,
        "max_steps": reqs[0]["max_steps"], "warmup_steps": warmup_steps,
        "pool_particles": pool_particles, "epoch_steps": 32, "se_batches": 16,
        "time_limit_s": time_limit, "wall_s": wall,
        "converged": len(conv), "capped": capped, "unfinished": unfinished,
        "latency_s_converged": {"p50": pct(lat, 50), "p99": pct(lat, 99),
                                "max": float(lat.max()) if lat.size else None},
        "queue_wait_s": {"p50": pct(qwait, 50), "p99": pct(qwait, 99)},
        "particle_steps_per_s": psteps / wall,
        "sequential_plain_solves": {
            "requests": len(seq), "converged": seq_conv, "seconds": t_seq,
            "micro_solves_per_s": seq_rate,
            "particle_steps_per_s": seq_psteps / t_seq if t_seq > 0 else None},
        "served_over_sequential": (served / seq_rate) if seq_rate else None,
    }


def run_serve(args, world, rank, local):
    """The serving workload alone, as its own JSON line (all ranks serve their own
    request streams: replicas)."""
    import torch
    from paper_2311_14140_gb300 import _build
    _build.build()
    torch.cuda.set_device(local)
    barrier(world)
    clocks = Clocks(local)
    clocks.start()
    leg = serve_leg(args.requests, args.rate, args.target_se, args.warmup_steps,
                    args.pool_particles, args.serve_time_limit, args.sequential_sample, rank)
    clk = clocks.stop()
    line = dict(leg)
    line.update({"value": world * leg["value"], "n_gpus": world, "higher_is_better": True,
                 "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                 "config": {"workload": leg["workload"], "parallelism": f"replicas x{world}"},
                 "clocks": clk})
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_batched_only(args, world, rank, local):
    """The batched workload alone, as its own JSON line: a fixed partition when
    --batch-span is given (no tuning, no sequential comparison: a profiling case)."""
    import torch
    from paper_2311_14140_gb300 import _build
    _build.build()
    torch.cuda.set_device(local)
    barrier(world)
    clocks = Clocks(local)
    clocks.start()
    leg = run_batched(args.steps, args.warmup, rank, span=args.batch_span,
                      sequential=not args.batch_span)
    clk = clocks.stop()
    line = {"metric": METRIC, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": leg["workload"], "parallelism": f"replicas x{world}"},
            "value": world * leg["value"], "ms_per_step": leg["ms_per_step"],
            "batched": leg, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2311_14140_gb300 import Dsmc, _build
    _build.build()
    torch.cuda.set_device(local)
    w = WORKLOAD
    stream = torch.cuda.current_stream()
    g = Dsmc(w.Kn, w.n_cells, w.ppc, omega=w.omega, body_force=w.body_force, seed=rank,
             sample_start=1, group_size=w.group_size, dt_factor=w.dt_factor)
    info = g.info()
    N = info["n_particles"]
    g.step(args.warmup)
    g.sync()

    # Device-timed region: K steps, CUDA events on the launch stream around the region
    # only (per-launch events would add about 2 % to a step).
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    t_dev = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
    # Kernel durations: the next K steps of the same run with an event pair around every
    # launch on the launch stream (the roofline's kernel time and the launch count).
    g.set_options(profile=True)
    g.reset_kernel_times()
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    g.step(args.steps)
    e3.record(stream)
    torch.cuda.synchronize()
    t_prof = e2.elapsed_time(e3) / 1e3
    kt = g.kernel_times()
    launches = sum(c for _, c in kt.values())
    g.sync()
    g.close()
    del g
    torch.cuda.synchronize()

    # End-to-end region through the public API, from host memory: the particle state
    # (a checkpoint in pinned host memory) is loaded into a new run (host-to-device copy
    # and sort into cells), then K steps, each followed by a read of the moment sums
    # into pinned host memory.
    g1 = Dsmc(w.Kn, w.n_cells, w.ppc, omega=w.omega, body_force=w.body_force,
              seed=1000 + rank, sample_start=1, group_size=w.group_size,
              dt_factor=w.dt_factor)
    g1.step(2)
    host = [torch.empty(N, dtype=torch.float32, pin_memory=True) for _ in range(4)]
    g1.state_into(*host)
    smax = g1.cells()[1]
    g1.close()
    del g1
    out = torch.empty((w.n_cells, 13), dtype=torch.float64, pin_memory=True)
    g2 = Dsmc(w.Kn, w.n_cells, w.ppc, omega=w.omega, body_force=w.body_force,
              seed=1000 + rank, sample_start=1, group_size=w.group_size,
              dt_factor=w.dt_factor)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g2.load_state(*host, smax=smax, step=2)
    for _ in range(args.steps):
        g2.step(1)
        g2.moments(out)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    g2.close()
    del g2, host

    value = world * N * args.steps / t_dev
    peak, peak_kind = peaks()
    dom = max(kt, key=lambda k: kt[k][0])
    ms_total, cnt = kt[dom]
    per_launch_s = ms_total / 1e3 / max(cnt, 1)
    alg = algorithmic_bytes(dom, N, w.n_cells, info["n_spans"])
    achieved = alg / per_launch_s / 1e9
    kernels = {k: {"ms_per_launch": (v[0] / v[1]) if v[1] else None, "launches": v[1],
                   "share": v[0] / sum(x[0] for x in kt.values()),
                   "alg_bytes_per_launch": algorithmic_bytes(k, N, w.n_cells, info["n_spans"]),
                   "gbs": (algorithmic_bytes(k, N, w.n_cells, info["n_spans"]) /
                           (v[0] / 1e3 / v[1]) / 1e9) if v[1] and v[0] > 0 else None}
               for k, v in kt.items() if v[1]}
    result = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(w, world),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic(dom), "alg_bytes_per_launch": alg},
        "effective_step": {"bytes_per_particle_step": 32,
                           "gbs": 32.0 * N * args.steps / t_dev / 1e9,
                           "frac": 32.0 * N * args.steps / t_dev / 1e9 / peak},
        "kernels": kernels,
        "kernel_timing": {"region": "the K steps after the headline's, with a CUDA event "
                                    "pair around every launch on the launch stream",
                          "ms_per_step": 1e3 * t_prof / args.steps},
        "clocks": clk,
        "e2e": {"value": world * N * args.steps / t_e2e, "unit": METRIC,
                "h2d_bytes_per_step": 16 * N / args.steps,
                "d2h_bytes_per_step": w.n_cells * 13 * 8,
                "includes": "a host checkpoint of the state (16 B per particle, pinned) "
                            "loaded into a run (copy and sort into cells; counted once and "
                            "spread over the K steps), K steps, a moment read into pinned "
                            "host memory after every step"},
        "gpu_launches": launches,
    }
    def leg(name, fn):
        try:
            result[name] = fn()
        except Exception as e:  # a failing extra leg must not lose the headline
            result[name] = {"error": f"{type(e).__name__}: {e}"}

    if world == 1 and not args.no_extras:
        leg("precision", lambda: run_precision(args.precision_steps))
        leg("hs_kn1", run_hs_kn1)
    if not args.no_batched:
        leg("batched", lambda: run_batched(args.steps, args.warmup, rank))
    if world == 1 and not args.no_serve:
        leg("serving", lambda: serve_leg(args.requests, args.rate, args.target_se,
                                         args.warmup_steps, args.pool_particles,
                                         args.serve_time_limit, args.sequential_sample,
                                         rank))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_sample()
        leg("cpu_all_cores", cpu_all_cores)
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 256-instance batched measurement")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving workload alone (its own JSON line)")
    ap.add_argument("--no-serve", action="store_true",
                    help="leave the serving workload out of the main line")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the precision and hard-sphere Kn = 1 measurements")
    ap.add_argument("--precision-steps", type=int, default=1000)
    ap.add_argument("--serve-time-limit", type=float, default=300.0,
                    help="seconds after which the request loop stops (unfinished requests "
                         "are reported as such)")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--target-se", type=float, default=0.01)
    ap.add_argument("--warmup-steps", type=int, default=256)
    ap.add_argument("--pool-particles", type=int, default=64_000_000)
    ap.add_argument("--sequential-sample", type=int, default=8)
    ap.add_argument("--batched-only", action="store_true",
                    help="run the 256-instance batched workload alone (its own JSON line)")
    ap.add_argument("--batch-span", type=int, default=0,
                    help="with --batched-only: particles per span instead of tuning, and "
                         "no sequential comparison (profiling cases)")
    ap.add_argument("--cells", type=int, default=None,
                    help="override the cell count (profiling cases only)")
    ap.add_argument("--ppc", type=int, default=None,
                    help="override particles per cell (profiling cases only)")
    args = ap.parse_args()
    global WORKLOAD
    if args.cells or args.ppc:
        WORKLOAD = W.scaled(WORKLOAD, n_cells=args.cells, ppc=args.ppc)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        if args.serve:
            return run_serve(args, world, rank, local)
        if args.batched_only:
            return run_batched_only(args, world, rank, local)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
