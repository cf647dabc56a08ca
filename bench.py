#!/usr/bin/env python
"""Benchmark of the USP-ESBGK particle update on GB300.

Default workload: the Sod shock tube of Sec. 4.3 (1000 cells, 360 / 45
particles per cell, Kn = 1e-4, dt = 10 tau_c, FP32 particles, moment sums and
per-cell parameters, FP64 field averages), as a batch of B independent tubes (seeds 1..B) advanced together
by the graph-captured batched launches.  One bench step is one time step of
every tube.  The particle state (B * 2.0e5 particles, two buffers) is larger
than the 129 MB L2, so no flush is needed between steps.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
FUSED_SRC = os.path.join(ROOT, "paper_1808_03801_gb300", "csrc", "usp_fused.cu")
# DRAM bytes per particle of one k_g2 launch (ncu dram__bytes_read.sum +
# dram__bytes_write.sum of the 32-tube Sod case divided by its particles),
# valid only for the k_g2 source with this SHA-1; any other source reports
# traffic as null until it is captured again
KG2_TRAFFIC = {"sha1": "c8068930dd8fadfe0692a64c667f3a533efa6603", "bytes_per_particle": 38.84}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="usp", choices=["usp", "reference"])
    ap.add_argument("--batch", type=int, default=64, help="independent Sod tubes per GPU")
    ap.add_argument("--pipeline", default="auto", choices=["auto", "plain", "fused"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch autotuner")
    ap.add_argument("--prof-tubes", type=int, default=0,
                    help="profiling case for ncu: N tubes, 3 steps, then the stages of one step; no timing")
    ap.add_argument("--prof-r", type=int, default=0, help="profiling case: tuning value fused_R (0: default)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the serving leg (0: skip); the full mix of 256 unless --serve-scaled")
    ap.add_argument("--serve-scaled", action="store_true",
                    help="smaller requests (N <= 4e5, 100-400 steps) for a quick serving check")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-config legs (C1-C4 alone)")
    ap.add_argument("--only-config", nargs="*", default=None)
    return ap.parse_args()


def workload_cfg(batch, pipeline):
    return {"workload": "sod_shock_tube_batch", "cells": 1000, "ppc_left": 360, "ppc_right": 45,
            "particles_per_tube": 202500, "global_batch": batch, "Kn": 1e-4, "dt_over_tauc": 10.0,
            "storage": "fp32", "moments": "fp32 centred sums and per-cell parameters, fp64 Eq. 34 averages", "pipeline": pipeline,
            "l2": "state larger than L2 (no flush)", "parallelism": "replicas"}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"),
                                          f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def reduce_max(value, dist, device="cpu"):
    """Max of a per-rank number over all ranks (the timed region's length)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(particles_per_rank, world, steps, elapsed_max):
    """Updates of all ranks divided by the slowest rank's time (weak scaling)."""
    return particles_per_rank * world * steps / elapsed_max


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("USP_BENCH_GLOO") is None else "gloo")
        return rank, world, dist
    return rank, world, None


# --------------------------------------------------------------------------- oracle (CPU)
def oracle_rate(seconds, steps=None, warmup=0, seed=1):
    """The FP64 CPU oracle on one Sod tube, as it stands, single thread."""
    import oracle
    from paper_1808_03801_gb300 import workloads as W
    w = W.sod(precision="fp64", seed=seed)
    s = oracle.OracleSim(w).init_particles()
    n = s.n
    if warmup:
        s.step(warmup)
    done, t0 = 0, time.perf_counter()
    if steps is not None:
        s.step(steps)
        done = steps
    else:
        while time.perf_counter() - t0 < seconds or done < 3:
            s.step(1)
            done += 1
    el = time.perf_counter() - t0
    return n * done / el, n, done, el


def _oracle_worker(job):
    seconds, steps, warmup, seed = job
    return oracle_rate(seconds, steps=steps, warmup=warmup, seed=seed)


def host_cpu():
    """CPU model and usable cores of this host."""
    import platform
    model = None
    impl = part = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":", 1)[0].strip().lower()
            if key == "model name" and model is None:
                model = line.split(":", 1)[1].strip()
            elif key == "cpu implementer" and impl is None:
                impl = line.split(":", 1)[1].strip()
            elif key == "cpu part" and part is None:
                part = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if model is None and part is not None:
        names = {("0x41", "0xd4f"): "Arm Neoverse V2", ("0x41", "0xd40"): "Arm Neoverse V1",
                 ("0x41", "0xd0c"): "Arm Neoverse N1"}
        model = names.get((impl, part), f"Arm implementer {impl} part {part}")
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return {"model": model or platform.machine(), "cores": cores}


def oracle_rate_all_cores(seconds, steps=None, warmup=0):
    """The oracle as it stands on every host core at once: one process per
    core, each on its own Sod tube (seeds 1..P), the batch workload's shape.
    Processes are spawned (never forked after the GPU was used).  Returns the
    summed rate, the cores used, and the slowest process's steps and time."""
    import multiprocessing as mp
    cores = host_cpu()["cores"]
    jobs = [(seconds, steps, warmup, 1 + i) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    rate = sum(r[0] for r in res)
    n = res[0][1]
    done = min(r[2] for r in res)
    el = max(r[3] for r in res)
    return rate, cores, n, done, el


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    rate, cores, n, done, el = oracle_rate_all_cores(None, steps=args.steps, warmup=args.warmup)
    line = {"metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / max(done, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_cfg(args.batch, "oracle"),
            "cpu_baseline": {"value": rate, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} Sod tubes ({n} particles each), one per core, "
                                       f"{done} steps each per timed run", "cpu": host_cpu()["model"]},
            "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU
def make_batch(U, W, torch, batch, pipeline, precision="fp32", seed0=1, stream=None, tuning=None):
    sims = []
    for i in range(batch):
        w = W.sod(precision=precision, seed=seed0 + i)
        w["params"]["pipeline"] = pipeline
        sims.append(U.Simulation(w, stream=stream).init_particles())
        if tuning:
            sims[-1].set_tuning(tuning["fused_R"], tuning["grid_per_sm"])
    B = U.Batch(hbm_budget=200 << 30, max_sims=max(batch, 1), stream=stream)
    for s in sims:
        rc = B.admit(s)
        assert rc == 0, rc
    return sims, B


def time_batch_steps(torch, B, steps):
    st = B.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    B.step(steps)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / 1e3


def stage_times(torch, B, stages, steps=3):
    """Per-stage device time (CUDA events on the batch stream), average over steps."""
    st = B.stream
    acc = {k: 0.0 for k in stages}
    for _ in range(steps):
        for k in stages:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            B.run_stage(k)
            b.record(st)
            b.synchronize()
            acc[k] += a.elapsed_time(b) / 1e3
    return {k: v / steps for k, v in acc.items()}


def e2e_rate(U, W, torch, batch, pipeline, steps, warmup, stream):
    """Through the public API with host buffers: each tube's initial state is
    uploaded from pinned host memory (usp_set_particles), the batch advances
    `steps` steps, and every tube's fields come back to the host.  Each tube
    has a stream of its own, so the set-up kernels of one upload run beside
    the next one.  One untimed pass of `warmup` steps over the same handles
    and host buffers comes first (the first device access to the freshly
    pinned pages and the batch's graph capture); the next pass is timed."""
    import numpy as np
    sims = []
    hosts = []
    for i in range(batch):
        w = W.sod(precision="fp32", seed=1 + i)
        w["params"]["pipeline"] = pipeline
        s = U.Simulation(w, stream=torch.cuda.Stream()).init_particles()
        P = s.particles()
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy() for k, v in P.items()
               if k in ("pos", "vel", "pid")}
        hosts.append(pin)
        sims.append(s)
    torch.cuda.synchronize()
    B = U.Batch(hbm_budget=200 << 30, max_sims=batch, stream=stream)

    def solve(nsteps):
        # every upload first (each returns once its arrays are read, its sort
        # running on the tube's stream), then the admissions, which wait for
        # each tube's stream
        for s, h in zip(sims, hosts):
            s.set_particles(h["pos"], h["vel"], h["pid"])
        for s in sims:
            B.admit(s)
        B.step(nsteps)
        for s in sims:
            B.retire(s)
        return [s.sample() for s in sims]

    solve(max(1, warmup))
    t0 = time.perf_counter()
    fields = solve(steps)
    el = time.perf_counter() - t0
    n = sum(len(h["pid"]) for h in hosts)
    h2d = sum(h["pos"].nbytes + h["vel"].nbytes + h["pid"].nbytes for h in hosts)
    d2h = sum(f.nbytes for f in fields)
    B.close()
    for s in sims:
        s.close()
    return n * steps / el, h2d / steps, d2h / steps


def serving_leg(W, args, capacity):
    """Continuous batching of independent solves arriving as a Poisson stream at
    80% of the measured batched capacity; p50 / p99 time to solution."""
    from paper_1808_03801_gb300.serve import serve_requests
    if args.serve_scaled:
        reqs = W.serving_requests(n=args.serve_requests, n_min=1e4, n_max=4e5, steps_min=100, steps_max=400)
    else:
        reqs = W.serving_requests(n=args.serve_requests)
    work = []
    for w in reqs:
        g = w["grid"]
        cells = (g["nx"] if g["dim"] == 2 else 1) * g["ny"]
        work.append(cells * w["params"]["ppc_ref"] * w["steps"])
    rate = 0.8 * capacity / (sum(work) / len(work))
    rep, _ = serve_requests(reqs, rate=rate, hbm_budget=64 << 30, pipeline="fused", precision="fp32")
    rep.update({"arrival_rate_per_s": rate, "mix": "couette/poiseuille/cavity, FP32 fused, log-uniform N, Kn",
                "full_mix": not args.serve_scaled and args.serve_requests == 256})
    return rep


def kg2_traffic(n_particles):
    """ncu DRAM bytes of one k_g2 launch scaled to n_particles, or None when the
    kernel source differs from the one that was captured."""
    import hashlib
    with open(FUSED_SRC, "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()
    return KG2_TRAFFIC["bytes_per_particle"] * n_particles if sha == KG2_TRAFFIC["sha1"] else None


class L2Flush:
    """A device buffer larger than the 129 MB L2, rewritten between timed steps."""

    def __init__(self, torch, stream, nbytes=512 << 20):
        self.buf = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
        self.stream = stream
        self.torch = torch

    def __call__(self):
        with self.torch.cuda.stream(self.stream):
            self.buf.fill_(1.0)


def check_counters(name, sims):
    """Particles lost to slot overflow (counter 5) or spilled past a full
    bucket (counter 6) invalidate a timed run."""
    over = sum(s.info()["counters"][5] for s in sims)
    spill = sum(s.info()["counters"][6] for s in sims)
    assert over == 0 and spill == 0, f"{name}: overflow {over}, spilled {spill}"
    return {"overflow": over, "spilled": spill}


RECORD_BYTES = {(1, "fp32"): 20, (2, "fp32"): 24, (1, "fp64"): 36, (2, "fp64"): 44}


def time_sim_steps(torch, sim, steps, flush):
    """Device time of `steps` single steps of one simulation, the L2 flushed
    (outside the timed interval) before each."""
    st = sim.stream
    tot = 0.0
    for _ in range(steps):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        sim.step(1)
        b.record(st)
        b.synchronize()
        tot += a.elapsed_time(b) / 1e3
    return tot


def sim_stage_times(torch, sim, stages, flush, steps=3):
    st = sim.stream
    acc = {k: 0.0 for k in stages}
    for _ in range(steps):
        for k in stages:
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            sim.run_stage(k)
            b.record(st)
            b.synchronize()
            acc[k] += a.elapsed_time(b) / 1e3
    return {k: v / steps for k, v in acc.items()}


def config_leg(U, W, torch, name, w, pipeline, steps, warmup, stream, flush, hbm, comparator=True, tuning=None):
    """One benchmark configuration as a single simulation: particle-updates/s
    over `steps` single steps (L2 flushed before each), the per-stage device
    times, the roofline of the dominant kernel, the overflow / spill counters
    and the plain per-simulation FP64 path on the same workload."""
    import copy
    w = copy.deepcopy(w)
    w["params"]["pipeline"] = pipeline
    prec = w["params"]["precision"]
    sim = U.Simulation(w, stream=stream).init_particles()
    if tuning:
        sim.set_tuning(tuning["fused_R"], tuning["grid_per_sm"])
    sim.step(warmup)
    sim.synchronize()
    n = sim.info()["n_particles"]
    el = time_sim_steps(torch, sim, steps, flush)
    counters = check_counters(name, [sim])
    reservoir = any(f["kind"] == "reservoir" for f in w["faces"])
    stages = U.stage_list(pipeline)
    if reservoir and pipeline == "fused":
        stages = stages[:1] + [(11, "k_inject_f")] + stages[1:]
    st = sim_stage_times(torch, sim, [k for k, _ in stages], flush)
    names = dict(stages)
    top = max(st, key=st.get)
    rec = RECORD_BYTES[(w["grid"]["dim"], prec)]
    alg = 2 * rec * n
    step_s = el / steps
    out = {"workload": name, "particles": n, "cells": sim.K, "precision": prec, "pipeline": pipeline,
           "steps": steps, "ms_per_step": 1e3 * step_s, "value": n / step_s, "unit": METRIC,
           "l2": "flushed before every timed step",
           "roofline": {"bound": "hbm", "kernel": names[top], "bytes_per_particle": 2 * rec,
                        "achieved": alg / st[top] / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": alg / st[top] / 1e9 / hbm, "step_frac": alg / step_s / 1e9 / hbm},
           "stage_ms": {names[k]: 1e3 * v for k, v in st.items()}, "counters": counters}
    sim.close()
    if comparator and not (pipeline == "plain" and prec == "fp64"):
        wp = W.with_precision(w, "fp64")
        wp["params"]["pipeline"] = "plain"
        sp = U.Simulation(wp, stream=stream).init_particles()
        sp.step(1)
        sp.synchronize()
        k = 3 if n > 2e6 else 6
        elp = time_sim_steps(torch, sp, k, flush)
        rate = sp.info()["n_particles"] * k / elp
        out["plain_fp64_per_sim"] = {"value": rate, "unit": METRIC, "ratio": out["value"] / rate}
        sp.close()
    torch.cuda.synchronize()
    return out


def weighted_leg(U, W, torch, stream, flush, steps=20, warmup=20):
    """C1 Couette with the weighted added particles of Table 2 (plain FP64
    pipeline, P_ne from Kn_GLL, Eq. 34-averaged weight fields): the full USP
    step.  Its stages run as one captured sequence (no per-stage timing)."""
    w = W.couette()
    w["params"].update(weighted=1, weight_average=1, capacity_factor=4.0)
    sim = U.Simulation(w, stream=stream).init_particles()
    n0 = sim.info()["n_particles"]
    sim.step(warmup)
    sim.synchronize()
    n = sim.info()["n_particles"]
    el = time_sim_steps(torch, sim, steps, flush)
    n1 = sim.info()["n_particles"]
    assert sim.info()["counters"][5] == 0, "weighted Couette: particles lost"
    sim.close()
    step_s = el / steps
    return {"workload": "C1_couette_fp64_weighted", "particles": n, "particles_initial": n0,
            "particles_end": n1, "cells": w["grid"]["ny"], "precision": "fp64", "pipeline": "plain+weighted",
            "steps": steps, "ms_per_step": 1e3 * step_s, "value": 0.5 * (n + n1) / step_s, "unit": METRIC,
            "l2": "flushed before every timed step", "roofline": None}


def config_legs(U, W, torch, args, stream, hbm, pipeline):
    """Every benchmark shape of the paper's Sec. 4 at one GPU, each alone."""
    from paper_1808_03801_gb300 import autotune
    flush = L2Flush(torch, stream)
    legs = {}
    specs = [("C1_couette_fp64", W.couette(), "plain", 20),
             ("C2_sod_single", W.sod(), pipeline, 20),
             ("C3_cavity_Kn1e-3", W.cavity(Kn=1e-3), pipeline, 10),
             ("C3_cavity_Kn1e-2", W.cavity(Kn=1e-2), pipeline, 10),
             ("C4_slit", W.slit(), pipeline, 8)]
    for name, w, pipe, steps in specs:
        if args.only_config and name not in args.only_config:
            continue
        tuning = None
        if pipe == "fused" and not args.no_tune:
            import copy
            wt = copy.deepcopy(w)
            wt["params"]["pipeline"] = pipe
            tuning = autotune.tune(wt, use_cache=False)
        legs[name] = config_leg(U, W, torch, name, w, pipe, steps, 3, stream, flush, hbm,
                                comparator=not args.no_comparator, tuning=tuning)
        if tuning:
            legs[name]["tuning"] = {k: v for k, v in tuning.items() if k != "tried"}
    if not args.only_config or "C1_couette_fp64_weighted" in args.only_config:
        legs["C1_couette_fp64_weighted"] = weighted_leg(U, W, torch, stream, flush)
    del flush
    torch.cuda.empty_cache()
    return legs


def run_gpu(args):
    import torch
    rank, world, dist = dist_setup(args.gpus)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_1808_03801_gb300 import usp as U, workloads as W
    from paper_1808_03801_gb300 import build as Bd
    if rank == 0:
        Bd.build()
    if dist:
        dist.barrier()
    U.lib()
    pipeline = args.pipeline
    if pipeline == "auto":
        pipeline = "fused" if U.fused_available() else "plain"
    stream = torch.cuda.Stream()
    tuning = None
    if not args.no_tune:
        from paper_1808_03801_gb300 import autotune
        tw = []
        for i in range(args.batch):
            w = W.sod(precision="fp32", seed=100 + i)
            w["params"]["pipeline"] = pipeline
            tw.append(w)
        tuning = autotune.tune_batch(tw, use_cache=False)
    sims, B = make_batch(U, W, torch, args.batch, pipeline, stream=stream, tuning=tuning)
    n_total = sum(s.info()["n_particles"] for s in sims)
    B.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    el = time_batch_steps(torch, B, args.steps)
    torch.cuda.synchronize()
    if dist:
        el = reduce_max(el, dist, "cuda")
    clocks.stop()
    headline_counters = check_counters("sod batch", sims)
    value = whole_job_rate(n_total, world, args.steps, el)
    ms = 1e3 * el / args.steps

    # dominant kernel: per-stage times outside the graph, on the same stream
    stages = U.stage_list(pipeline)
    st = stage_times(torch, B, [k for k, _ in stages])
    names = dict(stages)
    top = max(st, key=st.get)
    hbm, src = peaks()
    rec = 20                         # FP32 1-D record: y, c0, c1, c2 (4 B each), pid (4 B)
    alg = 2 * rec * n_total          # read and write each particle once per step
    achieved = alg / st[top] / 1e9
    traffic = kg2_traffic(n_total) if names[top] == "k_g2" else None
    roof = {"bound": "hbm", "kernel": names[top], "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "peak_source": f"{src} hbm_gbs (copy, burst)",
            "stage_ms": {names[k]: 1e3 * v for k, v in st.items()},
            "step_frac": alg / (el / args.steps) / 1e9 / hbm}
    launches = U.launches_per_step(pipeline, reservoir=False) * args.steps

    result = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic",
              "config": dict(workload_cfg(args.batch, pipeline),
                             tuning={k: v for k, v in (tuning or {}).items() if k != "tried"}),
              "clocks": clocks.summary(), "roofline": roof,
              "gpu_launches": launches, "counters": headline_counters}
    B.close()
    for s in sims:
        s.close()
    del sims
    torch.cuda.synchronize()

    if rank == 0:
        e2e, h2d, d2h = e2e_rate(U, W, torch, args.batch, pipeline, args.steps, args.warmup, stream)
        result["e2e"] = {"value": e2e * world, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                         "note": "initial state uploaded once per solve from pinned host memory (one stream per "
                                 "tube) and fields read back at the end; bytes amortised over the steps; "
                                 "one untimed solve of the same tubes first"}
        if not args.no_comparator:
            # plain per-simulation FP64 path on the same tubes (fewer, timed alone)
            nb = min(4, args.batch)
            cmp_rates = []
            for i in range(nb):
                w = W.sod(precision="fp64", seed=1 + i)
                s = U.Simulation(w, stream=stream).init_particles()
                s.step(2)
                s.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                k = max(5, min(args.steps, 20))
                a.record(stream)
                s.step(k)
                b.record(stream)
                b.synchronize()
                cmp_rates.append(s.info()["n_particles"] * k / (a.elapsed_time(b) / 1e3))
                s.close()
            result["plain_fp64_per_sim"] = {"value": statistics.mean(cmp_rates), "unit": METRIC,
                                            "ratio": value / statistics.mean(cmp_rates)}
        if not args.no_configs:
            result["configs"] = config_legs(U, W, torch, args, stream, hbm, pipeline)
        if args.serve_requests > 0:
            result["serving"] = serving_leg(W, args, value)
        if not args.no_configs and world == 1:
            result["precision"] = precision_leg(U, W)
        if not args.no_cpu_baseline and world == 1:
            rate1, n, done1, el1 = oracle_rate(args.cpu_seconds)
            rate, cores, n, done, elc = oracle_rate_all_cores(args.cpu_seconds)
            result["cpu_baseline"] = {"value": rate, "unit": METRIC, "cores": cores, "kind": "oracle",
                                      "sample": f"{cores} Sod tubes ({n} particles each), one process per core, "
                                                f">= {done} steps each in {elc:.1f} s",
                                      "single_core": {"value": rate1, "sample": f"one Sod tube, {done1} steps "
                                                                                  f"({el1:.1f} s)"},
                                      "cpu": host_cpu()["model"]}
        print(json.dumps(result), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


FIELD_NAMES = ["n", "u0", "u1", "u2", "T", "pxx", "pyy", "pzz", "pxy", "pxz", "pyz", "q0", "q1", "q2", "Pne"]


def precision_leg(U, W, seeds=8):
    """Error of each time-averaged field of the fused FP32 path against the
    FP64 GPU path (which matches the FP64 oracle particle by particle), on
    Sod tubes of 200 cells x 200 particles and 60 steps after 40: for each
    field the relative difference of the domain averages and the largest
    |difference| / standard error over the cells (standard errors from
    independent seeds on each side)."""
    import numpy as np

    def runs(precision, pipeline, seed0):
        out = []
        for s in range(seeds):
            w = W.with_precision(W.sod(ny=200, ppc_left=200, seed=seed0 + s), precision)
            w["params"]["pipeline"] = pipeline
            g = U.Simulation(w).init_particles()
            g.step(40)
            acc = None
            for _ in range(60):
                g.step(1)
                f = g.sample()[:len(FIELD_NAMES)]
                acc = f if acc is None else acc + f
            assert g.info()["counters"][5] == 0, f"precision {precision}: particles lost"
            g.close()
            out.append(acc / 60)
        return np.array(out)
    t0 = time.time()
    a = runs("fp32", "fused", 1)
    b = runs("fp64", "plain", 1001)
    rows = {}
    for k, name in enumerate(FIELD_NAMES):
        fa, fb = a[:, k], b[:, k]
        ma, mb = fa.mean(0), fb.mean(0)
        se = np.sqrt(fa.var(0, ddof=1) / seeds + fb.var(0, ddof=1) / seeds)
        z = np.where(se > 0, (ma - mb) / np.where(se > 0, se, 1.0), 0.0)
        da, db = fa.mean(1), fb.mean(1)
        sed = math.sqrt(da.var(ddof=1) / seeds + db.var(ddof=1) / seeds)
        den = abs(db.mean())
        rows[name] = {"rel_err_domain_mean": float(abs(da.mean() - db.mean()) / den) if den > 0 else 0.0,
                      "z_domain_mean": float((da.mean() - db.mean()) / sed) if sed > 0 else 0.0,
                      "max_abs_z_cell": float(np.abs(z).max()), "mean_z2_cell": float((z ** 2).mean())}
    return {"reference": "plain FP64 GPU path (per-particle parity with the FP64 oracle)",
            "case": f"Sod, 200 cells, 200/25 particles per cell, {seeds} seeds per side, fields averaged over "
                    "steps 41-100", "seconds": round(time.time() - t0, 1), "fields": rows}


def run_profile_case(args):
    """Small case of the bench workload for kernel captures: N Sod tubes in one
    batch, three warm-up steps, then the five stages of one step."""
    import torch
    from paper_1808_03801_gb300 import usp as U, workloads as W
    sims = []
    for i in range(args.prof_tubes):
        w = W.sod(precision="fp32", seed=1 + i)
        w["params"]["pipeline"] = "fused"
        sims.append(U.Simulation(w).init_particles())
        if args.prof_r:
            sims[-1].set_tuning(args.prof_r, 0)
    B = U.Batch(hbm_budget=64 << 30, max_sims=len(sims))
    for sim in sims:
        assert B.admit(sim) == 0
    B.step(3)
    torch.cuda.synchronize()
    for k, _ in U.stage_list("fused"):
        B.run_stage(k)
    torch.cuda.synchronize()
    print("profile case done:", sum(sim.info()["n_particles"] for sim in sims), "particles")


def main():
    args = parse()
    if args.prof_tubes:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
