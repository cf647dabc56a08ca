"""Autotuner for the launch parameters of the step kernels.

For a workload it times a few candidate settings on the device (CUDA events
on the simulation's stream, after warm-up) and keeps the fastest:

* fused_R: staging capacity of the fused relax/advect kernel (32 R particles
  per cell pass; cells above it take a second sweep that redraws the random
  numbers), so the best value depends on the particles-per-cell distribution;
* grid_per_sm: persistent blocks per SM of the tiled kernels.

Results are cached in a JSON file keyed by the workload shape (dimension,
cells, particles per cell, precision, pipeline, GPU name).
"""
from __future__ import annotations

import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), ".tune_cache.json")
CANDIDATES_R = (4, 8, 12)
CANDIDATES_GRID = (4, 8, 16)


def _key(w, device_name):
    g, p = w["grid"], w["params"]
    cells = (g["nx"] if g["dim"] == 2 else 1) * g["ny"]
    return f'{device_name}|{g["dim"]}|{cells}|{p["ppc_ref"]}|{p["precision"]}|{p.get("pipeline", "plain")}'


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_steps(sim, steps, warmup=2):
    import torch
    sim.step(warmup)
    sim.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(sim.stream)
    sim.step(steps)
    b.record(sim.stream)
    b.synchronize()
    return a.elapsed_time(b) / 1e3 / steps


def tune(w, steps=6, use_cache=True, candidates_R=CANDIDATES_R, candidates_grid=CANDIDATES_GRID):
    """Best {"fused_R", "grid_per_sm", "s_per_step"} for workload w."""
    import torch
    from . import usp as U
    key = _key(w, torch.cuda.get_device_name())
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]
    fused = w["params"].get("pipeline", "plain") == "fused"
    sim = U.Simulation(w).init_particles()
    results = []
    for R in (candidates_R if fused else (0,)):
        for gps in candidates_grid:
            sim.set_tuning(R, gps)
            results.append((time_steps(sim, steps), R or sim.tuning()["fused_R"], gps))
    sim.close()
    t, R, gps = min(results)
    best = {"fused_R": R, "grid_per_sm": gps, "s_per_step": t,
            "tried": [{"fused_R": r, "grid_per_sm": g, "s_per_step": x} for x, r, g in results]}
    if use_cache:
        cache[key] = best
        _store(cache)
    return best


def apply(sim, cfg):
    sim.set_tuning(cfg["fused_R"], cfg["grid_per_sm"])
    return sim


def tune_batch(workloads, steps=6, use_cache=True, candidates_R=CANDIDATES_R, candidates_grid=CANDIDATES_GRID):
    """Best setting for a batch of simulations shaped like `workloads`
    (timed as a batch, since the persistent grid is shared by its members)."""
    import torch
    from . import usp as U
    key = "batch:" + str(len(workloads)) + ":" + _key(workloads[0], torch.cuda.get_device_name())
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]
    fused = workloads[0]["params"].get("pipeline", "plain") == "fused"
    sims = [U.Simulation(w).init_particles() for w in workloads]
    results = []
    for R in (candidates_R if fused else (0,)):
        for gps in candidates_grid:
            B = U.Batch(hbm_budget=1 << 40, max_sims=len(sims))
            for s in sims:
                s.set_tuning(R, gps)
                assert B.admit(s) == 0
            B.step(2)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(B.stream)
            B.step(steps)
            b.record(B.stream)
            b.synchronize()
            results.append((a.elapsed_time(b) / 1e3 / steps, R or sims[0].tuning()["fused_R"], gps))
            for s in sims:
                B.retire(s)
            B.close()
    for s in sims:
        s.close()
    t, R, gps = min(results)
    best = {"fused_R": R, "grid_per_sm": gps, "s_per_step": t,
            "tried": [{"fused_R": r, "grid_per_sm": g, "s_per_step": x} for x, r, g in results]}
    if use_cache:
        cache[key] = best
        _store(cache)
    return best
