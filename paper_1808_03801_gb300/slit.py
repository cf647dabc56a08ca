"""Reduced mass flow rate through a slit (Sec. 4.5, Eqs. 40-41).

Runs the cases of Table 7 (delta = 20, vacuum downstream) on the GPU and
reports W = Mdot / Mdot_fm from the net particle count through the plane of
the slit (usp_params.flux_axis / flux_pos, counters[7]), averaged over the
last 60 % of the steps in blocks (mean and standard error of the blocks).

    python -m paper_1808_03801_gb300.slit --case 4 --ppc 100 --steps 10000
    python -m paper_1808_03801_gb300.slit --case 4 --ppc 40 --steps 8000 --chamber 10 20 40
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import usp as U
from . import workloads as W


def run_case(case: int = 4, ppc: int = 100, steps: int = 10000, mode: str = "usp", gll_average: int = 0,
             pipeline: str = "fused", seed: int = 1, blocks: int = 12, warm_frac: float = 0.4,
             chamber: float = 10.0) -> dict:
    w = W.slit_case(case, ppc=ppc, seed=seed, chamber=chamber)
    w["params"].update(pipeline=pipeline, mode=mode, gll_average=gll_average)
    if pipeline == "plain":
        w["params"]["precision"] = "fp64"
    t0 = time.time()
    g = U.Simulation(w).init_particles()
    try:
        dt = g.info()["dt"]
        warm = int(warm_frac * steps)
        g.step(warm)
        chunk = max(1, (steps - warm) // blocks)
        Ws = []
        c_prev = g.info()["counters"][7]
        for _ in range(blocks):
            g.step(chunk)
            c = g.info()["counters"][7]
            Ws.append(U.reduced_mass_flow(w, c - c_prev, chunk, dt))
            c_prev = c
        inf = g.info()
    finally:
        g.close()
    Ws = np.asarray(Ws)
    nx, ny, r = w["grid"]["nx"], w["grid"]["ny"], w["params"]["dt_over_tauc"]
    return {"case": case, "chamber_a": chamber, "cells": [nx, ny], "dt_over_tauc": r, "mode": mode,
            "gll_average": gll_average,
            "pipeline": pipeline, "ppc": ppc, "steps": steps, "reservoir_cols": w["params"]["reservoir_cols"],
            "W": float(Ws.mean()), "se": float(Ws.std(ddof=1) / math.sqrt(len(Ws))),
            "n_particles_end": int(inf["n_particles"]), "spilled": int(inf["counters"][6]),
            "lost": int(inf["counters"][5]), "wall_s": round(time.time() - t0, 2)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--case", type=int, nargs="+", default=[4])
    ap.add_argument("--ppc", type=int, default=100)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--mode", default="usp", choices=["usp", "sp"])
    ap.add_argument("--gll-average", type=int, default=0)
    ap.add_argument("--pipeline", default="fused", choices=["fused", "plain"])
    ap.add_argument("--chamber", type=float, nargs="+", default=[10.0],
                    help="half-length and height of the domain in slit widths (cells scaled to keep their size)")
    a = ap.parse_args(argv)
    for c in a.case:
        for ch in a.chamber:
            steps = int(round(a.steps * ch / 10.0))   # the flow develops over a time that grows with the domain
            print(json.dumps(run_case(c, a.ppc, steps, a.mode, a.gll_average, a.pipeline, chamber=ch)), flush=True)


if __name__ == "__main__":
    main()
