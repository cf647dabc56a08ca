"""Poiseuille flow against the Navier-Stokes solution (Sec. 4.2, Eqs. 38-39).

Runs a case of Table 3 on the GPU from rest, lets it reach its steady state,
then averages the instantaneous velocity and temperature profiles sampled
every `sample_every` steps over the last `avg_frac` of the run.  The
profiles are compared with the no-slip continuum solution

    U(y) = (dp/dx) (H y - y^2) / (2 mu)                                (Eq. 38)
    T(y) = T_w + (dp/dx)^2 [H^4 / 16 - (y - H/2)^4] / (12 mu kappa)    (Eq. 39)

with mu at the wall temperature and kappa = (15/4) (k / m) mu (Pr = 2/3).
Reported: the least-squares scale of each profile onto its continuum shape
(1 = Navier-Stokes; for U it is mu / mu_eff), the relative L2 error of U and
the relative L2 distance of U from its scaled parabola (the shape).

    python -m paper_1808_03801_gb300.poiseuille --case 4 --mode usp sp
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import usp as U
from . import workloads as W

KB = 1.380649e-23


def navier_stokes(w: dict, mu: float, y: np.ndarray):
    """Eqs. 38-39 at the cell centres y."""
    H = w["grid"]["hi"][1] - w["grid"]["lo"][1]
    dpdx = w["dpdx"]
    Tw = w["faces"][2]["T"]
    kappa = 15.0 / 4.0 * KB / w["gas"]["mass"] * mu
    u = dpdx * (H * y - y * y) / (2.0 * mu)
    T = Tw + dpdx ** 2 * (H ** 4 / 16.0 - (y - H / 2.0) ** 4) / (12.0 * mu * kappa)
    return u, T


def _slip_fit(u, u_ns):
    """Relative L2 residual of u against a * u_ns + b (a parabola with slip)."""
    A = np.stack([u_ns, np.ones_like(u_ns)], axis=1)
    coef, *_ = np.linalg.lstsq(A, u, rcond=None)
    fit = A @ coef
    return float(np.linalg.norm(u - fit) / np.linalg.norm(fit))


def run_case(case: int = 4, mode: str = "usp", ppc: int = 200, steps: int = 200000, sample_every: int = 100,
             avg_frac: float = 0.5, pipeline: str = "fused", seed: int = 1, cells: int | None = None) -> dict:
    w = W.poiseuille_case(case, ppc=ppc, mode=mode, seed=seed, cells=cells)
    w["params"]["pipeline"] = pipeline
    if pipeline == "plain":
        w["params"]["precision"] = "fp64"
    t0 = time.time()
    g = U.Simulation(w).init_particles()
    try:
        inf = g.info()
        mu = inf["mu_ref"] * (w["faces"][2]["T"] / w["gas"]["T_ref"]) ** w["gas"]["omega"]
        g.step(int((1.0 - avg_frac) * steps))
        nsamp = max(1, int(avg_frac * steps) // sample_every)
        su = np.zeros(g.K)
        sT = np.zeros(g.K)
        for _ in range(nsamp):
            g.step(sample_every)
            F = g.sample()
            su += F[1]
            sT += F[4]
        inf = g.info()
    finally:
        g.close()
    u, T = su / nsamp, sT / nsamp
    ny = w["grid"]["ny"]
    H = w["grid"]["hi"][1] - w["grid"]["lo"][1]
    y = (np.arange(ny) + 0.5) * H / ny
    u_ns, T_ns = navier_stokes(w, mu, y)
    Tw = w["faces"][2]["T"]
    u_scale = float(np.dot(u, u_ns) / np.dot(u_ns, u_ns))
    T_scale = float(np.dot(T - Tw, T_ns - Tw) / np.dot(T_ns - Tw, T_ns - Tw))
    Kn, dpdx, _, r = W.POISEUILLE_CASES[case]
    return {"case": case, "Kn": Kn, "dt_over_tauc": r, "cells": ny, "mode": mode, "pipeline": pipeline,
            "ppc": ppc, "steps": steps, "samples": nsamp,
            "u_scale": u_scale, "u_rel_l2": float(np.linalg.norm(u - u_ns) / np.linalg.norm(u_ns)),
            "u_shape_l2": float(np.linalg.norm(u - u_scale * u_ns) / np.linalg.norm(u_scale * u_ns)),
            "u_slip_fit_l2": _slip_fit(u, u_ns),
            "u_max": float(u.max()), "u_max_ns": float(u_ns.max()),
            "T_scale": T_scale, "dT_max": float(T.max() - Tw), "dT_max_ns": float(T_ns.max() - Tw),
            "n_particles": int(inf["n_particles"]), "lost": int(inf["counters"][5]),
            "wall_s": round(time.time() - t0, 2)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--case", type=int, nargs="+", default=[4])
    ap.add_argument("--mode", nargs="+", default=["usp"], choices=["usp", "sp"])
    ap.add_argument("--ppc", type=int, default=200)
    ap.add_argument("--steps", type=int, default=200000)
    ap.add_argument("--pipeline", default="fused", choices=["fused", "plain"])
    ap.add_argument("--cells", type=int, default=None, help="override the cell count of Table 3")
    a = ap.parse_args(argv)
    for c in a.case:
        for m in a.mode:
            print(json.dumps(run_case(c, m, a.ppc, a.steps, pipeline=a.pipeline, cells=a.cells)), flush=True)


if __name__ == "__main__":
    main()
