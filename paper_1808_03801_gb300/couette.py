"""Transport coefficients from Couette and thermal Couette flows (Sec. 4.1).

Couette: diffuse plates moving at -/+ u_w; thermal Couette: plates at rest
at T_w + dT (bottom) and T_w - dT (top), dT = 10 K.  After the steady state
is reached, the instantaneous fields are sampled every step (every fifth
below dt = tau_c);
in the central 60 % of the gap the shear stress p_xy (heat flux q_y) is
averaged and the velocity (temperature) profile fitted by a line.  The bulk
ratios

    mu_eff / mu    = -p_xy / (mu(T) du/dy)
    kappa_eff / kappa = -q_y / (kappa(T) dT/dy),   kappa = (15/4)(k/m) mu (Pr = 2/3)

need no slip or jump model; they are 1 for a scheme with the transport
coefficients of the gas (Fig. 1 plots the stress and heat flux themselves).
The sampled stress and heat flux are those of Eq. 33.

    python -m paper_1808_03801_gb300.couette --kind shear thermal --dt 0.2 1 5
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import usp as U
from . import workloads as W

KB = 1.380649e-23


def workload(kind: str, dt_over_tauc: float, ppc: int, mode: str, Kn: float = 0.01, ny: int = 100,
             seed: int = 1, gll_average: int = 0) -> dict:
    u_w = 20.0 if kind == "shear" else 0.0
    w = W.couette(ny=ny, ppc=ppc, Kn=Kn, u_wall=u_w, dt_over_tauc=dt_over_tauc, precision="fp32", seed=seed,
                  omega=0.81)
    if kind == "thermal":
        w["faces"][2]["T"] = W.T0 + 10.0
        w["faces"][3]["T"] = W.T0 - 10.0
    w["params"]["mode"] = mode
    w["params"]["pipeline"] = "fused"
    w["params"]["gll_average"] = gll_average
    return w


def run(kind: str = "thermal", dt_over_tauc: float = 1.0, mode: str = "usp", ppc: int = 1000,
        relax_times: float = 6.0, avg_times: float = 8.0, min_samples: int = 20000, seed: int = 1,
        gll_average: int = 0) -> dict:
    w = workload(kind, dt_over_tauc, ppc, mode, seed=seed, gll_average=gll_average)
    t0 = time.time()
    g = U.Simulation(w).init_particles()
    try:
        inf = g.info()
        dt, mu_ref = inf["dt"], inf["mu_ref"]
        H = w["grid"]["hi"][1] - w["grid"]["lo"][1]
        rho = W.N0 * w["gas"]["mass"]
        # slowest diffusive time of the gap (momentum: mu / rho; heat: 1.5 mu / rho)
        t_diff = H * H / (math.pi ** 2 * mu_ref / rho)
        n_relax = int(relax_times * t_diff / dt)
        # one sample per step once a step relaxes most particles (samples
        # nearly independent), else every fifth; at least min_samples
        sample_every = 1 if dt_over_tauc >= 1.0 else 5
        n_avg = max(int(avg_times * t_diff / dt), min_samples * sample_every)
        g.step(n_relax)
        nsamp = n_avg // sample_every
        acc = np.zeros((16, g.K))   # the sampled fields, [field][cell]
        for _ in range(nsamp):
            g.step(sample_every)
            acc += g.sample()
        inf = g.info()
    finally:
        g.close()
    F = acc / nsamp
    ny = w["grid"]["ny"]
    y = (np.arange(ny) + 0.5) * H / ny
    c = slice(int(0.2 * ny), int(0.8 * ny))
    T = float(F[4][c].mean())
    mu = mu_ref * (T / w["gas"]["T_ref"]) ** w["gas"]["omega"]
    if kind == "shear":
        slope = np.polyfit(y[c], F[1][c], 1)[0]
        flux = float(F[8][c].mean())
        ratio = -flux / (mu * slope)
    else:
        slope = np.polyfit(y[c], F[4][c], 1)[0]
        flux = float(F[12][c].mean())
        kappa = 15.0 / 4.0 * KB / w["gas"]["mass"] * mu
        ratio = -flux / (kappa * slope)
    # standard error of the bulk flux from the spread over the central cells
    se = float(F[8 if kind == "shear" else 12][c].std(ddof=1) / math.sqrt(c.stop - c.start))
    return {"kind": kind, "dt_over_tauc": dt_over_tauc, "mode": mode, "gll_average": gll_average, "ppc": ppc,
            "cells": ny,
            "steps": n_relax + nsamp * sample_every, "samples": nsamp, "ratio": float(ratio),
            "ratio_se": abs(float(ratio)) * se / max(abs(flux), 1e-300), "flux": flux, "slope": float(slope),
            "T_bulk": T, "lost": int(inf["counters"][5]), "wall_s": round(time.time() - t0, 2)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--kind", nargs="+", default=["thermal"], choices=["shear", "thermal"])
    ap.add_argument("--dt", type=float, nargs="+", default=[1.0])
    ap.add_argument("--mode", nargs="+", default=["usp"], choices=["usp", "sp"])
    ap.add_argument("--ppc", type=int, default=1000)
    ap.add_argument("--gll-average", type=int, default=0)
    a = ap.parse_args(argv)
    for k in a.kind:
        for r in a.dt:
            for m in a.mode:
                print(json.dumps(run(k, r, m, a.ppc, gll_average=a.gll_average)), flush=True)


if __name__ == "__main__":
    main()
