"""Seeded synthetic workloads shaped like the paper's benchmark problems.

This module only states inputs: gas constants, grids, boundary conditions,
run parameters, initial regions, seeds, and a seeded numpy generator for
arbitrary particle states.  It holds none of the method's arithmetic; the
CUDA library and the CPU oracle each derive everything else (viscosity from
Kn, the time step from tau_c, particle counts, ...) on their own.

A workload is a plain dict:

    gas     : mass [kg], T_ref [K], mu_ref (0: derive from Kn), omega, Pr
    grid    : dim (1: y resolved; 2: x and y), nx, ny, lo, hi [m]
    faces   : four dicts (x-lo, x-hi, y-lo, y-hi): kind, T [K], u [m/s], n [1/m^3]
    segments: zero-thickness plates normal to x: pos, lo, hi, kind, T, u
    params  : Kn, L_ref, n_ref, dt [s] (0: use dt_over_tauc), dt_over_tauc,
              body_accel, ppc_ref, n_avg, mode ('usp' | 'sp' | 'fixed'),
              fixed_pne, reservoir_cols, precision ('fp64' | 'fp32'),
              flux_axis / flux_pos (optional counting plane)
    regions : initial uniform boxes: lo, hi, n, T, u
    seed    : key of the counter-based generator
    steps   : number of time steps of the full problem

The paper's cases (Sec. 4) use argon; the hard-sphere variant (omega = 0.5)
is used where the workload says so.
"""
from __future__ import annotations

import copy
import math

import numpy as np

M_AR = 6.63e-26          # kg, argon-like molecular mass
T0 = 273.0               # K
N0 = 2.687e25            # 1/m^3, 1 atm at 273 K
PR_MONO = 2.0 / 3.0      # Prandtl number of a monatomic gas


def _face(kind, T=T0, u=(0.0, 0.0, 0.0), n=0.0):
    return {"kind": kind, "T": float(T), "u": tuple(float(x) for x in u), "n": float(n)}


def _base(dim, nx, ny, lo, hi, faces, *, Kn, L_ref, dt_over_tauc, ppc, omega=0.5,
          precision="fp64", mode="usp", steps=100, seed=1, regions=None, n_ref=N0):
    return {
        "gas": {"mass": M_AR, "T_ref": T0, "mu_ref": 0.0, "omega": omega, "Pr": PR_MONO},
        "grid": {"dim": dim, "nx": nx, "ny": ny, "lo": tuple(lo), "hi": tuple(hi)},
        "faces": faces,
        "segments": [],
        "params": {"Kn": Kn, "L_ref": L_ref, "n_ref": n_ref, "dt": 0.0, "dt_over_tauc": dt_over_tauc,
                   "body_accel": (0.0, 0.0, 0.0), "ppc_ref": ppc, "n_avg": 1000, "mode": mode,
                   "fixed_pne": 0.0, "reservoir_cols": 0, "precision": precision},
        "regions": regions if regions is not None else
        [{"lo": tuple(lo), "hi": tuple(hi), "n": n_ref, "T": T0, "u": (0.0, 0.0, 0.0)}],
        "seed": seed,
        "steps": steps,
    }


def couette(ny=100, ppc=100, Kn=0.1, u_wall=50.0, dt_over_tauc=0.5, precision="fp64", steps=2000,
            seed=1, omega=0.5):
    """1-D Couette flow (Sec. 4.1): diffuse plates at y = 0 and y = H moving at -/+ u_wall."""
    H = 5.0e-7
    faces = [_face("periodic"), _face("periodic"),
             _face("diffuse", T0, (-u_wall, 0, 0)), _face("diffuse", T0, (u_wall, 0, 0))]
    return _base(1, 1, ny, (0.0, 0.0), (1.0, H), faces, Kn=Kn, L_ref=H, dt_over_tauc=dt_over_tauc,
                 ppc=ppc, omega=omega, precision=precision, steps=steps, seed=seed)


def poiseuille(ny=50, ppc=100, Kn=0.1, accel=None, dt_over_tauc=0.2, precision="fp64", steps=2000,
               seed=1, omega=0.81):
    """1-D Poiseuille flow (Sec. 4.2, Table 3): diffuse plates at rest, body force along x.

    The pressure gradient dp/dx of Table 3 enters as a body acceleration a_x = -(dp/dx)/rho."""
    H = 5.0e-7
    faces = [_face("periodic"), _face("periodic"), _face("diffuse"), _face("diffuse")]
    w = _base(1, 1, ny, (0.0, 0.0), (1.0, H), faces, Kn=Kn, L_ref=H, dt_over_tauc=dt_over_tauc,
              ppc=ppc, omega=omega, precision=precision, steps=steps, seed=seed)
    w["params"]["body_accel"] = (accel if accel is not None else 1.5e10, 0.0, 0.0)
    return w


# Table 3: Kn, dp/dx [Pa/m], cells, dt / tau_c of the paper's Poiseuille cases (USP-ESBGK column)
POISEUILLE_CASES = {1: (0.100, 2.70e10, 50, 0.2), 2: (0.020, 1.60e9, 70, 0.5), 3: (0.004, 6.68e7, 100, 2.0),
                    4: (0.001, 4.00e6, 100, 5.0)}
# mean free path of argon at 1 atm and 273 K by Eq. 36 with mu = 2.117e-5 Pa s
# (the usual argon reference viscosity; the paper gives Kn and dp/dx only)
LAMBDA_AR_STD = 6.36e-8


def poiseuille_case(case=4, ppc=200, precision="fp32", steps=200000, seed=1, mode="usp", cells=None):
    """A Poiseuille case of Table 3 (Sec. 4.2): argon (omega = 0.81) at 1 atm
    and 273 K between diffuse plates at 273 K, gap H = lambda / Kn, driven by
    the printed dp/dx as a body acceleration (dp/dx) / rho along x.  `cells`
    overrides the printed cell count."""
    Kn, dpdx, ncell, r = POISEUILLE_CASES[case]
    ncell = cells or ncell
    H = LAMBDA_AR_STD / Kn
    faces = [_face("periodic"), _face("periodic"), _face("diffuse"), _face("diffuse")]
    w = _base(1, 1, ncell, (0.0, 0.0), (1.0, H), faces, Kn=Kn, L_ref=H, dt_over_tauc=r, ppc=ppc,
              omega=0.81, precision=precision, mode=mode, steps=steps, seed=seed)
    w["params"]["body_accel"] = (dpdx / (N0 * M_AR), 0.0, 0.0)
    w["dpdx"] = dpdx
    return w


def sod(ny=1000, ppc_left=360, Kn=1e-4, dt_over_tauc=10.0, precision="fp32", steps=500, seed=1):
    """1-D Sod shock tube (Sec. 4.3) in the normalised form rho_L = 1, p_L = 1,
    rho_R = 0.125, p_R = 0.1, u = 0, with specular end walls.  The density
    ratio 8 is carried by the particle counts (ppc_left : ppc_left / 8) and
    the pressure ratio by T_R = 0.8 T_L."""
    L = 1.0
    faces = [_face("periodic"), _face("periodic"), _face("specular"), _face("specular")]
    regions = [
        {"lo": (0.0, 0.0), "hi": (1.0, 0.5 * L), "n": N0, "T": T0, "u": (0.0, 0.0, 0.0)},
        {"lo": (0.0, 0.5 * L), "hi": (1.0, L), "n": N0 / 8.0, "T": 0.8 * T0, "u": (0.0, 0.0, 0.0)},
    ]
    return _base(1, 1, ny, (0.0, 0.0), (1.0, L), faces, Kn=Kn, L_ref=L, dt_over_tauc=dt_over_tauc,
                 ppc=ppc_left, precision=precision, steps=steps, seed=seed, regions=regions)


def cavity(n=200, ppc=100, Kn=1e-3, dt_over_tauc=None, u_lid=50.0, precision="fp32", steps=5000,
           seed=1, omega=0.81):
    """2-D lid-driven cavity (Sec. 4.4, Tables 5-6): diffuse walls at 273 K, the
    y-hi wall moving at u_lid along x.  The default time step follows the
    paper's rule dt / tau_c = 0.3 dx / lambda with dx = L / n, lambda = Kn L."""
    L = 1.0e-4
    if dt_over_tauc is None:
        dt_over_tauc = 0.3 / (n * Kn)
    faces = [_face("diffuse"), _face("diffuse"), _face("diffuse"), _face("diffuse", T0, (u_lid, 0, 0))]
    return _base(2, n, n, (0.0, 0.0), (L, L), faces, Kn=Kn, L_ref=L, dt_over_tauc=dt_over_tauc,
                 ppc=ppc, omega=omega, precision=precision, steps=steps, seed=seed)


def slit(nx=400, ny=200, ppc=200, Kn=1e-2, dt_over_tauc=1.0, pressure_ratio=10.0, precision="fp32",
         steps=2000, seed=1, reservoir_cols=2, delta=None, chamber=10.0):
    """2-D flow through a slit (Sec. 4.5), upper half domain: x in [-c a, c a],
    y in [0, c a] with c = `chamber` (10 by default, the paper's height of
    20a for the full domain); specular symmetry plane at y = 0; diffuse wall at y = c a;
    a zero-thickness diffuse plate at x = 0 for y >= a/2; reservoir buffer
    columns at both x ends (upstream n_1, downstream n_1 / pressure_ratio at
    the same temperature; pressure_ratio = inf gives the paper's vacuum).
    Hard-sphere gas; Kn refers to the slit width a, unless the rarefaction
    parameter delta is given: then the viscosity at the upstream state
    follows Eq. 40 (mu_1 = a p_1 / (delta v_1), v_1 = sqrt(2 k T_1 / m)).
    The whole domain starts at the upstream state.  A counting plane at
    x = 0 gives the net particle flow through the slit (Eq. 41)."""
    a = 1.0e-5
    lo, hi = (-chamber * a, 0.0), (chamber * a, chamber * a)
    n_down = 0.0 if math.isinf(pressure_ratio) else N0 / pressure_ratio
    faces = [_face("reservoir", T0, (0, 0, 0), N0), _face("reservoir", T0, (0, 0, 0), n_down),
             _face("specular"), _face("diffuse")]
    w = _base(2, nx, ny, lo, hi, faces, Kn=Kn, L_ref=a, dt_over_tauc=dt_over_tauc, ppc=ppc, omega=0.5,
              precision=precision, steps=steps, seed=seed)
    w["segments"] = [{"pos": 0.0, "lo": 0.5 * a, "hi": chamber * a, "kind": "diffuse", "T": T0,
                      "u": (0.0, 0.0, 0.0)}]
    w["params"]["reservoir_cols"] = reservoir_cols
    w["params"]["flux_axis"] = 1
    w["params"]["flux_pos"] = 0.0
    w["slit_width"] = a
    if delta is not None:
        kB = 1.380649e-23
        p1 = N0 * kB * T0
        v1 = math.sqrt(2.0 * kB * T0 / M_AR)
        w["gas"]["mu_ref"] = a * p1 / (delta * v1)
    return w


# Table 7: (cells along x, cells along y, dt / tau_c,1) of the paper's slit cases
SLIT_CASES = {1: (580, 280, 0.2), 2: (580, 280, 1.0), 3: (580, 280, 2.0), 4: (280, 140, 3.0),
              5: (160, 80, 4.0), 6: (160, 80, 5.0)}


def slit_case(case=4, ppc=100, precision="fp32", steps=4000, seed=1, buffer_flights=3.0, chamber=10.0):
    """A slit case of Table 7: delta = 20, vacuum downstream.  `chamber` scales
    the domain (half-length and height, in slit widths) at the case's cell
    size (the printed cell counts are for chamber = 10).

    The reservoir buffer must be deeper than a particle flies in one step, or
    the particles that would enter from beyond it are missing and the
    upstream chamber is starved.  With Eq. 36 at the upstream state, Eq. 37
    and Eq. 40, a most-probable-speed flight is v_1 dt = 0.8 (dt / tau_c,1)
    a / delta; the buffer is `buffer_flights` such flights deep (at least 2
    cells)."""
    nx, ny, r = SLIT_CASES[case]
    delta = 20.0
    dx_over_a = 20.0 / nx
    cols = max(2, math.ceil(buffer_flights * 0.8 * r / (delta * dx_over_a)))
    scale = chamber / 10.0
    return slit(nx=int(round(nx * scale)), ny=int(round(ny * scale)), ppc=ppc, dt_over_tauc=r,
                pressure_ratio=math.inf, precision=precision, steps=steps, seed=seed, delta=delta,
                reservoir_cols=cols, chamber=chamber)


def homogeneous_box(ppc=1000, Kn=0.05, dt_over_tauc=0.5, mode="usp", precision="fp64", Pr=PR_MONO,
                    fixed_pne=0.0):
    """A single periodic cell: no gradients, so the relaxation acts alone."""
    H = 1.0e-6
    faces = [_face("periodic")] * 4
    w = _base(1, 1, 1, (0.0, 0.0), (1.0, H), faces, Kn=Kn, L_ref=H, dt_over_tauc=dt_over_tauc,
              ppc=ppc, precision=precision, mode=mode, steps=10)
    w["gas"]["Pr"] = Pr
    w["params"]["fixed_pne"] = fixed_pne
    return w


def homogeneous_column(ny=2000, ppc=500, Kn=0.05, dt_over_tauc=0.5, mode="usp", precision="fp64", Pr=PR_MONO,
                       fixed_pne=0.0):
    """ny periodic cells of the homogeneous box's size stacked along y: a
    uniform gas, so every cell relaxes alone, with cells small enough for
    the per-cell work of the fused pipeline (positions y in [0, ny 1e-6])."""
    H = 1.0e-6
    faces = [_face("periodic")] * 4
    w = _base(1, 1, ny, (0.0, 0.0), (1.0, ny * H), faces, Kn=Kn, L_ref=H, dt_over_tauc=dt_over_tauc,
              ppc=ppc, precision=precision, mode=mode, steps=10)
    w["gas"]["Pr"] = Pr
    w["params"]["fixed_pne"] = fixed_pne
    return w


def bimaxwellian(n, T=(1.3 * T0, 0.85 * T0, 0.85 * T0), u=(0.0, 0.0, 0.0), y_range=(0.0, 1.0e-6),
                 x_range=(0.0, 1.0), seed=7, heat_skew=0.0):
    """Seeded particle state: positions uniform in the box, velocity component i
    Gaussian with variance k_B T_i / m (k_B written out as a number), plus an
    optional skew along y that gives the state a heat flux.  Returns
    (pos[n, 2], vel[n, 3], pid[n])."""
    rng = np.random.default_rng(seed)
    kb_over_m = 1.380649e-23 / M_AR
    pos = np.empty((n, 2))
    pos[:, 0] = rng.uniform(x_range[0], x_range[1], n)
    pos[:, 1] = rng.uniform(y_range[0], y_range[1], n)
    vel = np.empty((n, 3))
    for i in range(3):
        vel[:, i] = u[i] + math.sqrt(kb_over_m * T[i]) * rng.standard_normal(n)
    if heat_skew:
        e = rng.standard_exponential(n) - 1.0
        vel[:, 1] += heat_skew * math.sqrt(kb_over_m * T[1]) * e
    pid = rng.permutation(n).astype(np.uint32)
    return pos, vel, pid


def serving_requests(n=256, seed=12345, n_min=1e4, n_max=4e6, steps_min=500, steps_max=5000):
    """Request stream for the continuous-batching server: problem type uniform
    over Couette / Poiseuille / cavity, particle count log-uniform in
    [n_min, n_max], Kn log-uniform in [1e-3, 1], steps uniform in
    [steps_min, steps_max]; each request keeps its own seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = ["couette", "poiseuille", "cavity"][int(rng.integers(0, 3))]
        npart = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        Kn = float(np.exp(rng.uniform(np.log(1e-3), np.log(1.0))))
        steps = int(rng.integers(steps_min, steps_max + 1))
        if kind == "cavity":
            ncell = max(4, int(round(math.sqrt(npart / 100.0))))
            w = cavity(n=ncell, ppc=100, Kn=Kn, precision="fp32", steps=steps, seed=i + 1)
        elif kind == "couette":
            ny = max(4, int(round(npart / 100.0)))
            w = couette(ny=ny, ppc=100, Kn=Kn, precision="fp32", steps=steps, seed=i + 1)
        else:
            ny = max(4, int(round(npart / 100.0)))
            w = poiseuille(ny=ny, ppc=100, Kn=Kn, precision="fp32", steps=steps, seed=i + 1)
        w["name"] = f"req{i}:{kind}"
        w["steps"] = steps
        out.append(w)
    return out


def with_precision(w, precision):
    w = copy.deepcopy(w)
    w["params"]["precision"] = precision
    return w


# The five benchmark shapes: Couette FP64, Sod, cavity, slit, serving mix.
def C1():
    return couette()


def C2():
    return sod()


def C3(Kn=1e-3):
    return cavity(Kn=Kn)


def C4():
    return slit()
