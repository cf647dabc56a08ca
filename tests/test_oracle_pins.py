"""Pins of the oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself: closed-form
free flight, exact invariants of the relaxation, numpy's sample moments, the
closed-form expectation of one homogeneous relaxation step derived from
Eqs. 8b, 29-33, the Maxwellian fixed point of Eqs. 5-6, the Pr = 1 (BGK)
special case, the exact central difference of a linear profile (Eq. 18), and
the identity nu * tau_c = 0.8 that follows from Eqs. 36-37 with nu = p/mu.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import (PH_MOMENTS, PH_PARAMS, PH_RELAX, PH_RESERVOIR, PH_SAMPLE, PH_SORT,
                    PH_STREAM)
from paper_1808_03801_gb300 import workloads as W

KB_M = 1.380649e-23 / W.M_AR


def _run_phases(s, phases):
    for ph in phases:
        s.phase(ph)


def _by_pid(P):
    o = np.argsort(P["pid"])
    return {k: v[o] for k, v in P.items()}


# --------------------------------------------------------------------------- streaming
def test_specular_free_flight_closed_form():
    """1-D specular walls: the final position and velocity follow from unfolding
    the straight path y + c dt into [0, H] (mirror images)."""
    w = W.sod(ny=10, ppc_left=8, precision="fp64")
    w["params"]["dt"] = 3.0e-4
    s = oracle.OracleSim(w)
    rng = np.random.default_rng(3)
    n = 2000
    pos = np.column_stack([np.zeros(n), rng.uniform(0, 1, n)])
    vel = rng.normal(0, 2000.0, (n, 3))
    pid = np.arange(n, dtype=np.uint32)
    s.set_particles(pos, vel, pid)
    s.phase(PH_STREAM)
    P = _by_pid(s.particles())
    yy = pos[:, 1] + vel[:, 1] * 3.0e-4
    m = np.floor(yy)
    r = yy - m
    even = (m.astype(np.int64) % 2) == 0
    y_exp = np.where(even, r, 1.0 - r)
    vy_exp = np.where(even, vel[:, 1], -vel[:, 1])
    assert np.allclose(P["pos"][:, 1], y_exp, rtol=0, atol=1e-12)
    assert np.array_equal(P["vel"][:, 1], vy_exp)
    assert np.array_equal(P["vel"][:, [0, 2]], vel[:, [0, 2]])


def test_periodic_wrap_and_body_force():
    w = W.poiseuille(ny=8, ppc=4, accel=1.0e9, precision="fp64")
    w["faces"][2] = {"kind": "periodic", "T": 273.0, "u": (0, 0, 0), "n": 0.0}
    w["faces"][3] = dict(w["faces"][2])
    w["params"]["dt"] = 1.0e-8
    s = oracle.OracleSim(w)
    rng = np.random.default_rng(5)
    n = 500
    H = w["grid"]["hi"][1]
    pos = np.column_stack([np.zeros(n), rng.uniform(0, H, n)])
    vel = rng.normal(0, 300.0, (n, 3))
    s.set_particles(pos, vel, np.arange(n, dtype=np.uint32))
    s.phase(PH_STREAM)
    P = _by_pid(s.particles())
    y_exp = np.mod(pos[:, 1] + vel[:, 1] * 1e-8, H)
    assert np.allclose(P["pos"][:, 1], y_exp, rtol=0, atol=1e-18)
    assert np.allclose(P["vel"][:, 0], vel[:, 0] + 1.0e9 * 1e-8, rtol=1e-14)


def test_diffuse_wall_reemission_distribution():
    """Full accommodation: after a hit on the moving upper wall the normal speed is
    Rayleigh distributed with scale sqrt(R T_w) (flux-weighted Maxwellian) and the
    tangential components are N(u_w, R T_w); the remaining flight is straight."""
    w = W.couette(ny=10, ppc=10, u_wall=50.0, precision="fp64")
    H = w["grid"]["hi"][1]
    dt = 1.0e-11
    w["params"]["dt"] = dt
    s = oracle.OracleSim(w)
    n = 20000
    rng = np.random.default_rng(11)
    y0 = H - rng.uniform(0, 0.5 * 400.0 * dt, n)
    vel = np.column_stack([rng.normal(0, 300, n), np.full(n, 400.0), rng.normal(0, 300, n)])
    s.set_particles(np.column_stack([np.zeros(n), y0]), vel, np.arange(n, dtype=np.uint32))
    s.phase(PH_STREAM)
    P = _by_pid(s.particles())
    th = KB_M * 273.0
    cn = -P["vel"][:, 1]
    assert np.all(cn > 0)
    assert stats.kstest(cn / math.sqrt(th), "rayleigh").pvalue > 1e-3
    assert stats.kstest((P["vel"][:, 0] - 50.0) / math.sqrt(th), "norm").pvalue > 1e-3
    assert stats.kstest(P["vel"][:, 2] / math.sqrt(th), "norm").pvalue > 1e-3
    t_hit = (H - y0) / 400.0
    assert np.allclose(P["pos"][:, 1], H + P["vel"][:, 1] * (dt - t_hit), rtol=0, atol=1e-15 * H + 1e-20)


# --------------------------------------------------------------------------- sort and moments
def _couette_after(phases, steps_before=3, **kw):
    w = W.couette(ny=20, ppc=50, precision="fp64", **kw)
    s = oracle.OracleSim(w).init_particles()
    s.step(steps_before)
    _run_phases(s, phases)
    return w, s


def test_sort_is_cell_then_pid_and_counts_sum():
    w, s = _couette_after([PH_STREAM, PH_RESERVOIR, PH_SORT])
    P = s.particles()
    H = w["grid"]["hi"][1]
    cell = np.clip(np.floor(P["pos"][:, 1] / (H / 20)).astype(int), 0, 19)
    assert np.array_equal(cell, P["cell"])
    order = np.lexsort((P["pid"], P["cell"]))
    assert np.array_equal(order, np.arange(len(order)))
    assert s.counts().sum() == s.n == 1000
    assert np.array_equal(np.bincount(cell, minlength=20), s.counts())


def test_moments_match_numpy_sample_moments():
    w, s = _couette_after([PH_STREAM, PH_RESERVOIR, PH_SORT, PH_MOMENTS, PH_PARAMS])
    P = s.particles()
    prm = s.params()
    s.phase(PH_RELAX)
    s.phase(PH_SAMPLE)
    F = s.fields()
    for c in range(20):
        v = P["vel"][P["cell"] == c]
        u = v.mean(axis=0)
        cov = np.cov(v.T, bias=True)
        theta = np.trace(cov) / 3.0
        assert np.allclose(prm[c, 0:3], u, rtol=1e-13, atol=1e-10)
        assert math.isclose(prm[c, 3], theta, rel_tol=1e-12)
        assert math.isclose(F[4, c], theta / KB_M, rel_tol=1e-12)
        n = len(v) * W.N0 / 50
        assert math.isclose(F[0, c], n, rel_tol=1e-14)
        assert F[15, c] == len(v)


# --------------------------------------------------------------------------- relaxation
def test_relaxation_conserves_mass_momentum_energy_per_cell():
    w, s = _couette_after([PH_STREAM, PH_RESERVOIR, PH_SORT, PH_MOMENTS, PH_PARAMS])
    before = s.particles()
    s.phase(PH_RELAX)
    after = s.particles()
    assert np.array_equal(before["pid"], after["pid"])
    assert np.array_equal(before["pos"], after["pos"])
    prm = s.params()
    changed = 0
    for c in range(20):
        sel = before["cell"] == c
        vb, va = before["vel"][sel], after["vel"][sel]
        scale = np.abs(vb).sum()
        assert np.all(np.abs(vb.sum(0) - va.sum(0)) <= 1e-13 * scale)
        eb, ea = (vb ** 2).sum(), (va ** 2).sum()
        assert abs(eb - ea) <= 1e-13 * eb
        moved = np.any(vb != va, axis=1).sum()
        assert moved == prm[c, 15]
        changed += moved
    # relaxed fraction follows 1 - exp(-nu_ES dt) (Eqs. 8b, 9): binomial within 5 sigma
    ntot = len(before["pid"])
    p = np.array([prm[c, 10] for c in before["cell"]])
    mean, sd = p.sum(), math.sqrt((p * (1 - p)).sum())
    assert abs(changed - mean) < 5 * sd + 2 * 20   # lone relaxed particles are reverted


def test_nu_tau_c_identity_and_dt():
    """nu tau_c = 0.8 at any state (Eqs. 36-37 with nu = p/mu), so at the reference
    state nu dt = 0.8 dt/tau_c; nu scales as n T^(1 - omega) (Eq. 35)."""
    w = W.homogeneous_box(ppc=2000, dt_over_tauc=0.7)
    s = oracle.OracleSim(w).init_particles()
    _run_phases(s, [PH_STREAM, PH_RESERVOIR, PH_SORT, PH_MOMENTS, PH_PARAMS])
    prm = s.params()[0]
    theta = prm[3]
    T = theta / KB_M
    N = s.counts()[0]
    nu_expected_ref = 0.8 * 0.7 / s.dt
    scale = (N / 2000.0) * (T / W.T0) ** (1.0 - 0.5)
    assert math.isclose(prm[11], nu_expected_ref * scale, rel_tol=1e-12)
    assert math.isclose(prm[12], W.PR_MONO * prm[11], rel_tol=1e-14)
    assert math.isclose(prm[10], 1.0 - math.exp(-prm[12] * s.dt), rel_tol=1e-12)


def _stress_heat(v):
    u = v.mean(axis=0)
    C = v - u
    cov = C.T @ C / len(v)
    theta = np.trace(cov) / 3.0
    sig = cov - theta * np.eye(3)
    q = 0.5 * ((C ** 2).sum(1)[:, None] * C).mean(0)
    return sig, q, theta


@pytest.mark.parametrize("mode", ["usp", "sp"])
def test_homogeneous_relaxation_closed_form(mode):
    """One relaxation step of an anisotropic homogeneous gas.  With no gradients
    Kn_GLL = 0 and P_ne = 1 (USP); in SP mode P_ne = 0.  Unrelaxed particles keep
    their stress; relaxed ones carry (1 - 1/Pr) s sigma*, s from Eq. 32 averaged
    over g_time (Eqs. 29-30), sigma* from Eq. 33:
        E[sigma'] = sigma [e^-a + (1 - e^-a)(1 - 1/Pr) kappa],  a = nu_ES dt,
        USP: kappa = 1 / (1 + nu dt / 2)
        SP : kappa = E[e^(-nu t)] = a (e^((nu_ES - nu) dt) - 1) / ((nu_ES - nu) dt (e^a - 1))."""
    n = 1_000_000
    w = W.homogeneous_box(ppc=n, dt_over_tauc=5.0, mode=mode)
    pos, vel, pid = W.bimaxwellian(n, seed=21)
    s = oracle.OracleSim(w).set_particles(pos, vel, pid)
    _run_phases(s, [PH_STREAM, PH_RESERVOIR, PH_SORT, PH_MOMENTS, PH_PARAMS])
    prm = s.params()[0]
    sig0, _, theta = _stress_heat(s.particles()["vel"])
    assert prm[13] == (1.0 if mode == "usp" else 0.0)
    s.phase(PH_RELAX)
    sig1, _, _ = _stress_heat(s.particles()["vel"])
    nu, nu_es, dt = prm[11], prm[12], s.dt
    a = nu_es * dt
    if mode == "usp":
        kappa = 1.0 / (1.0 + 0.5 * nu * dt)
    else:
        d = (nu_es - nu) * dt
        kappa = a * math.expm1(d) / (d * math.expm1(a))
    r = math.exp(-a) + (1 - math.exp(-a)) * (1 - 1 / W.PR_MONO) * kappa
    se = theta * math.sqrt(2.0 / n)
    for i in range(3):
        assert abs(sig1[i, i] - r * sig0[i, i]) < 4 * se, (i, sig1[i, i], r * sig0[i, i], se)


def test_heat_flux_decays_at_nu_es():
    """Relaxed particles are Gaussian (no heat flux), unrelaxed ones keep theirs:
    E[q'] = e^(-nu_ES dt) q (Eq. 8b)."""
    n = 1_000_000
    w = W.homogeneous_box(ppc=n, dt_over_tauc=1.5)
    pos, vel, pid = W.bimaxwellian(n, seed=5, heat_skew=1.0)
    s = oracle.OracleSim(w).set_particles(pos, vel, pid)
    _run_phases(s, [PH_STREAM, PH_RESERVOIR, PH_SORT, PH_MOMENTS, PH_PARAMS])
    prm = s.params()[0]
    v0 = s.particles()["vel"]
    _, q0, theta = _stress_heat(v0)
    s.phase(PH_RELAX)
    _, q1, _ = _stress_heat(s.particles()["vel"])
    r = math.exp(-prm[12] * s.dt)
    se = math.sqrt(np.var(0.5 * ((v0 - v0.mean(0)) ** 2).sum(1) * (v0[:, 1] - v0[:, 1].mean())) / n)
    assert abs(q0[1]) > 20 * se
    assert abs(q1[1] - r * q0[1]) < 5 * se
    r_wrong = math.exp(-prm[11] * s.dt)
    assert abs(q1[1] - r_wrong * q0[1]) > 4 * se


def test_maxwellian_is_preserved():
    """sigma = 0, q = 0 make f_G the Maxwellian (Eqs. 5-6): after many large steps
    the velocities stay N(u, RT) and the temperature is exactly conserved."""
    n = 200_000
    w = W.homogeneous_box(ppc=n, dt_over_tauc=5.0)
    pos, vel, pid = W.bimaxwellian(n, T=(W.T0,) * 3, u=(30.0, -10.0, 5.0), seed=9)
    s = oracle.OracleSim(w).set_particles(pos, vel, pid)
    s.step(20)
    v = s.particles()["vel"]
    assert np.allclose(v.mean(0), vel.mean(0), rtol=0, atol=1e-9)
    assert math.isclose(((v - v.mean(0)) ** 2).sum(), ((vel - vel.mean(0)) ** 2).sum(), rel_tol=1e-12)
    th = ((v - v.mean(0)) ** 2).sum() / (3 * n)
    for d in range(3):
        z = (v[:, d] - v[:, d].mean()) / math.sqrt(th)
        assert stats.kstest(z, "norm").pvalue > 1e-3
        assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 4 * math.sqrt(24.0 / n)


def test_bgk_special_case_and_cholesky_consistency():
    """Pr = 1 turns the ES Gaussian into the Maxwellian: L = sqrt(RT) I.  For any
    Pr the factor satisfies L L^T = RT I + (1 - 1/Pr) sigma*/rho, with sigma* the
    stress that the sampled pressure tensor reports."""
    n = 50_000
    pos, vel, pid = W.bimaxwellian(n, seed=4)
    w = W.homogeneous_box(ppc=n, Pr=1.0)
    s = oracle.OracleSim(w).set_particles(pos, vel, pid)
    s.step(1)
    prm = s.params()[0]
    r = math.sqrt(prm[3])
    assert np.allclose(prm[4:10], [r, 0, r, 0, 0, r], rtol=1e-15, atol=0)

    w = W.homogeneous_box(ppc=n)
    s = oracle.OracleSim(w).set_particles(pos, vel, pid)
    s.step(1)
    prm = s.params()[0]
    F = s.fields()[:, 0]
    L = np.zeros((3, 3))
    L[0, 0], L[1, 0], L[1, 1], L[2, 0], L[2, 1], L[2, 2] = prm[4:10]
    rho = F[0] * W.M_AR
    p = rho * prm[3]
    S = np.array([[F[5] - p, F[8], F[9]], [F[8], F[6] - p, F[10]], [F[9], F[10], F[7] - p]]) / rho
    A = prm[3] * np.eye(3) + (1 - 1 / W.PR_MONO) * S
    assert np.allclose(L @ L.T, A, rtol=1e-12, atol=1e-12 * prm[3])


def test_gll_knudsen_linear_density_profile():
    """Eq. 18 on a linear density profile with uniform temperature and zero
    velocity: the central (and one-sided) differences are exact, so
    Kn_GLL = lambda * slope / n in every cell and P_ne = exp(-Kn_GLL / 0.1)."""
    ny = 12
    w = W.sod(ny=ny, ppc_left=1000, Kn=0.02, precision="fp64")
    H = w["grid"]["hi"][1]
    dy = H / ny
    counts = 400 + 60 * np.arange(ny)
    rng = np.random.default_rng(8)
    pos, vel = [], []
    for c, m in enumerate(counts):
        half = rng.normal(0, 1, (m // 2, 3))
        half /= np.sqrt((half ** 2).sum() / (3 * (m // 2)))        # exact unit temperature
        v = np.empty((m, 3))
        v[0::2], v[1::2] = half, -half                             # exact zero mean, pairs adjacent
        vel.append(v * math.sqrt(KB_M * W.T0))
        pos.append(np.column_stack([np.zeros(m), (c + 0.5) * dy + np.zeros(m)]))
    pos, vel = np.vstack(pos), np.vstack(vel)
    s = oracle.OracleSim(w).set_particles(pos, vel, np.arange(len(pos), dtype=np.uint32))
    _run_phases(s, [PH_SORT, PH_MOMENTS, PH_PARAMS])
    prm = s.params()
    cbar = math.sqrt(8 * KB_M * W.T0 / math.pi)
    for c in range(ny):
        lam = 0.8 * cbar / prm[c, 11]           # lambda = tau_c * cbar, nu tau_c = 0.8
        kn = lam * (60.0 / dy) / counts[c]
        assert math.isclose(prm[c, 13], math.exp(-kn / 0.1), rel_tol=1e-9), c


def test_exponential_average_eq34():
    w = W.couette(ny=10, ppc=30, precision="fp64")
    w["params"]["n_avg"] = 7
    s = oracle.OracleSim(w).init_particles()
    acc = None
    for k in range(12):
        s.step(1)
        inst = s.fields()
        acc = inst.copy() if acc is None else (6.0 / 7.0) * acc + inst / 7.0
    assert np.allclose(s.fields(averaged=True), acc, rtol=1e-13, atol=1e-300)
