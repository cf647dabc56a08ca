"""Pins of the oracle's weighted added particles (Table 2 steps 2, 4, 7;
Eqs. 22-28 and the third term of Eq. 27).

What the paper and the mathematics fix:

* one step of a homogeneous gas with P_ne = 1: step 2 gives the streamed
  distribution the stress sigma^n (1 - x/2) (J removes stress at nu), Eq. 33
  divides it by 1 + x/2, and the three terms of Eq. 27 add back up to
  sigma* (e^-a from the unselected particles, (1 - e^-a)(1 - 1/Pr) from
  f_G, (1 - e^-a)/Pr from step 7), so sigma^{n+1} = sigma^n (1 - x/2) /
  (1 + x/2), x = nu dt, the trapezoidal (Crank-Nicolson) decay of Eq. 20;
  likewise q^{n+1} = q^n (1 - x Pr/2) / (1 + x Pr/2).  The scheme without
  the added particles gives sigma*/sigma^n = 1 / (1 + x/2) instead (opposite
  sign at x = 4);
* every weight 1 and P_ne = 0: nothing is added (Eq. 26 vanishes) and the
  step is the plain one;
* mass, momentum and energy are kept in expectation (the weights of
  Eq. 26 have zero mean, momentum and energy moments against the
  Maxwellian, and Eq. 28 keeps the selected weight up to its rounding);
* steady Couette shear at x = 4: the same three terms make sigma* = -mu du/dy
  for every x (the moment balance sigma*(1 + x/2) = sigma*(1 - x/2) - p du/dy
  dt), so the viscosity ratio is 1, where the split scheme gives 1.23;
  meanwhile the population stays bounded.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1808_03801_gb300 import workloads as W

KB_M = 1.380649e-23 / W.M_AR
PR = 2.0 / 3.0


def _box(n, weighted=True, mode="fixed", pne=1.0, dt_over_tauc=5.0, r_p=1.0):
    w = W.homogeneous_box(ppc=n, dt_over_tauc=dt_over_tauc, mode=mode, fixed_pne=pne)
    w["params"]["weighted"] = int(weighted)
    w["params"]["r_p"] = r_p
    return w


def _stress_heat(P):
    v, wt = P["vel"], P["w"]
    m = wt.sum()
    u = (wt[:, None] * v).sum(0) / m
    C = v - u
    th = (wt * (C ** 2).sum(1)).sum() / (3 * m)
    sxx = (wt * C[:, 0] ** 2).sum() / m - th
    qy = 0.5 * (wt * (C ** 2).sum(1) * C[:, 1]).sum() / m
    return sxx, qy, th


def _sampled(o):
    """sigma*_xx and q*_y per unit density from the sampled fields (Eq. 33)."""
    F = o.fields()[:, 0]
    rho = F[0] * W.M_AR
    p = rho * KB_M * F[4]
    return (F[5] - p) / rho, F[12] / rho, o.params()[0, 11] * o.dt


def _mean_se(v):
    v = np.asarray(v)
    return v.mean(), v.std(ddof=1) / math.sqrt(len(v))


def test_homogeneous_step_is_crank_nicolson():
    """Twelve independent runs (initial state and the scheme's own random
    numbers both seeded apart) of 100 000 particles, r_p = 1, nu dt near 4:
    sigma*/sigma^n and q*/q^n average to the trapezoidal factors within four
    standard errors, far from the split scheme's 1/(1 + x/2) and
    1/(1 + x Pr/2); one step later sigma* is the trapezoidal factor times
    the last one (the relaxation returned sigma^{n+1} = sigma*)."""
    n, T0 = 100_000, W.T0
    d_s, d_q, d_s2, split_s, split_q = [], [], [], [], []
    for seed in range(12):
        pos, vel, pid = W.bimaxwellian(n, T=(1.6 * T0, 0.7 * T0, 0.7 * T0), seed=seed, heat_skew=0.5)
        o = oracle.OracleSim(_box(n)).set_particles(pos, vel, pid, seed=1000 + seed)
        s0, q0, _ = _stress_heat(o.particles())
        o.step(1)
        s1, q1, x = _sampled(o)
        assert 3.5 < x < 4.5
        cn_s = (1 - x / 2) / (1 + x / 2)
        cn_q = (1 - x * PR / 2) / (1 + x * PR / 2)
        d_s.append((s1 - cn_s * s0) / abs(s0))
        d_q.append((q1 - cn_q * q0) / abs(q0))
        split_s.append((s1 - s0 / (1 + x / 2)) / abs(s0))
        split_q.append((q1 - q0 / (1 + x * PR / 2)) / abs(q0))
        o.step(1)
        s2, _, x2 = _sampled(o)
        d_s2.append((s2 - (1 - x2 / 2) / (1 + x2 / 2) * s1) / abs(s0))
    for d in (d_s, d_q, d_s2):
        m, se = _mean_se(d)
        assert abs(m) < 4 * se + 1e-3, (m, se)
        assert se < 0.03, se
    for d in (split_s, split_q):
        m, se = _mean_se(d)
        assert abs(m) > 20 * se, (m, se)


def test_weights_one_and_no_pne_is_the_plain_step():
    n = 20_000
    pos, vel, pid = W.bimaxwellian(n, seed=3)
    a = oracle.OracleSim(_box(n, weighted=True, mode="sp")).set_particles(pos, vel, pid)
    b = oracle.OracleSim(_box(n, weighted=False, mode="sp")).set_particles(pos, vel, pid)
    a.step(3)
    b.step(3)
    A, B = a.particles(), b.particles()
    assert a.n == b.n == n
    assert np.all(A["w"] == 1.0)
    oa, ob = np.argsort(A["pid"]), np.argsort(B["pid"])
    assert np.array_equal(A["pid"][oa], B["pid"][ob])
    sc = math.sqrt(KB_M * W.T0)
    assert np.allclose(A["vel"][oa], B["vel"][ob], rtol=0, atol=1e-10 * sc)


def test_mass_momentum_energy_kept_in_expectation():
    """Eq. 26 weights have zero mean, zero first moments and zero energy
    moment over the Maxwellian they are drawn from (sigma is traceless; the
    heat-flux term vanishes against 1 and C^2 by symmetry and against C
    because <C_i C_k C^2> = 5 theta^2 delta_ik), and Eq. 28 keeps the
    selected weight up to its rounding; so over twelve independent runs of
    four steps the change of mass, momentum and energy averages to zero
    within four standard errors, while the added particles do move each run
    (weights present)."""
    n = 50_000
    dm, dp, de = [], [], []
    for seed in range(12):
        pos, vel, pid = W.bimaxwellian(n, seed=50 + seed, u=(50.0, -20.0, 10.0), heat_skew=0.5)
        o = oracle.OracleSim(_box(n)).set_particles(pos, vel, pid, seed=2000 + seed)
        P = o.particles()
        m0 = P["w"].sum()
        p0 = (P["w"][:, None] * P["vel"]).sum(0)
        e0 = (P["w"] * (P["vel"] ** 2).sum(1)).sum()
        o.step(4)
        P = o.particles()
        assert np.any(P["w"] != 1.0)
        sc = math.sqrt(KB_M * W.T0)
        dm.append((P["w"].sum() - m0) / m0)
        dp.append(((P["w"][:, None] * P["vel"]).sum(0) - p0) / (m0 * sc))
        de.append(((P["w"] * (P["vel"] ** 2).sum(1)).sum() - e0) / e0)
    for d in [dm, de] + list(np.array(dp).T):
        m, se = _mean_se(d)
        assert abs(m) < 4 * se + 1e-12, (m, se)
        assert se > 0


@pytest.mark.slow
def test_couette_viscosity_independent_of_dt():
    """Steady Couette (Kn = 0.01, 50 cells, 300 per cell, P_ne = 1, x = 4):
    with the weighted particles the sampled shear stress over mu du/dy is 1,
    not the split scheme's 1.23; the weights use Eq. 34 averages (n_a = 100)
    of their fields.  The population stays within 30 % of its start."""
    ny, ppc = 50, 300
    w = W.couette(ny=ny, ppc=ppc, Kn=0.01, u_wall=20.0, dt_over_tauc=5.0, omega=0.81, seed=4)
    w["params"].update(mode="fixed", fixed_pne=1.0, weighted=1, weight_average=1, n_avg=100)
    o = oracle.OracleSim(w).init_particles()
    n0 = o.n
    H = w["grid"]["hi"][1]
    y = (np.arange(ny) + 0.5) * H / ny
    c = slice(int(0.2 * ny), int(0.8 * ny))
    counts = []
    for _ in range(15):
        o.step(100)
        counts.append(o.n)
    ratios = []
    for _ in range(10):
        acc = np.zeros((16, ny))
        for _ in range(200):
            o.step(1)
            acc += o.fields()
        counts.append(o.n)
        F = acc / 200
        mu = o.mu_ref * (F[4][c].mean() / W.T0) ** 0.81
        slope = np.polyfit(y[c], F[1][c], 1)[0]
        ratios.append(-F[8][c].mean() / (mu * slope))
    r = np.array(ratios)
    m, se = r.mean(), r.std(ddof=1) / math.sqrt(len(r))
    assert abs(m - 1.0) < 4 * se + 0.04, (m, se)
    assert abs(m - 1.23) > 4 * se + 0.05, (m, se)
    assert max(counts) < 1.3 * n0 and min(counts) > n0, (n0, min(counts), max(counts))


@pytest.mark.slow
def test_thermal_couette_conductivity_independent_of_dt():
    """Steady thermal Couette (plates at T0 -/+ 50 K, Kn = 0.01, 50 cells,
    300 per cell, P_ne = 1, x = nu dt near 4): with the weighted particles
    the sampled heat flux over kappa dT/dy (kappa = 15/4 k/m mu) is 1 -- the
    moment balance of the heat flux, with Pr in Eq. 33 and in J, gives kappa
    at every x -- where the split scheme gives (2/3) x / (1 - e^{-Pr x}) /
    (1 + x Pr / 2) = 1.23."""
    ny, ppc = 50, 300
    w = W.couette(ny=ny, ppc=ppc, Kn=0.01, u_wall=0.0, dt_over_tauc=5.0, omega=0.81, seed=8)
    w["faces"][2]["T"] = W.T0 + 50.0
    w["faces"][3]["T"] = W.T0 - 50.0
    w["params"].update(mode="fixed", fixed_pne=1.0, weighted=1, weight_average=1, n_avg=100)
    o = oracle.OracleSim(w).init_particles()
    n0 = o.n
    H = w["grid"]["hi"][1]
    y = (np.arange(ny) + 0.5) * H / ny
    c = slice(int(0.2 * ny), int(0.8 * ny))
    counts = []
    for _ in range(15):
        o.step(100)
        counts.append(o.n)
    ratios, xs = [], []
    for _ in range(10):
        acc = np.zeros((16, ny))
        for _ in range(200):
            o.step(1)
            acc += o.fields()
        counts.append(o.n)
        xs.append(o.params()[c, 11].mean() * o.dt)
        F = acc / 200
        kappa = 15.0 / 4.0 * KB_M * o.mu_ref * (F[4][c].mean() / W.T0) ** 0.81
        ratios.append(-F[12][c].mean() / (kappa * np.polyfit(y[c], F[4][c], 1)[0]))
    m, se = _mean_se(ratios)
    x = float(np.mean(xs))
    split = (2.0 / 3.0) * x / (1.0 - math.exp(-PR * x)) / (1.0 + x * PR / 2.0)
    assert 3.0 < x < 5.5, x
    assert abs(m - 1.0) < 4 * se + 0.02, (m, se)
    assert abs(m - split) > 4 * se + 0.05, (m, se, split)
    assert max(counts) < 1.3 * n0 and min(counts) > n0, (n0, min(counts), max(counts))
