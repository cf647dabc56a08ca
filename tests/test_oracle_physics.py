"""Physics pins of the whole oracle step at small Knudsen number.

* Sod shock tube (Sec. 4.3): at Kn = 1e-4 the gas is in the continuum limit
  and the density, velocity and temperature profiles must approach the exact
  solution of the Euler Riemann problem for a monatomic gas (gamma = 5/3),
  computed here with the textbook exact solver (pressure star by root
  finding, then the wave pattern).
* Couette flow (Sec. 4.1): momentum balance makes the steady shear stress
  uniform across the gap, and the velocity profile is antisymmetric.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_1808_03801_gb300 import workloads as W

KB_M = 1.380649e-23 / W.M_AR
GAMMA = 5.0 / 3.0


def exact_riemann(rl, ul, pl, rr, ur, pr, x, t, x0=0.5, g=GAMMA):
    """Exact solution of the 1-D Euler Riemann problem (ideal gas)."""
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)

    def f(p, rk, pk, ck):
        if p > pk:
            A, B = 2 / ((g + 1) * rk), (g - 1) / (g + 1) * pk
            return (p - pk) * math.sqrt(A / (p + B))
        return 2 * ck / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)

    ps = brentq(lambda p: f(p, rl, pl, cl) + f(p, rr, pr, cr) + ur - ul, 1e-8, 10 * max(pl, pr))
    us = 0.5 * (ul + ur) + 0.5 * (f(ps, rr, pr, cr) - f(ps, rl, pl, cl))
    rho = np.empty_like(x)
    u = np.empty_like(x)
    p = np.empty_like(x)
    for i, xi in enumerate(x):
        s = (xi - x0) / t
        if s < us:  # left of contact
            if ps <= pl:  # left rarefaction
                shl = ul - cl
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - cs
                if s < shl:
                    r, v, pp = rl, ul, pl
                elif s > stl:
                    r, v, pp = rl * (ps / pl) ** (1 / g), us, ps
                else:
                    v = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    r = rl * (c / cl) ** (2 / (g - 1))
                    pp = pl * (c / cl) ** (2 * g / (g - 1))
            else:
                raise NotImplementedError
        else:  # right of contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s > sr:
                    r, v, pp = rr, ur, pr
                else:
                    r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                    v, pp = us, ps
            else:
                raise NotImplementedError
        rho[i], u[i], p[i] = r, v, pp
    return rho, u, p, ps, us


def test_exact_riemann_solver_sod_values():
    """The solver reproduces the well-known star state of Sod's problem for gamma = 1.4."""
    _, _, _, ps, us = exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, np.array([0.5]), 0.2, g=1.4)
    assert math.isclose(ps, 0.30313, rel_tol=1e-4)
    assert math.isclose(us, 0.92745, rel_tol=1e-4)


@pytest.mark.slow
def test_sod_continuum_limit_matches_euler():
    ny, ppc = 200, 800
    w = W.sod(ny=ny, ppc_left=ppc, precision="fp64")
    s = oracle.OracleSim(w).init_particles()
    theta_l = KB_M * W.T0
    t_norm = 0.15
    t_phys = t_norm * 1.0 / math.sqrt(theta_l)
    nsteps = int(round(t_phys / s.dt))
    s.step(nsteps)
    t_norm = nsteps * s.dt * math.sqrt(theta_l)
    F = s.fields()
    y = (np.arange(ny) + 0.5) / ny
    rho = F[0] / W.N0
    u = F[2] / math.sqrt(theta_l)
    T = F[4] / W.T0
    r_ex, u_ex, p_ex, ps, us = exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, y, t_norm)
    T_ex = p_ex / r_ex
    # block averages of 5 cells reduce particle noise; compare L1 errors
    def blk(a):
        return a.reshape(-1, 5).mean(1)
    e_rho = np.abs(blk(rho) - blk(r_ex)).mean() / 1.0
    e_u = np.abs(blk(u) - blk(u_ex)).mean() / max(u_ex)
    e_T = np.abs(blk(T) - blk(T_ex)).mean() / max(T_ex)
    assert e_rho < 0.03 and e_u < 0.05 and e_T < 0.03, (e_rho, e_u, e_T)
    # mass is conserved exactly with specular ends
    assert s.n == int(ny / 2 * ppc + ny / 2 * ppc / 8)
    # plateau between contact and shock carries the star velocity and pressure
    sel = (y > 0.5 + (us + 0.1) * t_norm) & (y < 0.5 + (us + 0.55) * t_norm)
    assert sel.sum() >= 4
    assert abs(u[sel].mean() - us) < 0.05 * us
    assert abs((rho * T)[sel].mean() - ps) < 0.05 * ps


@pytest.mark.slow
def test_couette_steady_shear_uniform_and_antisymmetric():
    ny = 40
    w = W.couette(ny=ny, ppc=100, Kn=0.1, precision="fp64")
    s = oracle.OracleSim(w).init_particles()
    s.step(400)
    acc = []
    for k in range(30):
        blk = np.zeros((16, ny))
        for j in range(40):
            s.step(1)
            blk += s.fields()
        acc.append(blk / 40)
    acc = np.array(acc)
    mean = acc.mean(0)
    se = acc.std(0, ddof=1) / math.sqrt(len(acc))
    pxy, ux = mean[8], mean[1]
    # antisymmetry of u_x about the mid plane
    d = ux + ux[::-1]
    sd = np.sqrt(se[1] ** 2 + se[1][::-1] ** 2)
    assert np.all(np.abs(d) < 4 * sd + 1e-9)
    # uniform shear stress: slope of a linear fit consistent with zero, and each
    # cell within 4 standard errors of the gap average
    y = np.arange(ny) - (ny - 1) / 2
    slope = np.polyfit(y, pxy, 1)[0]
    avg = pxy.mean()
    assert avg < 0
    assert abs(slope * ny) < 0.1 * abs(avg)
    assert np.all(np.abs(pxy - avg) < 4 * se[8] + 0.02 * abs(avg))


def _couette_sampled_stress_ratio(mode, fixed_pne=0.0, r=5.0, ny=50, ppc=300, relax_steps=1500, blocks=10,
                                  block_steps=250, u_wall=100.0):
    """Steady Couette (plates at -/+ u_wall, Kn = 0.01): mean and standard
    error over time blocks of -p_xy / (mu du/dy) in the central 60 % of the
    gap, and x = nu dt at the bulk state."""
    w = W.couette(ny=ny, ppc=ppc, Kn=0.01, u_wall=u_wall, dt_over_tauc=r, omega=0.81, seed=7)
    w["params"]["mode"] = mode
    w["params"]["fixed_pne"] = fixed_pne
    o = oracle.OracleSim(w).init_particles()
    o.step(relax_steps)
    H = w["grid"]["hi"][1]
    y = (np.arange(ny) + 0.5) * H / ny
    c = slice(int(0.2 * ny), int(0.8 * ny))
    ratios, xs = [], []
    for _ in range(blocks):
        acc = np.zeros((16, ny))
        nu = 0.0
        for _ in range(block_steps):
            o.step(1)
            acc += o.fields()
            nu += o.params()[c, 11].mean()
        F = acc / block_steps
        T = F[4][c].mean()
        mu = o.mu_ref * (T / W.T0) ** 0.81
        slope = np.polyfit(y[c], F[1][c], 1)[0]
        ratios.append(-F[8][c].mean() / (mu * slope))
        xs.append(nu / block_steps * o.dt)
    ratios = np.array(ratios)
    return ratios.mean(), ratios.std(ddof=1) / math.sqrt(blocks), float(np.mean(xs))


def test_couette_sampled_stress_matches_splitting_closed_form():
    """Streaming and relaxation alternate, so in steady shear the stress
    sampled after a flight, sigma', obeys sigma'(1 - R) = -p gamma dt, with R
    the fraction of stress one relaxation leaves (selection probability
    1 - e^-a, a = nu_ES dt, Eq. 9; target stress (1 - 1/Pr) times sigma(t) of
    Eq. 32).  P_ne = 0: sigma(t) = e^{-nu t} sigma' with t drawn from g_time
    (Eqs. 29-30), so R = e^-a + (1 - e^-a)(1 - 1/Pr) E[e^{-nu t}] and the
    sampled ratio is x / (1 - R), x = nu dt.  P_ne = 1: sigma(t) = sigma* =
    sigma' / (1 + x/2) (Eq. 33), R = e^-a + (1 - e^-a)(1 - 1/Pr) / (1 + x/2),
    and the sampled sigma* gives x / ((1 - R)(1 + x/2)).  A wrong factor in
    Eq. 33 (e.g. Pr on the stress), the selection rate or the sampling point
    moves these by more than the tolerance."""
    Pr = 2.0 / 3.0
    m_sp, se_sp, x = _couette_sampled_stress_ratio("sp")
    a = Pr * x
    nes = Pr
    k_sp = nes / (nes - 1.0) * (math.exp((nes - 1.0) * x) - 1.0) / (math.exp(a) - 1.0)   # E[e^{-nu t}]
    R_sp = math.exp(-a) + (1 - math.exp(-a)) * (1 - 1 / Pr) * k_sp
    want_sp = x / (1 - R_sp)
    assert abs(m_sp - want_sp) < 4 * se_sp + 0.01 * want_sp, (m_sp, se_sp, want_sp)
    m_u, se_u, x = _couette_sampled_stress_ratio("fixed", fixed_pne=1.0)
    a = Pr * x
    R_u = math.exp(-a) + (1 - math.exp(-a)) * (1 - 1 / Pr) / (1 + x / 2)
    want_u = x / ((1 - R_u) * (1 + x / 2))
    assert abs(m_u - want_u) < 4 * se_u + 0.01 * want_u, (m_u, se_u, want_u)
    assert want_sp / want_u > 3.0   # the Eq. 33 correction is what separates them


def _thermal_couette_heat_ratio(mode, fixed_pne=0.0, r=5.0, ny=50, ppc=300, relax_steps=1500, blocks=10,
                                block_steps=250, dT=50.0):
    """Steady thermal Couette (plates at T0 +/- dT, Kn = 0.01): mean and
    standard error over time blocks of -q_y / (kappa dT/dy) in the central
    60 % of the gap (kappa = 15/4 k/m mu(T)), and x = nu dt in the bulk."""
    w = W.couette(ny=ny, ppc=ppc, Kn=0.01, u_wall=0.0, dt_over_tauc=r, omega=0.81, seed=8)
    w["faces"][2]["T"] = W.T0 + dT
    w["faces"][3]["T"] = W.T0 - dT
    w["params"]["mode"] = mode
    w["params"]["fixed_pne"] = fixed_pne
    o = oracle.OracleSim(w).init_particles()
    o.step(relax_steps)
    H = w["grid"]["hi"][1]
    y = (np.arange(ny) + 0.5) * H / ny
    c = slice(int(0.2 * ny), int(0.8 * ny))
    ratios, xs = [], []
    for _ in range(blocks):
        acc = np.zeros((16, ny))
        nu = 0.0
        for _ in range(block_steps):
            o.step(1)
            acc += o.fields()
            nu += o.params()[c, 11].mean()
        F = acc / block_steps
        T = F[4][c].mean()
        kappa = 15.0 / 4.0 * KB_M * o.mu_ref * (T / W.T0) ** 0.81
        slope = np.polyfit(y[c], F[4][c], 1)[0]
        ratios.append(-F[12][c].mean() / (kappa * slope))
        xs.append(nu / block_steps * o.dt)
    ratios = np.array(ratios)
    return ratios.mean(), ratios.std(ddof=1) / math.sqrt(blocks), float(np.mean(xs))


def test_thermal_couette_heat_flux_matches_splitting_closed_form():
    """In a temperature gradient a free flight builds heat flux at
    -(5/2)(k/m) p dT/dy per unit time and a relaxation leaves e^-a of it
    (relaxed particles are Gaussian, Eq. 8b; a = nu_ES dt), so the heat flux
    sampled after a flight is (5/2)(k/m) p dt / (1 - e^-a) times -dT/dy: over
    kappa = (15/4)(k/m) mu that is (2/3) x / (1 - e^-a) with x = nu dt.
    USP samples q* = that / (1 + x Pr / 2) (Eq. 33 with P_ne = 1).  A heat
    flux corrected without Pr, or relaxed at nu instead of nu_ES, misses."""
    Pr = 2.0 / 3.0
    m_sp, se_sp, x = _thermal_couette_heat_ratio("sp")
    want_sp = (2.0 / 3.0) * x / (1.0 - math.exp(-Pr * x))
    assert abs(m_sp - want_sp) < 4 * se_sp + 0.03 * want_sp, (m_sp, se_sp, want_sp)
    m_u, se_u, x = _thermal_couette_heat_ratio("fixed", fixed_pne=1.0)
    want_u = (2.0 / 3.0) * x / (1.0 - math.exp(-Pr * x)) / (1.0 + x * Pr / 2.0)
    assert abs(m_u - want_u) < 4 * se_u + 0.03 * want_u, (m_u, se_u, want_u)
    wrong = (2.0 / 3.0) * x / (1.0 - math.exp(-Pr * x)) / (1.0 + x / 2.0)   # no Pr in the q* factor
    assert abs(m_u - wrong) > 4 * se_u + 0.03 * want_u
