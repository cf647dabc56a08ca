"""Pins of every branch of the gradient-length local Knudsen number (Eqs. 16-18).

Each case builds a state whose per-cell moments are exact by construction
(a zero-mean, unit-temperature velocity set scaled and shifted per cell) and
whose fields are linear across cells, so that the central and one-sided
differences of the stencil are exact.  The expected P_ne is then written out
from the definitions, independently of the oracle:

    lambda = 16 / (5 sqrt(2 pi)) mu / sqrt(rho p)        Eq. 36
    mu     = mu_ref (T / T_ref)^omega                     Eq. 35
    Kn_Q   = lambda |grad Q| / Q                          Eq. 18, Q = rho, T
    Kn_u   = lambda |grad |u|| / max(|u|, sqrt(gamma R T)) Eq. 18, Q = |u|
    Kn     = max(Kn_rho, Kn_T, Kn_u)                      Eq. 17
    P_ne   = exp(-Kn / 0.1)                               Eq. 16

|grad Q| is the Euclidean norm over the resolved axes.  A swapped
normalisation (the T gradient divided by n, |grad |u|| divided by |u| alone
or by the sound speed alone), a sum instead of the maximum, or a sum of
absolute components instead of the norm each fails one of these cases.
"""
import math

import numpy as np

import oracle
from oracle import PH_MOMENTS, PH_PARAMS, PH_SORT
from paper_1808_03801_gb300 import workloads as W

KB = 1.380649e-23
R = KB / W.M_AR
GAMMA = 5.0 / 3.0


def _unit_set(m, rng):
    """m velocities (m even) with exactly zero mean and sum |v|^2 / (3 m) = 1."""
    half = rng.normal(0, 1, (m // 2, 3))
    half /= np.sqrt((half ** 2).sum() / (3 * (m // 2)))
    v = np.empty((m, 3))
    v[0::2], v[1::2] = half, -half
    return v


def _state(centres, counts, thetas, us, seed=8):
    """Particles at the given cell centres: cell k holds counts[k] particles
    with mean velocity us[k] and temperature thetas[k] / R (exact moments)."""
    rng = np.random.default_rng(seed)
    pos, vel = [], []
    for (x, y), m, th, u in zip(centres, counts, thetas, us):
        vel.append(np.asarray(u)[None, :] + math.sqrt(th) * _unit_set(int(m), rng))
        pos.append(np.column_stack([np.full(m, x), np.full(m, y)]))
    pos, vel = np.vstack(pos), np.vstack(vel)
    return pos, vel, np.arange(len(pos), dtype=np.uint32)


def _pne_of(w, pos, vel, pid):
    s = oracle.OracleSim(w).set_particles(pos, vel, pid)
    for ph in (PH_SORT, PH_MOMENTS, PH_PARAMS):
        s.phase(ph)
    return s, s.params()[:, 13]


def _lambda(mu_ref, omega, n, theta):
    T = theta / R
    mu = mu_ref * (T / W.T0) ** omega
    rho = n * W.M_AR
    return 16.0 / (5.0 * math.sqrt(2.0 * math.pi)) * mu / math.sqrt(rho * rho * theta)


def _grad_1d(q, h):
    """Exact derivative of a linear profile: central inside, one-sided at the ends."""
    g = np.empty_like(q)
    g[1:-1] = (q[2:] - q[:-2]) / (2 * h)
    g[0] = (q[1] - q[0]) / h
    g[-1] = (q[-1] - q[-2]) / h
    return g


def _tube(ny=12, Kn=0.02):
    w = W.sod(ny=ny, ppc_left=600, Kn=Kn, precision="fp64")
    H = w["grid"]["hi"][1]
    dy = H / ny
    centres = [(0.0, (c + 0.5) * dy) for c in range(ny)]
    return w, dy, centres


def _n_of(counts, w):
    return np.asarray(counts, dtype=float) * w["params"]["n_ref"] / w["params"]["ppc_ref"]


def test_temperature_branch_linear_T():
    """Uniform n, zero u, T linear across the tube: Kn_GLL = lambda |dT/dy| / T."""
    ny = 12
    w, dy, centres = _tube(ny)
    th0 = R * W.T0
    counts = np.full(ny, 600)
    thetas = th0 * (1.0 + 0.08 * np.arange(ny))
    pos, vel, pid = _state(centres, counts, thetas, [(0.0, 0.0, 0.0)] * ny)
    s, pne = _pne_of(w, pos, vel, pid)
    n = _n_of(counts, w)
    T = thetas / R
    gT = np.abs(_grad_1d(T, dy))
    for c in range(ny):
        kn = _lambda(s.mu_ref, w["gas"]["omega"], n[c], thetas[c]) * gT[c] / T[c]
        assert 0.005 < kn < 0.1
        assert math.isclose(pne[c], math.exp(-kn / 0.1), rel_tol=1e-9), (c, pne[c], math.exp(-kn / 0.1))


def _velocity_case(u0, du):
    ny = 12
    w, dy, centres = _tube(ny)
    th0 = R * W.T0
    counts = np.full(ny, 600)
    ux = u0 + du * np.arange(ny)
    pos, vel, pid = _state(centres, counts, np.full(ny, th0), [(u, 0.0, 0.0) for u in ux])
    s, pne = _pne_of(w, pos, vel, pid)
    n = _n_of(counts, w)
    gu = np.abs(_grad_1d(ux, dy))
    a = math.sqrt(GAMMA * th0)
    lam = _lambda(s.mu_ref, w["gas"]["omega"], n[0], th0)
    return pne, ux, gu, a, lam


def test_velocity_branch_subsonic_uses_sound_speed():
    """Uniform n and T, u_x linear with |u| below sqrt(gamma R T): the |u| branch
    is normalised by the sound speed, Kn = lambda |d|u|/dy| / sqrt(gamma R T)."""
    pne, ux, gu, a, lam = _velocity_case(20.0, 15.0)
    assert ux.max() < a
    for c in range(len(ux)):
        kn = lam * gu[c] / a
        assert math.isclose(pne[c], math.exp(-kn / 0.1), rel_tol=1e-9), c
        # normalising by |u| alone would give a different value in every cell
        assert not math.isclose(pne[c], math.exp(-lam * gu[c] / ux[c] / 0.1), rel_tol=1e-3)


def test_velocity_branch_supersonic_uses_speed():
    """Uniform n and T, u_x linear with |u| above the sound speed: the |u| branch
    is normalised by |u|, Kn = lambda |d|u|/dy| / |u|."""
    pne, ux, gu, a, lam = _velocity_case(420.0, 30.0)
    assert ux.min() > a
    for c in range(len(ux)):
        kn = lam * gu[c] / ux[c]
        assert math.isclose(pne[c], math.exp(-kn / 0.1), rel_tol=1e-9), c
        assert not math.isclose(pne[c], math.exp(-lam * gu[c] / a / 0.1), rel_tol=1e-3)


def test_maximum_over_quantities():
    """n and T both linear along the tube with different relative slopes: Eq. 17
    takes the larger of Kn_rho and Kn_T, not their sum."""
    ny = 12
    w, dy, centres = _tube(ny)
    th0 = R * W.T0
    counts = 500 + 40 * np.arange(ny)
    thetas = th0 * (1.0 + 0.03 * np.arange(ny))
    pos, vel, pid = _state(centres, counts, thetas, [(0.0, 0.0, 0.0)] * ny)
    s, pne = _pne_of(w, pos, vel, pid)
    n = _n_of(counts, w)
    T = thetas / R
    gn, gT = np.abs(_grad_1d(n, dy)), np.abs(_grad_1d(T, dy))
    both = 0
    for c in range(ny):
        lam = _lambda(s.mu_ref, w["gas"]["omega"], n[c], thetas[c])
        k_rho, k_T = lam * gn[c] / n[c], lam * gT[c] / T[c]
        assert math.isclose(pne[c], math.exp(-max(k_rho, k_T) / 0.1), rel_tol=1e-9), c
        if min(k_rho, k_T) > 0.2 * max(k_rho, k_T):
            both += 1
            assert not math.isclose(pne[c], math.exp(-(k_rho + k_T) / 0.1), rel_tol=1e-3)
    assert both >= 6


def test_two_dimensional_gradient_is_euclidean_norm():
    """2-D grid, uniform n, zero u, T linear in x and in y: |grad T| is the
    Euclidean norm of the two exact differences (central inside, one-sided on
    the edges), so Kn = lambda sqrt(T_x^2 + T_y^2) / T."""
    nx, ny = 6, 5
    w = W.cavity(n=nx, ppc=400, Kn=0.02, precision="fp64")
    w["grid"]["ny"] = ny
    Lx, Ly = w["grid"]["hi"][0], w["grid"]["hi"][1]
    dx, dy = Lx / nx, Ly / ny
    th0 = R * W.T0
    centres, thetas = [], []
    for iy in range(ny):
        for ix in range(nx):
            centres.append(((ix + 0.5) * dx, (iy + 0.5) * dy))
            thetas.append(th0 * (1.0 + 0.05 * ix + 0.07 * iy))
    counts = np.full(nx * ny, 400)
    pos, vel, pid = _state(centres, counts, thetas, [(0.0, 0.0, 0.0)] * (nx * ny))
    s, pne = _pne_of(w, pos, vel, pid)
    n = _n_of(counts, w)
    T = (np.asarray(thetas) / R).reshape(ny, nx)
    gx = np.stack([_grad_1d(T[iy], dx) for iy in range(ny)])
    gy = np.stack([_grad_1d(T[:, ix], dy) for ix in range(nx)], axis=1)
    for iy in range(ny):
        for ix in range(nx):
            c = iy * nx + ix
            lam = _lambda(s.mu_ref, w["gas"]["omega"], n[c], thetas[c])
            kn = lam * math.hypot(gx[iy, ix], gy[iy, ix]) / T[iy, ix]
            assert math.isclose(pne[c], math.exp(-kn / 0.1), rel_tol=1e-9), (ix, iy)
            l1 = lam * (abs(gx[iy, ix]) + abs(gy[iy, ix])) / T[iy, ix]
            assert not math.isclose(pne[c], math.exp(-l1 / 0.1), rel_tol=1e-3)
