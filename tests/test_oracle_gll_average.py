"""Pins of the oracle's time-averaged Kn_GLL option (params gll_average = 1):
the stencil of Eqs. 17-18 reads the Eq. 34 averages of n, u, T instead of
the instantaneous moments (Sec. 3 averages steady flows to cut statistical
noise).

* Before the first sample there is no average: the first step equals the
  instantaneous reading particle for particle.
* In a uniform gas at rest there is no gradient, so 1 - P_ne measures noise
  alone; averaging over ~n_a steps must cut it (P_ne closer to 1).
* Plumbing: P_ne of a step follows from the averaged fields as they stood
  before that step (the stencil restated here from its definition: central
  differences between valid neighbours, one-sided at a missing one).
"""
import copy
import math

import numpy as np

import oracle
from paper_1808_03801_gb300 import workloads as W

KB = 1.380649e-23


def _uniform_gas(n_avg):
    w = W.couette(ny=50, ppc=50, Kn=0.01, u_wall=0.0, dt_over_tauc=1.0)
    w["faces"][2]["kind"] = w["faces"][3]["kind"] = "specular"
    w["params"]["n_avg"] = n_avg
    return w


def test_first_step_equals_instantaneous_reading():
    w = W.sod(ny=100, ppc_left=60, precision="fp64")
    w2 = copy.deepcopy(w)
    w2["params"]["gll_average"] = 1
    a = oracle.OracleSim(w).init_particles().step(1)
    b = oracle.OracleSim(w2).init_particles().step(1)
    assert np.array_equal(a.params(), b.params())
    Pa, Pb = a.particles(), b.particles()
    assert np.array_equal(Pa["vel"], Pb["vel"]) and np.array_equal(Pa["pos"], Pb["pos"])
    a.step(1)
    b.step(1)
    assert not np.array_equal(a.params()[:, 13], b.params()[:, 13])   # from the second step on they differ


def test_averaging_removes_noise_gradients():
    means = {}
    for ga in (0, 1):
        w = _uniform_gas(n_avg=20)
        w["params"]["gll_average"] = ga
        o = oracle.OracleSim(w).init_particles()
        pn = []
        for k in range(120):
            o.step(1)
            if k >= 60:
                pn.append(o.params()[:, 13].mean())
        means[ga] = float(np.mean(pn))
    assert means[1] > means[0] + 0.15, means
    assert means[1] > 0.7


def _pne_from_fields(F, w, dt):
    """P_ne of every cell of a 1-D grid from fields [field][cell] (n, u, T)."""
    g, pr = w["gas"], w["params"]
    R = KB / g["mass"]
    ny = w["grid"]["ny"]
    h = (w["grid"]["hi"][1] - w["grid"]["lo"][1]) / ny
    n, T = F[0], F[4]
    um = np.sqrt(F[1] ** 2 + F[2] ** 2 + F[3] ** 2)
    valid = (n > 0) & (T > 0)
    mu_ref = _mu_ref(w)
    out = np.ones(ny)
    for i in range(ny):
        if not valid[i]:
            continue
        rho = n[i] * g["mass"]
        p = rho * R * T[i]
        mu = mu_ref * (T[i] / g["T_ref"]) ** g["omega"]
        lam = 16.0 / (5.0 * math.sqrt(2.0 * math.pi)) * mu / math.sqrt(rho * p)
        a_s = math.sqrt(5.0 / 3.0 * R * T[i])
        kn = 0.0
        for Q, scale in ((n, n[i]), (T, T[i]), (um, max(um[i], a_s))):
            m = i - 1 if i > 0 and valid[i - 1] else None
            q = i + 1 if i < ny - 1 and valid[i + 1] else None
            if m is not None and q is not None:
                d = (Q[q] - Q[m]) / (2 * h)
            elif q is not None:
                d = (Q[q] - Q[i]) / h
            elif m is not None:
                d = (Q[i] - Q[m]) / h
            else:
                d = 0.0
            kn = max(kn, lam * abs(d) / scale)
        out[i] = math.exp(-kn / 0.1)
    return out


def _mu_ref(w):
    o = oracle.OracleSim(w)
    return o.mu_ref


def test_pne_follows_the_averaged_fields():
    w = W.sod(ny=80, ppc_left=60, precision="fp64")
    w["params"]["gll_average"] = 1
    w["params"]["n_avg"] = 10
    o = oracle.OracleSim(w).init_particles().step(15)
    F = o.fields(averaged=True)
    o.step(1)
    P = o.params()
    sel = P[:, 14] > 0
    want = _pne_from_fields(F, w, o.dt)
    assert np.allclose(P[sel, 13], want[sel], rtol=1e-10, atol=1e-14)
    # and not the instantaneous fields of that step
    assert not np.allclose(P[sel, 13], _pne_from_fields(o.fields(), w, o.dt)[sel], rtol=1e-6)
