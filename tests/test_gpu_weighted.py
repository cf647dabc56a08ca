"""GPU parity of the weighted added particles (Table 2 steps 2, 4, 7;
Eqs. 22-28 and the third term of Eq. 27) on the plain FP64 pipeline,
through the C ABI, against the FP64 oracle.

The two sides draw every random number from the same counters (the added
particles' ids, the cells for the counts of Eq. 25 and Eq. 28), so after
each step the particle sets agree id by id and every position, velocity and
weight to 1e-10 relative: sums taken in another order differ in the last
bits and enter the weights through Eq. 26, and a rounding of Eq. 25 or
Eq. 28 that lands within those bits of an integer could split the two
(not seen here).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1808_03801_gb300 import workloads as W
from tests._util import KB_M_AR, assert_particles_close, by_pid

pytestmark = pytest.mark.gpu

VSCALE = math.sqrt(KB_M_AR * W.T0)


@pytest.fixture(scope="module")
def usp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_03801_gb300 import usp as U
    U.lib()
    return U


def _weighted_couette(**opt):
    w = W.couette(ny=20, ppc=60, Kn=0.01, u_wall=30.0, dt_over_tauc=5.0, omega=0.81, precision="fp64", seed=6)
    # the instantaneous weight fields of 60 particles per cell let the
    # population grow (+40 % in three steps, on both sides): room for it
    w["params"].update(mode="fixed", fixed_pne=1.0, weighted=1, capacity_factor=8.0)
    w["params"].update(opt)
    return w


def _compare(g, o, w, rtol=1e-10):
    P, Q = g.particles(), o.particles()
    dy = (w["grid"]["hi"][1] - w["grid"]["lo"][1]) / w["grid"]["ny"]
    assert_particles_close(P, Q, VSCALE, dy, rtol=rtol)
    a, b = by_pid(P), by_pid(Q)
    scale = max(1.0, np.abs(b["w"]).max())
    assert np.allclose(a["w"], b["w"], rtol=0, atol=rtol * scale), np.abs(a["w"] - b["w"]).max()
    return a, b


@pytest.mark.parametrize("opt", [dict(), dict(weight_average=1, n_avg=50), dict(r_p=2.0), dict(mode="usp")],
                         ids=["instantaneous", "averaged", "r_p=2", "usp"])
def test_weighted_steps_match_oracle_per_particle(usp, opt):
    w = _weighted_couette(**opt)
    g = usp.Simulation(w).init_particles()
    o = oracle.OracleSim(w).init_particles()
    n0 = o.n
    for steps in (1, 1, 2):
        g.step(steps)
        o.step(steps)
        a, b = _compare(g, o, w)
    if opt.get("mode") != "usp":
        assert np.any(b["w"] != 1.0) and len(b["pid"]) != n0   # particles were added and removed
    F, G = g.sample(), o.fields()
    for k in range(16):
        assert np.allclose(F[k], G[k], rtol=1e-9, atol=1e-9 * max(1e-30, np.abs(G[k]).max())), k
    assert g.info()["counters"][5] == 0


def test_weighted_without_pne_is_the_plain_step(usp):
    """P_ne = 0: Eq. 26 gives weight 0 to nothing -- no particle is added,
    every weight stays 1, and the step is the plain pipeline's."""
    w = _weighted_couette(mode="sp")
    p = W.couette(ny=20, ppc=60, Kn=0.01, u_wall=30.0, dt_over_tauc=5.0, omega=0.81, precision="fp64", seed=6)
    p["params"].update(mode="sp")
    g = usp.Simulation(w).init_particles()
    h = usp.Simulation(p).init_particles()
    g.step(4)
    h.step(4)
    a, b = by_pid(g.particles()), by_pid(h.particles())
    assert np.all(a["w"] == 1.0)
    assert np.array_equal(a["pid"], b["pid"])
    assert np.allclose(a["vel"], b["vel"], rtol=0, atol=1e-12 * VSCALE)


def test_weighted_handle_rejects_unsupported_options(usp):
    for change in (dict(pipeline="fused", precision="fp32"), dict(selection="fixed_count"), dict(r_p=0.0)):
        w = _weighted_couette()
        w["params"].update(change)
        with pytest.raises(usp.UspError):
            usp.Simulation(w)


@pytest.mark.parametrize("kind", ["shear", "heat"])
def test_weighted_transport_independent_of_dt_on_the_gpu(usp, kind):
    """The GPU weighted path reproduces what the oracle's pins establish:
    steady Couette (shear) or thermal Couette (heat) at Kn = 0.01, 50 cells,
    2000 particles per cell, P_ne = 1, dt = 5 tau_c (x = nu dt near 4),
    Eq. 34-averaged weight fields (n_a = 100): mu_eff / mu (or kappa_eff /
    kappa) is 1 within noise, where the scheme without the added particles
    gives 1.23 (the closed forms of the transport section)."""
    ny, ppc = 50, 2000
    if kind == "shear":
        w = W.couette(ny=ny, ppc=ppc, Kn=0.01, u_wall=20.0, dt_over_tauc=5.0, omega=0.81, precision="fp64", seed=4)
    else:
        w = W.couette(ny=ny, ppc=ppc, Kn=0.01, u_wall=0.0, dt_over_tauc=5.0, omega=0.81, precision="fp64", seed=8)
        w["faces"][2]["T"] = W.T0 + 50.0
        w["faces"][3]["T"] = W.T0 - 50.0
    w["params"].update(mode="fixed", fixed_pne=1.0, weighted=1, weight_average=1, n_avg=100, capacity_factor=4.0)
    g = usp.Simulation(w).init_particles()
    n0 = g.info()["n_particles"]
    H = w["grid"]["hi"][1]
    y = (np.arange(ny) + 0.5) * H / ny
    c = slice(int(0.2 * ny), int(0.8 * ny))
    g.step(1500)
    ratios, counts = [], []
    for _ in range(24):
        acc = np.zeros((16, ny))
        for _ in range(200):
            g.step(1)
            acc += g.sample()
        counts.append(g.info()["n_particles"])
        F = acc / 200
        mu = g.info()["mu_ref"] * (F[4][c].mean() / W.T0) ** 0.81
        if kind == "shear":
            ratios.append(-F[8][c].mean() / (mu * np.polyfit(y[c], F[1][c], 1)[0]))
        else:
            kappa = 15.0 / 4.0 * KB_M_AR * mu
            ratios.append(-F[12][c].mean() / (kappa * np.polyfit(y[c], F[4][c], 1)[0]))
    r = np.array(ratios)
    m, se = r.mean(), r.std(ddof=1) / math.sqrt(len(r))
    assert abs(m - 1.0) < 4 * se + 0.03, (m, se)
    assert abs(m - 1.23) > 4 * se + 0.05, (m, se)
    assert max(counts) < 1.3 * n0 and min(counts) > n0, (n0, min(counts), max(counts))
    assert g.info()["counters"][5] == 0
