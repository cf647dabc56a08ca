"""GPU tests of the slab decomposition (one domain as slab handles of one
batch, particles crossing slab boundaries written into the neighbour's
buckets, the Kn_GLL stencil reading the neighbour's row).

* one step from the same particles: the decomposed domain and the whole
  domain hold the same particles in the same cells at the same positions
  (advection and scatter are exact in FP32; no relaxation is pending in the
  first step); velocities agree to FP32 rounding (reading the particles
  applies the relaxation computed from FP32 sums taken in another order);
* later steps: the relaxation's FP32 moment sums run in a different order,
  so agreement is statistical: density, velocity and temperature profiles
  over several seeds within their standard errors; particles conserved;
* errors: a slab stepped alone, slabs admitted out of order, a grid that
  does not split evenly.
"""
import math

import numpy as np
import pytest

from paper_1808_03801_gb300 import workloads as W
from tests._util import by_pid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_03801_gb300 import usp as U, decomp as D
    U.lib()
    return U, D


def _fused(w):
    w = W.with_precision(w, "fp32")
    w["params"]["pipeline"] = "fused"
    w["params"]["capacity_factor"] = 3.0
    return w


def _case(name, seed=1):
    if name == "sod":
        return _fused(W.sod(ny=200, ppc_left=80, seed=seed))
    return _fused(W.cavity(n=24, ppc=30, Kn=0.01, seed=seed))


@pytest.mark.parametrize("name,nslabs", [("sod", 4), ("cavity", 3)])
def test_one_step_identical_to_whole_domain(env, name, nslabs):
    U, D = env
    w = _case(name)
    g = U.Simulation(w).init_particles()
    P = g.particles()
    whole = U.Simulation(w).set_particles(P["pos"], P["vel"], P["pid"])
    dec = D.DecomposedSim(w, nslabs).load(P)
    whole.step(1)
    dec.step(1)
    a, b = by_pid(whole.particles()), by_pid(dec.particles())
    for k in ("pid", "pos", "cell"):
        assert np.array_equal(a[k], b[k]), k
    scale = np.sqrt(np.mean(a["vel"] ** 2))
    assert np.max(np.abs(a["vel"] - b["vel"])) < 1e-4 * scale
    assert dec.counters()[5] == 0
    dec.close()


def test_profiles_match_whole_domain_statistically(env):
    U, D = env
    pw, pd = [], []
    for seed in range(1, 7):
        w = _case("sod", seed)
        g = U.Simulation(w).init_particles()
        P = g.particles()
        n0 = len(P["pid"])
        whole = U.Simulation(w).set_particles(P["pos"], P["vel"], P["pid"])
        dec = D.DecomposedSim(w, 4).load(P)
        whole.step(40)
        dec.step(40)
        pw.append(whole.sample()[[0, 2, 4]])
        pd.append(dec.sample()[[0, 2, 4]])
        assert dec.n_particles() == n0
        c = dec.counters()
        assert c[5] == 0 and c[4] > 0          # nothing lost; relaxations happened
        Q = dec.particles()
        assert len(Q["pid"]) == n0 and len(np.unique(Q["pid"])) == n0
        dec.close()
    a, b = np.array(pw), np.array(pd)
    z = (a.mean(0) - b.mean(0)) / np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b) + 1e-300)
    assert np.abs(z).max() < 5.0
    assert (z ** 2).mean() < 2.5


def test_slab_errors(env):
    U, D = env
    w = _case("sod")
    ws = D.slab_workloads(w, 4)
    s0 = U.Simulation(ws[0])
    P = U.Simulation(w).init_particles().particles()
    part = D.split(P, w, 4)[0]
    s0.set_particles(part["pos"], part["vel"], part["pid"])
    with pytest.raises(U.UspError):
        s0.step(1)                                   # a slab alone
    with pytest.raises(U.UspError):
        s0.init_particles()                          # slabs are loaded, not initialised
    sims = [s0] + [U.Simulation(x) for x in ws[1:]]
    for s, part in zip(sims[1:], D.split(P, w, 4)[1:]):
        s.set_particles(part["pos"], part["vel"], part["pid"])
    B = U.Batch(hbm_budget=8 << 30, max_sims=4)
    for s in (sims[1], sims[0], sims[2], sims[3]):  # out of slab order
        assert B.admit(s) == 0
    with pytest.raises(U.UspError):
        B.step(1)
    B.close()
    bad = dict(ws[0])
    bad["grid"] = dict(bad["grid"], ny=202)          # not a multiple of 4
    with pytest.raises(U.UspError):
        U.Simulation(bad)
