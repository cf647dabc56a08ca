"""Continuous batching on the GPU: solves that arrive while others are
running are admitted into the resident batch, advanced together and retired
at their own step counts, and each result equals the same solve run alone.

In FP64 the comparison is per particle at 1e-12 (the batch changes only the
summation order inside cells); the FP32 fused server is checked on bulk
time averages."""
import math

import numpy as np
import pytest

from paper_1808_03801_gb300 import workloads as W
from tests._util import KB_M_AR, assert_particles_close

pytestmark = pytest.mark.gpu
VSCALE = math.sqrt(KB_M_AR * W.T0)


def _requests():
    reqs = [W.couette(ny=30, ppc=40, steps=24, seed=3), W.cavity(n=12, ppc=20, Kn=0.05, steps=16, seed=4),
            W.sod(ny=60, ppc_left=40, steps=40, seed=5), W.poiseuille(ny=20, ppc=30, steps=9, seed=6),
            W.slit(nx=20, ny=10, ppc=12, steps=20, seed=7), W.couette(ny=12, ppc=25, Kn=0.5, steps=31, seed=8)]
    return [W.with_precision(w, "fp64") for w in reqs]


def test_served_fp64_results_equal_alone():
    from paper_1808_03801_gb300 import usp as U
    from paper_1808_03801_gb300.serve import serve_requests
    reqs = _requests()
    rep, finished = serve_requests(reqs, rate=400.0, hbm_budget=4 << 30, pipeline="plain", precision="fp64",
                                   chunk=8, keep_results=True)
    assert rep["requests"] == len(reqs)
    assert rep["p99_s"] >= rep["p50_s"] > 0
    for r in finished:
        sim = r.result["sim"]
        assert sim.info()["step"] == r.steps
        alone = U.Simulation(reqs[r.rid]).init_particles()
        alone.step(r.steps)
        gr = reqs[r.rid]["grid"]
        assert_particles_close(sim.particles(), alone.particles(), VSCALE,
                               (gr["hi"][1] - gr["lo"][1]) / gr["ny"])
        assert np.allclose(r.result["fields"], alone.sample(averaged=True), rtol=1e-10,
                           atol=1e-10 * np.abs(r.result["fields"]).max())
        sim.close()
        alone.close()


def test_served_fp32_fused_many_requests_finish():
    from paper_1808_03801_gb300.serve import serve_requests
    reqs = W.serving_requests(n=24, seed=3, n_min=1e4, n_max=2e5, steps_min=20, steps_max=80)
    rep, finished = serve_requests(reqs, rate=200.0, hbm_budget=8 << 30, pipeline="fused", precision="fp32")
    assert rep["requests"] == 24
    assert rep["aggregate_updates_per_s"] > 0
    assert all(r.done > r.arrival for r in finished)
