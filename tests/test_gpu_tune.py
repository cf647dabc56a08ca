"""Autotuner: candidate launch settings all give a working step and the
chosen one is among the fastest measured."""
import pytest

from paper_1808_03801_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_measured_setting():
    from paper_1808_03801_gb300 import autotune
    w = W.with_precision(W.cavity(n=40, ppc=60, Kn=0.01), "fp32")
    w["params"]["pipeline"] = "fused"
    best = autotune.tune(w, steps=3, use_cache=False, candidates_R=(4, 8), candidates_grid=(4, 8))
    times = [t["s_per_step"] for t in best["tried"]]
    assert len(times) == 4 and best["s_per_step"] == min(times)
    assert best["fused_R"] in (4, 8) and best["grid_per_sm"] in (4, 8)


def test_tuning_does_not_change_fp64_results():
    import numpy as np
    from paper_1808_03801_gb300 import usp as U
    w = W.couette(ny=30, ppc=40, precision="fp64")
    a = U.Simulation(w).init_particles()
    b = U.Simulation(w).init_particles().set_tuning(0, 2)
    a.step(8)
    b.step(8)
    pa, pb = a.particles(), b.particles()
    oa, ob = np.argsort(pa["pid"]), np.argsort(pb["pid"])
    assert np.allclose(pa["vel"][oa], pb["vel"][ob], rtol=1e-12, atol=1e-9)
