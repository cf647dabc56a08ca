"""Helpers shared by the tests (comparison only; no method arithmetic)."""
import math

import numpy as np

KB_M_AR = 1.380649e-23 / 6.63e-26


def by_pid(P):
    o = np.argsort(P["pid"], kind="stable")
    return {k: v[o] for k, v in P.items()}


def assert_particles_close(gpu, orc, vel_scale, pos_scale, rtol=1e-12, check_cells=True):
    """Per-particle comparison matched by pid: |a - b| <= rtol * max(|b|, scale)."""
    g, o = by_pid(gpu), by_pid(orc)
    assert len(g["pid"]) == len(o["pid"]), (len(g["pid"]), len(o["pid"]))
    assert np.array_equal(g["pid"], o["pid"])
    dv = np.abs(g["vel"] - o["vel"])
    tv = rtol * np.maximum(np.abs(o["vel"]), vel_scale)
    bad = dv > tv
    if bad.any():
        i = np.argwhere(bad)[0][0]
        rel = (dv / np.maximum(np.abs(o["vel"]), vel_scale)).max()
        raise AssertionError(f"velocity mismatch at pid {o['pid'][i]}: gpu {g['vel'][i]!r} oracle {o['vel'][i]!r}; "
                             f"{bad.any(1).sum()} particles differ, max relative difference {rel:.3e}")
    dp = np.abs(g["pos"] - o["pos"])
    tp = rtol * np.maximum(np.abs(o["pos"]), pos_scale)
    bad = dp > tp
    if bad.any():
        i = np.argwhere(bad)[0][0]
        raise AssertionError(f"position mismatch at pid {o['pid'][i]}: gpu {g['pos'][i]} oracle {o['pos'][i]}")
    if check_cells:
        assert np.array_equal(g["cell"], o["cell"]), "cell ids differ"


def block_stats(samples):
    """Mean and standard error from a list of block means (axis 0)."""
    a = np.asarray(samples)
    return a.mean(0), a.std(0, ddof=1) / math.sqrt(len(a))
