"""Pins of the oracle's counter-based generator and variates.

* Philox4x32-10 words against an independent implementation: PyTorch's
  header-only at::philox_engine (compiled here with g++), which takes
  key = seed and counter = (offset, subsequence).
* the uniform map lands strictly inside (0, 1);
* initial velocities (Box-Muller normals) are Maxwellian: KS test and
  moments within their standard errors.
"""
import os
import shutil
import subprocess
import sys
import tempfile

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1808_03801_gb300 import workloads as W

_TORCH_PHILOX = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main() {
  unsigned k0, k1, c0, c1, c2, c3;
  while (scanf("%u %u %u %u %u %u", &k0, &k1, &c0, &c1, &c2, &c3) == 6) {
    uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
    uint64_t off = (uint64_t)c0 | ((uint64_t)c1 << 32);
    uint64_t sub = (uint64_t)c2 | ((uint64_t)c3 << 32);
    at::philox_engine e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _torch_include():
    try:
        import torch
    except Exception:
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    return inc if os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) else None


def test_philox_matches_pytorch_engine():
    inc = _torch_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("PyTorch Philox header or g++ unavailable")
    rng = np.random.default_rng(2024)
    cases = rng.integers(0, 2**32, size=(300, 6), dtype=np.uint64)
    cases[:5] = 0
    cases[1, 0] = 1
    cases[2, 2] = 2**32 - 1
    cases[3, 5] = 7
    cases[4, :] = 2**32 - 1
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cpp")
        exe = os.path.join(d, "p")
        open(src, "w").write(_TORCH_PHILOX)
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-I" + inc, "-o", exe, src])
        inp = "\n".join(" ".join(str(int(v)) for v in row) for row in cases) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    ref = np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()], dtype=np.uint64)
    assert ref.shape == (len(cases), 4)
    for row, want in zip(cases, ref):
        key = row[:2].astype(np.uint32)
        ctr = row[2:].astype(np.uint32)
        got = oracle.philox(ctr, key)
        assert np.array_equal(got.astype(np.uint64), want), (row, got, want)


def test_uniform_open_interval():
    assert oracle.u01(0) == 2.0**-33
    assert oracle.u01(2**32 - 1) == 1.0 - 2.0**-33
    assert 0.0 < oracle.u01(0) < oracle.u01(1) < oracle.u01(2**31) < 1.0


def test_philox_words_uniform():
    key = (12345, 678)
    words = np.array([oracle.philox((i, 3, 1, 0), key) for i in range(4000)], dtype=np.float64)
    u = (words.ravel() + 0.5) / 2**32
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # distinct counters give distinct outputs (Philox is a bijection per key)
    assert len({tuple(w) for w in words.astype(np.uint64)}) == len(words)


def test_init_counts_positions_and_maxwellian():
    w = W.cavity(n=6, ppc=400, Kn=0.05, precision="fp64", steps=1)
    w["regions"] = [dict(w["regions"][0]), {"lo": (0.0, 0.0), "hi": (0.5e-4, 1e-4), "n": W.N0 * 0.5,
                                              "T": 400.0, "u": (100.0, -50.0, 10.0)}]
    s = oracle.OracleSim(w).init_particles()
    P = s.particles()
    counts = s.counts().reshape(6, 6)
    # left half (x centre < 0.5e-4) is the second region: 200 per cell; right half 400 per cell
    assert np.all(counts[:, :3] == 200) and np.all(counts[:, 3:] == 400)
    assert np.array_equal(P["pid"], np.arange(len(P["pid"]), dtype=np.uint32))
    # positions inside their own cells; pids in cell order
    assert np.all(np.diff(P["cell"]) >= 0)
    dx = 1e-4 / 6
    ix = np.floor(P["pos"][:, 0] / dx).astype(int)
    iy = np.floor(P["pos"][:, 1] / dx).astype(int)
    assert np.array_equal(iy * 6 + ix, P["cell"])
    # Maxwellian velocities per region
    kb_m = 1.380649e-23 / W.M_AR
    left = ix < 3
    for sel, T, u in ((left, 400.0, (100.0, -50.0, 10.0)), (~left, W.T0, (0.0, 0.0, 0.0))):
        v = P["vel"][sel]
        z = (v - np.array(u)) / np.sqrt(kb_m * T)
        for d in range(3):
            assert stats.kstest(z[:, d], "norm").pvalue > 1e-3
            assert abs(z[:, d].mean()) < 4.0 / np.sqrt(len(z))
            assert abs(z[:, d].var() - 1.0) < 4.0 * np.sqrt(2.0 / len(z))
