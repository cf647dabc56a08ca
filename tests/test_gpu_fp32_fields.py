"""Time-averaged fields of the fused FP32 pipeline against the FP64 CPU oracle.

The bar: every field of every cell within 1e-3 relative or 3 standard
errors of the oracle (Eq. 1 moments, Eq. 33 stress and heat flux, Eq. 16
P_ne, Eq. 34-style time averages).  The standard errors come from
independent seeds: twelve GPU runs (seeds 1..12) and twelve oracle runs
(seeds 101..112) of each case, each averaged over the same window of steps,
so the two sides share no random numbers.  With hundreds of values per
field a per-value 3-SE test fails a few values by chance, so each field
must pass two checks:

* the domain average of each run (it carries the fluctuations that move a
  whole profile at once, such as the energy of a closed gap) agrees by
  Welch's t at the 99.99 % level; the cell checks below use the profiles
  with each run's domain average removed;
* the number of values beyond 3 SE (and beyond 1e-3 relative) stays
  within the 99.99 % binomial bound for the tail probability of Welch's t
  at each value's degrees of freedom;
* each Welch t is mapped to the normal score of the same tail probability,
  and the mean of its square stays below the 99.99 % quantile of
  chi^2(n) / n: a bias of b standard errors adds about b^2 where it
  acts (checked below on synthetic samples: a uniform one-standard-error
  bias fails the domain average, two standard errors in every other cell
  fail the profile; and the false-failure rate).

Neighbouring cells fluctuate together (a shock that runs a little ahead in
one seed moves the velocity of many cells), so z is correlated along the
cell order.  Both checks therefore count independent values, n / tau, with
tau the integrated autocorrelation time of z along the cells (sum of the
lag correlations up to the first that is not positive; the mean of z is
removed first, so a uniform bias does not lengthen it); exceedances are
allowed to come in clusters of tau cells.

The per-field table (largest |z|, mean z^2, relative error of the
domain-averaged field) is written to $USP_FIELD_REPORT when that variable
names a file.
"""
import json
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
from paper_1808_03801_gb300 import workloads as W
from tests._stats import FIELDS, assert_fields_agree, autocorrelation_time, compare, failed


@pytest.fixture(scope="module")
def usp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_03801_gb300 import usp as U
    U.lib()
    assert U.fused_available()
    return U


SEEDS_GPU = list(range(1, 13))
SEEDS_ORC = list(range(101, 113))


def _case(name, seed):
    if name == "sod":
        return W.sod(ny=200, ppc_left=200, seed=seed), 100, 40
    if name == "couette":
        return W.couette(ny=50, ppc=200, Kn=0.1, seed=seed), 300, 100
    if name == "cavity":
        return W.cavity(n=48, ppc=60, Kn=1e-2, seed=seed), 120, 60
    if name == "slit":
        return W.slit(nx=120, ny=60, ppc=40, Kn=1e-2, seed=seed), 100, 50
    raise KeyError(name)


CASES = ["sod", "couette", "cavity", "slit"]


def _oracle_job(job):
    name, seed = job
    w, steps, t0 = _case(name, seed)
    w = W.with_precision(w, "fp64")
    o = oracle.OracleSim(w).init_particles()
    o.step(t0)
    acc = None
    for _ in range(steps - t0):
        o.step(1)
        f = o.fields()[:len(FIELDS)]
        acc = f if acc is None else acc + f
    return name, seed, acc / (steps - t0)


@pytest.fixture(scope="module")
def oracle_means():
    jobs = [(c, s) for c in CASES for s in SEEDS_ORC]
    procs = min(len(jobs), max(1, (os.cpu_count() or 2)))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_job, jobs)
    out = {c: [] for c in CASES}
    for name, seed, m in res:
        out[name].append(m)
    return {c: np.array(v) for c, v in out.items()}


def _gpu_means(usp, name):
    out = []
    for seed in SEEDS_GPU:
        w, steps, t0 = _case(name, seed)
        w = W.with_precision(w, "fp32")
        w["params"]["pipeline"] = "fused"
        g = usp.Simulation(w).init_particles()
        g.step(t0)
        acc = None
        for _ in range(steps - t0):
            g.step(1)
            f = g.sample()[:len(FIELDS)]
            acc = f if acc is None else acc + f
        assert g.info()["counters"][5] == 0
        out.append(acc / (steps - t0))
        g.close()
    return np.array(out)


@pytest.mark.gpu
@pytest.mark.parametrize("name", CASES)
def test_fp32_fields_within_three_standard_errors(usp, oracle_means, name):
    gpu = _gpu_means(usp, name)
    rows = compare(gpu, oracle_means[name])
    report = os.environ.get("USP_FIELD_REPORT")
    if report:
        try:
            cur = json.load(open(report))
        except Exception:
            cur = {}
        cur[name] = rows
        json.dump(cur, open(report, "w"), indent=1)
    assert_fields_agree(rows, name)


def test_compare_detects_a_one_standard_error_bias():
    """The criterion itself: a bias of one standard error in every cell of a
    field fails it; unbiased samples pass."""
    rng = np.random.default_rng(3)
    n = len(SEEDS_GPU)
    a = rng.normal(0, 1, (n, len(FIELDS), 400))
    b = rng.normal(0, 1, (n, len(FIELDS), 400))
    rows = compare(a, b)
    assert not any(failed(r) for r in rows.values())
    se = math.sqrt(2.0 / n)
    # a uniform bias of one standard error of a single cell shows in the domain average
    rows = compare(a + se, b)
    assert all(failed(r) for r in rows.values())
    # a bias of two standard errors in every other cell shows in the profile
    half = np.zeros(400)
    half[::2] = 2.0 * se
    rows = compare(a + half, b)
    assert all(r["mean_z2"] > r["z2_limit"] for r in rows.values())
    # correlated values (a moving average over 5 cells): tau near 5, the
    # unbiased samples still pass and a two-standard-error bias in every
    # other cell still fails
    k = np.ones(5) / math.sqrt(5.0)
    ca = np.apply_along_axis(lambda r: np.convolve(r, k, mode="same"), 2, a)
    cb = np.apply_along_axis(lambda r: np.convolve(r, k, mode="same"), 2, b)
    rows = compare(ca, cb)
    assert all(2.0 < r["tau"] < 10.0 for r in rows.values())
    assert not any(failed(r) for r in rows.values())
    rows = compare(ca + half, cb)
    assert all(r["mean_z2"] > r["z2_limit"] for r in rows.values())


def test_compare_false_failure_rate():
    """Unbiased samples of the sizes used here (eight or twelve seeds, 16 to
    400 values, each run's profile also shifted as a whole) fail a 15-field
    comparison in well under 1 % of draws."""
    rng = np.random.default_rng(11)
    fails = 0
    trials = 0
    for nseed, ncell in ((8, 16), (12, 50), (12, 400)):
        for _ in range(100):
            a = rng.normal(0, 1, (nseed, len(FIELDS), ncell))
            b = rng.normal(0, 1, (nseed, len(FIELDS), ncell))
            # each run's whole profile also moves by a random offset
            a += rng.normal(0, 2, (nseed, len(FIELDS), 1))
            b += rng.normal(0, 2, (nseed, len(FIELDS), 1))
            rows = compare(a, b)
            fails += any(failed(r) for r in rows.values())
            trials += 1
    assert fails <= 2, fails


def test_autocorrelation_time_of_an_ar1_sequence():
    """tau of an AR(1) series with coefficient r is (1 + r)/(1 - r)."""
    rng = np.random.default_rng(5)
    r = 0.6
    x = np.zeros(200000)
    e = rng.normal(size=len(x))
    for i in range(1, len(x)):
        x[i] = r * x[i - 1] + e[i]
    assert abs(autocorrelation_time(x) - (1 + r) / (1 - r)) < 0.25
    assert abs(autocorrelation_time(e) - 1.0) < 0.05
