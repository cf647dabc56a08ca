"""Statistical comparison of two sets of independent runs, field by field.

Shared by the GPU tests that hold the fused FP32 pipeline to the FP64
oracle (or to another GPU path): every value within 1e-3 relative or 3
standard errors, judged per field by the count of exceedances and by the
mean of z^2, both over the number of independent values (comparison only;
no method arithmetic).
"""
import math

import numpy as np
from scipy import stats

FIELDS = ["n", "u0", "u1", "u2", "T", "pxx", "pyy", "pzz", "pxy", "pxz", "pyz", "q0", "q1", "q2", "Pne"]
Q = 0.9999   # quantile of the per-field bounds: about 1.5e-3 false failures per 15-field comparison


def autocorrelation_time(z, max_lag=50):
    """1 + 2 * (sum of the lag correlations of z up to the first that is not
    positive), at least 1."""
    z = np.asarray(z, dtype=float) - np.mean(z)
    c0 = float(np.mean(z * z))
    if c0 <= 0.0:
        return 1.0
    s = 0.0
    for lag in range(1, min(max_lag, len(z) - 1)):
        r = float(np.mean(z[:-lag] * z[lag:])) / c0
        if r <= 0.0:
            break
        s += r
    return 1.0 + 2.0 * s


def _welch(a, b):
    """Difference of the seed means, its standard error and Welch's degrees
    of freedom (arrays over the trailing axes)."""
    n, m = len(a), len(b)
    va, vb = a.var(0, ddof=1) / n, b.var(0, ddof=1) / m
    se2 = va + vb
    df = se2 ** 2 / np.maximum(va ** 2 / (n - 1) + vb ** 2 / (m - 1), 1e-300)
    return a.mean(0) - b.mean(0), np.sqrt(se2), df


def compare(a, b):
    """Per field of two sets of independent runs a[seed, field, cell] and
    b[seed, field, cell]:

    * the domain average of each run (which carries the fluctuations that
      move a whole profile together, such as the total energy of a closed
      gap) by Welch's t over the seeds;
    * the profile with each run's domain average removed, cell by cell:
      values beyond 3 SE (and beyond 1e-3 relative) within their binomial
      bound, and the mean square of the normal scores of the per-cell t
      within the chi^2 quantile, both over n / tau independent values.
    """
    rows = {}
    for k, name in enumerate(FIELDS):
        fa, fb = a[:, k], b[:, k]
        ma, mb = fa.mean(0), fb.mean(0)
        # domain averages
        da, db = fa.mean(1), fb.mean(1)
        d_dom, se_dom, df_dom = _welch(da, db)
        z_dom = float(d_dom / se_dom) if se_dom > 0 else 0.0
        if se_dom == 0 and d_dom != 0:
            z_dom = float("inf")
        dom_limit = float(stats.t.isf((1.0 - Q) / 2.0, max(float(df_dom), 2.0))) if se_dom > 0 else 0.0
        rel = abs(float(ma.mean() - mb.mean())) / max(abs(float(mb.mean())), 1e-300)
        # profiles about each run's domain average
        ra, rb = fa - da[:, None], fb - db[:, None]
        d, se, df = _welch(ra, rb)
        live = se > 0
        if not live.any():
            assert np.all(d == 0) and z_dom == 0.0, name    # a field identically zero or uniform on both sides
            continue
        z = np.where(live, d / np.where(live, se, 1.0), 0.0)
        ok_rel = np.abs(ma - mb) <= 1e-3 * np.abs(mb)
        v = np.maximum(df[live], 2.0)
        p_tail = 2 * stats.t.sf(3.0, v)
        bad = int(np.sum(live & ~ok_rel & (np.abs(z) > 3.0)))
        nv = int(live.sum())
        tau = autocorrelation_time(z[live])
        n_eff = max(1, int(nv / tau))
        bound = int(math.ceil(tau)) * (int(stats.binom.ppf(Q, n_eff, float(p_tail.mean()))) + 1)
        # each Welch t mapped to the standard normal score of the same tail
        # probability, so that the mean of its square follows chi^2(n) / n
        zl = z[live]
        zn = np.sign(zl) * stats.norm.isf(np.clip(stats.t.sf(np.abs(zl), v), 1e-300, 0.5))
        rows[name] = {"values": nv, "tau": tau, "beyond_3se": bad, "bound": bound,
                      "max_abs_z": float(np.abs(zl).max()), "mean_z2": float(np.mean(zn ** 2)),
                      "z2_limit": float(stats.chi2.ppf(Q, n_eff) / n_eff), "z_domain_mean": z_dom,
                      "z_domain_limit": dom_limit, "rel_err_domain_mean": rel}
    return rows


def failed(r):
    return (r["beyond_3se"] > r["bound"] or r["mean_z2"] >= r["z2_limit"]
            or abs(r["z_domain_mean"]) > r["z_domain_limit"])


def assert_fields_agree(rows, what=""):
    for field, r in rows.items():
        assert not failed(r), (what, field, r)
