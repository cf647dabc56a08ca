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


def compare(a, b):
    """Per field: z of the seed means, values beyond the bar, the binomial
    bound, mean z^2 and the relative error of the domain average."""
    ma, mb = a.mean(0), b.mean(0)
    va, vb = a.var(0, ddof=1) / len(a), b.var(0, ddof=1) / len(b)
    se = np.sqrt(va + vb)
    rows = {}
    for k, name in enumerate(FIELDS):
        d = ma[k] - mb[k]
        ok_rel = np.abs(d) <= 1e-3 * np.abs(mb[k])
        live = se[k] > 0
        if not live.any():                      # a field that is identically zero on both sides
            assert np.all(d == 0), name
            continue
        z = np.where(live, d / np.where(live, se[k], 1.0), 0.0)
        # Welch-Satterthwaite degrees of freedom of each value
        n = len(a)
        df = np.where(live, (va[k] + vb[k]) ** 2 / np.maximum(va[k] ** 2 / (n - 1) + vb[k] ** 2 / (n - 1), 1e-300),
                      2 * (n - 1))
        v = np.maximum(df[live], 5.0)
        p_tail = 2 * stats.t.sf(3.0, v)
        bad = int(np.sum(live & ~ok_rel & (np.abs(z) > 3.0)))
        nv = int(live.sum())
        tau = autocorrelation_time(z[live])
        n_eff = max(1, int(nv / tau))
        bound = int(math.ceil(tau)) * (int(stats.binom.ppf(0.999, n_eff, float(p_tail.mean()))) + 1)
        e2 = v / (v - 2.0)
        var2 = 3.0 * v * v / ((v - 2.0) * (v - 4.0)) - e2 ** 2
        z2_limit = float(e2.mean() + 4.0 * math.sqrt(var2.mean() / n_eff))
        dom_a, dom_b = ma[k].mean(), mb[k].mean()
        rel = abs(dom_a - dom_b) / max(abs(dom_b), 1e-300)
        # the domain average of each run, compared over the seeds
        da, db = a[:, k].mean(1), b[:, k].mean(1)
        se_dom = math.sqrt(da.var(ddof=1) / len(da) + db.var(ddof=1) / len(db))
        z_dom = (dom_a - dom_b) / se_dom if se_dom > 0 else 0.0
        rows[name] = {"values": nv, "tau": tau, "beyond_3se": bad, "bound": bound,
                      "max_abs_z": float(np.abs(z[live]).max()), "mean_z2": float(np.mean(z[live] ** 2)),
                      "z2_limit": z2_limit, "rel_err_domain_mean": float(rel), "z_domain_mean": float(z_dom)}
    return rows


def assert_fields_agree(rows, what=""):
    for field, r in rows.items():
        assert r["beyond_3se"] <= r["bound"], (what, field, r)
        assert r["mean_z2"] < r["z2_limit"], (what, field, r)
