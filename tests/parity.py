"""Comparison helpers between the CUDA path and the oracle.

Acceptance (statistical, independent or matched random streams):
* every tally bin within 3 sigma, allowing the number of 3-sigma excursions
  expected by chance over many bins: count <= N p + 3 sqrt(N p (1-p)),
  p = 0.0027;
* chi^2 over bins with enough counts has p > 0.01.
Sigma comes from Poisson counts or, for correlated tallies, from the spread of
per-batch results (primary-id batches).
"""
import math

import numpy as np

P3 = 0.0027
N_SPECIES = 4                  # e-, T2+, T3+, T+ (ledger layout of the C ABI and the oracle)
BIRTHS, DEATHS = 12, 16


def excursions_ok(z: np.ndarray) -> bool:
    n = z.size
    if n == 0:
        return True
    bad = int(np.sum(np.abs(z) > 3.0))
    return bad <= n * P3 + 3.0 * math.sqrt(n * P3 * (1 - P3)) + 1


def poisson_two_sample(a: np.ndarray, b: np.ndarray, min_count: int = 10):
    """z-scores and chi^2 p-value for two Poisson histograms of equal expectation."""
    from scipy import stats
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    tot = a + b
    m = tot > 0
    z = (a[m] - b[m]) / np.sqrt(tot[m])
    big = tot >= min_count
    chi2 = float(np.sum((a[big] - b[big]) ** 2 / tot[big]))
    dof = int(np.sum(big))
    p = float(stats.chi2.sf(chi2, dof)) if dof > 0 else 1.0
    return z, p


def batch_means(batches: np.ndarray):
    """Mean and standard error over the first axis (batches)."""
    b = np.asarray(batches, np.float64)
    k = b.shape[0]
    return b.mean(axis=0), b.std(axis=0, ddof=1) / math.sqrt(k)


def batch_two_sample(ga: np.ndarray, ob: np.ndarray, min_se_frac: float = 0.0):
    """z-scores of two batched tallies [k, ...] and chi^2 p over bins with spread."""
    from scipy import stats
    ma, sa = batch_means(ga)
    mb, sb = batch_means(ob)
    se = np.sqrt(sa ** 2 + sb ** 2)
    m = se > 0
    z = (ma[m] - mb[m]) / se[m]
    chi2 = float(np.sum(z ** 2))
    dof = int(z.size)
    p = float(stats.chi2.sf(chi2, dof)) if dof > 0 else 1.0
    return z, p


def ledger_balances(L) -> bool:
    e_in = int(L[0]) + int(L[1])
    e_out = int(np.sum(L[2:12]))
    births = np.asarray(L[BIRTHS:BIRTHS + N_SPECIES])
    deaths = np.asarray(L[DEATHS:DEATHS + 8 * N_SPECIES]).reshape(N_SPECIES, 8).sum(axis=1)
    return e_in == e_out and np.array_equal(births, deaths)


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    d = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / d) if d > 0 else float(np.linalg.norm(a))


def hotelling_two_sample(a: np.ndarray, b: np.ndarray) -> float:
    """p-value of Hotelling's two-sample T^2 test on batch vectors a [k1, d],
    b [k2, d]: equal means, correlated components, common covariance."""
    from scipy import stats
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n1, d = a.shape
    n2 = b.shape[0]
    diff = a.mean(0) - b.mean(0)
    s = ((n1 - 1) * np.cov(a, rowvar=False) + (n2 - 1) * np.cov(b, rowvar=False)) / (n1 + n2 - 2)
    s = np.atleast_2d(s)
    t2 = n1 * n2 / (n1 + n2) * float(diff @ np.linalg.solve(s, diff))
    f = (n1 + n2 - d - 1) / (d * (n1 + n2 - 2)) * t2
    return float(stats.f.sf(f, d, n1 + n2 - d - 1))


def coarse_groups(x: np.ndarray, groups: int) -> np.ndarray:
    """Sum the last axis of [k, n] into `groups` contiguous groups."""
    k, n = x.shape
    edges = np.linspace(0, n, groups + 1).astype(int)
    return np.stack([x[:, a:b].sum(1) for a, b in zip(edges[:-1], edges[1:])], axis=1)


def excursion_bound(n: int, p: float) -> float:
    """Largest count of bins beyond the threshold that chance allows in n
    independent bins of tail probability p (mean + 3 standard deviations)."""
    return n * p + 3.0 * math.sqrt(n * p * (1.0 - p)) + 1


def deviation_summary(z: np.ndarray, dof: int) -> dict:
    """Per-bin deviations z (in standard errors) of one tally: median and
    largest |z|, the count beyond 3 with the count chance allows for a
    t distribution of `dof` degrees of freedom (standard errors estimated from
    batches), and the chi^2 p-value of sum z^2."""
    from scipy import stats
    z = np.asarray(z, np.float64).ravel()
    n = int(z.size)
    if n == 0:
        return {"bins": 0, "median_abs_z": 0.0, "max_abs_z": 0.0, "beyond_3": 0,
                "allowed_beyond_3": 1.0, "chi2_p": 1.0}
    p3 = float(2.0 * stats.t.sf(3.0, dof))
    # sum of squared t variables: compare with n * dof/(dof-2) mean by a
    # chi^2 of the rescaled statistic (close for dof >= 30)
    scale = dof / (dof - 2.0) if dof > 2 else 1.0
    chi2 = float(np.sum(z ** 2) / scale)
    return {"bins": n, "median_abs_z": float(np.median(np.abs(z))),
            "max_abs_z": float(np.max(np.abs(z))), "beyond_3": int(np.sum(np.abs(z) > 3.0)),
            "allowed_beyond_3": excursion_bound(n, p3), "chi2_p": float(stats.chi2.sf(chi2, n))}


def batches_vs_total(g_batches: np.ndarray, o_total: np.ndarray, min_mean: float = 0.0):
    """z-scores of the summed batches of one implementation against the total
    of another run of the same primaries, with the variance of either total
    estimated from the batches (both totals have it when they agree in law).
    Bins whose batch mean is at most min_mean, or have no spread, are left out."""
    g = np.asarray(g_batches, np.float64)
    k = g.shape[0]
    g = g.reshape(k, -1)
    o = np.asarray(o_total, np.float64).ravel()
    var_tot = k * g.var(axis=0, ddof=1)
    keep = (var_tot > 0) & (g.mean(axis=0) > min_mean)
    z = (g.sum(axis=0)[keep] - o[keep]) / np.sqrt(2.0 * var_tot[keep])
    return z, k - 1
