"""Error bars of FCIQMC estimators from the engine's records.

QMC series are serially correlated, so the paper obtains error bars by
reblocking (Flyvbjerg and Petersen: average neighbouring pairs repeatedly until
the standard error of the blocked series stops growing; the block length is
chosen by the criterion of Lee et al., Phys. Rev. E 83, 066706 (2011)), and
reports the projected energy as a ratio of the averaged numerator and
denominator (App. A.1).  Host-side numpy only.
"""
from __future__ import annotations

import numpy as np


def blocking_levels(series):
    """(blocks, mean, standard error) at block lengths 1, 2, 4, ..."""
    y = np.asarray(series, dtype=np.float64)
    levels = []
    while y.size >= 2:
        levels.append((y.size, float(y.mean()), float(np.sqrt(y.var(ddof=1) / y.size))))
        y = y[: y.size // 2 * 2].reshape(-1, 2).mean(axis=1)
    return levels


def optimal_block(series) -> int:
    """log2 of the block length: the first level k with 2^(3k) > 2 n (s_k / s_0)^4."""
    levels = blocking_levels(series)
    if not levels or levels[0][2] == 0.0:
        return 0
    n, s0 = levels[0][0], levels[0][2]
    for k, (_, _, s) in enumerate(levels):
        if 8.0 ** k > 2.0 * n * (s / s0) ** 4:
            return k
    return len(levels) - 1


def mean_error(series):
    """Mean and reblocked standard error of a series."""
    levels = blocking_levels(series)
    k = optimal_block(series)
    return levels[k][1], levels[k][2]


def projected_energy(records: dict, e_ref: float, start: int = 0):
    """E_proj = E_ref + <num> / <n0> over records[start:], with the error of the
    ratio from the blocked numerator and denominator and their covariance."""
    num = np.asarray(records["num"][start:], dtype=np.float64)
    den = np.asarray(records["n0"][start:], dtype=np.float64)
    k = max(optimal_block(num), optimal_block(den))
    b = 1 << k
    m = num.size // b
    bn = num[: m * b].reshape(m, b).mean(axis=1)
    bd = den[: m * b].reshape(m, b).mean(axis=1)
    r = bn.mean() / bd.mean()
    if m < 2:
        return e_ref + r, float("inf")
    cov = np.cov(np.vstack([bn, bd])) / m
    rel = cov[0, 0] / bn.mean() ** 2 + cov[1, 1] / bd.mean() ** 2 - 2.0 * cov[0, 1] / (bn.mean() * bd.mean())
    return e_ref + r, float(abs(r) * np.sqrt(max(rel, 0.0)))
