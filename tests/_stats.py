"""Flyvbjerg-Petersen blocking analysis (the reblocking the paper uses to remove
serial correlation from QMC error bars, Sec. 3.1 and App. A.1), test tooling."""
from __future__ import annotations

import numpy as np


def reblock(x: np.ndarray):
    """Per blocking level: (n_blocks, mean, std_err, std_err_err)."""
    x = np.asarray(x, dtype=np.float64)
    out = []
    while len(x) >= 2:
        n = len(x)
        m = x.mean()
        var = x.var(ddof=1)
        se = np.sqrt(var / n)
        out.append((n, m, se, se / np.sqrt(2.0 * (n - 1))))
        if n % 2:
            x = x[:-1]
        x = 0.5 * (x[0::2] + x[1::2])
    return out


def optimal_level(x: np.ndarray) -> int:
    """Index k of the optimal blocking level: the smallest block size B = 2^k
    with B^3 > 2 N (se_k / se_0)^4 (Lee, Needs et al., PRE 83, 066706 (2011));
    the last level if none qualifies."""
    levels = reblock(x)
    n0, se0 = levels[0][0], levels[0][2]
    if se0 == 0.0:
        return 0
    for k, (n, m, se, see) in enumerate(levels):
        if (2 ** k) ** 3 > 2.0 * n0 * (se / se0) ** 4:
            return k
    return len(levels) - 1


def optimal_error(x: np.ndarray) -> tuple[float, float]:
    """Mean and standard error at the optimal block length."""
    levels = reblock(x)
    k = optimal_level(x)
    return levels[k][1], levels[k][2]


def ratio_estimate(num: np.ndarray, den: np.ndarray):
    """mean(num)/mean(den) and its standard error, both series blocked at the
    larger of their optimal block lengths (numerator and denominator are
    averaged separately before dividing, App. A.1)."""
    num = np.asarray(num, dtype=np.float64)
    den = np.asarray(den, dtype=np.float64)
    k = max(optimal_level(num), optimal_level(den))
    Bk = 2 ** k
    nb = len(num) // Bk
    bn = num[: nb * Bk].reshape(nb, Bk).mean(axis=1)
    bd = den[: nb * Bk].reshape(nb, Bk).mean(axis=1)
    mn, md = bn.mean(), bd.mean()
    r = mn / md
    if nb < 2:
        return r, float("inf")
    c = np.cov(bn, bd) / nb
    var = r * r * (c[0, 0] / mn ** 2 + c[1, 1] / md ** 2 - 2.0 * c[0, 1] / (mn * md))
    return r, float(np.sqrt(max(var, 0.0)))
