"""Reblocking of the package's analysis module against closed forms: the
standard error of the mean of an AR(1) series x_t = phi x_(t-1) + e_t is
sigma / ((1 - phi) sqrt(N)) for long series; an uncorrelated series needs no
blocking beyond the criterion's minimum; the ratio estimator of constant series is exact."""
from __future__ import annotations

import numpy as np

from paper_1811_11679_gb300 import analysis


def test_ar1_standard_error():
    rng = np.random.Generator(np.random.Philox(4))
    n, phi = 1 << 17, 0.8
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    m, se = analysis.mean_error(x)
    exact = 1.0 / ((1 - phi) * np.sqrt(n))
    assert abs(se - exact) < 0.15 * exact, (se, exact)
    assert abs(m) < 4 * exact


def test_uncorrelated_series_and_exact_ratio():
    rng = np.random.Generator(np.random.Philox(5))
    x = rng.normal(size=1 << 14)
    # the criterion's block length is about (2N)^(1/3) when nothing is correlated,
    # and the error there is still sigma / sqrt(N)
    assert 2 ** analysis.optimal_block(x) <= 4 * (2 * len(x)) ** (1 / 3)
    _, se = analysis.mean_error(x)
    assert abs(se - 1 / np.sqrt(len(x))) < 0.2 / np.sqrt(len(x))
    rec = {"num": np.full(1000, -3.0), "n0": np.full(1000, 2.0)}
    E, err = analysis.projected_energy(rec, 1.25)
    assert E == 1.25 - 1.5 and err == 0.0
