"""Pins of the 2D real-space Hubbard model (the paper's `lattice` input; its
semi-stochastic example is the half-filled 18-site cluster at U/t = 1.3).

The site set and the hops are rebuilt here independently (floating-point
fractional coordinates instead of the oracle's exact integer ones), the
Hamiltonian by brute-force second quantisation on those hops, and the
non-interacting ground state from the tight-binding band -2t (cos k_x + cos k_y)
on the cluster's allowed momenta.  The oracle's matrix elements, spectrum,
generator and FCIQMC energies must agree with them."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import _brute as B
import _stats as S
import oracle
from paper_1811_11679_gb300 import inputs
from test_oracle_pins import _check_generator, _connected_reachable

TILTED8 = [[2, 2], [2, -2]]
TILTED18 = [[3, 3], [3, -3]]


def _sites_and_hops(lat):
    A = np.asarray(lat, dtype=np.float64)
    d = A.shape[0]
    Ainv = np.linalg.inv(A)
    corners = [sum(A[i] for i in range(d) if (m >> i) & 1) if m else np.zeros(d) for m in range(1 << d)]
    lo = np.floor(np.min(corners, axis=0)).astype(int)
    hi = np.ceil(np.max(corners, axis=0)).astype(int)
    sites = []
    for r in itertools.product(*[range(lo[j], hi[j] + 1) for j in range(d)]):
        f = np.array(r, dtype=np.float64) @ Ainv
        if np.all(f > -1e-9) and np.all(f < 1 - 1e-9):
            sites.append(tuple(r))
    sites.sort()
    # bipartite cell (even coordinate sums of every lattice vector): alternate
    # the even- and odd-parity sites
    if len(sites) % 2 == 0 and all(int(sum(v)) % 2 == 0 for v in np.asarray(lat)):
        ev = [x for x in sites if sum(x) % 2 == 0]
        od = [x for x in sites if sum(x) % 2 != 0]
        if len(ev) == len(od):
            sites = [x for pair in zip(ev, od) for x in pair]
    index = {s: i for i, s in enumerate(sites)}

    def reduce(r):
        f = np.array(r, dtype=np.float64) @ Ainv
        n = np.floor(f + 1e-9)
        return tuple(int(round(x)) for x in np.array(r) - n @ A)

    hops = []
    for s in sites:
        row = []
        for k in range(2 * d):
            r = list(s)
            r[k // 2] += -1 if k & 1 else 1
            row.append(index[reduce(r)])
        hops.append(row)
    return sites, hops


def _hubbard_brute(lat, nalpha, nbeta, t, U):
    sites, hops = _sites_and_hops(lat)
    L = len(sites)
    bonds = {(min(i, j), max(i, j)) for i, row in enumerate(hops) for j in row}
    dets = B.determinants(L, nalpha, nbeta)

    def one(p, q):
        if (p & 1) != (q & 1):
            return 0.0
        return -t if (min(p >> 1, q >> 1), max(p >> 1, q >> 1)) in bonds else 0.0

    def two(p, q, r, s):
        if p == r and q == s and (p >> 1) == (q >> 1) and (p & 1) != (q & 1):
            return U
        return 0.0

    return dets, B.hamiltonian(dets, 2 * L, one, two)


@pytest.mark.parametrize("lat,n", [(TILTED8, 8), (TILTED18, 18), ([[4, 0], [0, 3]], 12), ([[5]], 5)])
def test_lattice_sites_and_hops(lat, n):
    sites, hops = _sites_and_hops(lat)
    assert len(sites) == n
    for i, row in enumerate(hops):
        assert len(set(row)) == len(row) and i not in row
        for j in row:
            assert i in hops[j]            # hopping is symmetric


def _oracle_H(orc, dets):
    index = {d: i for i, d in enumerate(dets)}
    H = np.zeros((len(dets), len(dets)))
    for j, d in enumerate(dets):
        key = B.bits_to_words(d, 1)
        H[j, j] = orc.hdiag(key) - orc.e_ref + orc.e_ref
        ch, _ = orc.enumerate(key)
        for c in {B.words_to_bits(x) for x in ch}:
            if c == 0:
                continue
            H[index[c], j] = orc.hij(key, B.bits_to_words(c, 1))
    return H


def test_slater_condon_2d_lattice_vs_brute_force():
    sysd = inputs.hubbard_lattice_system(TILTED8, 2, 2, t=1.0, U=3.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets, Hb = _hubbard_brute(TILTED8, 2, 2, 1.0, 3.0)
    Ho = _oracle_H(orc, dets)
    assert np.array_equal(Ho, Hb)


def test_2d_noninteracting_ground_state_is_the_filled_band():
    """U = 0 on the tilted 8-site cluster: E0 = sum over spins of the lowest
    tight-binding levels -2t (cos k_x + cos k_y), k = 2 pi A^-1 m."""
    t = 1.0
    A = np.asarray(TILTED8, dtype=np.float64)
    ks = {}
    for m in itertools.product(range(-4, 5), repeat=2):
        k = 2 * np.pi * np.linalg.solve(A, np.array(m, dtype=np.float64))
        k = (k + np.pi) % (2 * np.pi) - np.pi
        ks[tuple(np.round(k, 6))] = k          # one representative per momentum
    eps = sorted(-2 * t * (np.cos(k[0]) + np.cos(k[1])) for k in ks.values())
    assert len(eps) == 8
    e0 = 2 * sum(eps[:4])
    sysd = inputs.hubbard_lattice_system(TILTED8, 4, 4, t=t, U=0.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets = B.determinants(8, 4, 4)
    H = _oracle_H(orc, dets)
    assert abs(np.linalg.eigvalsh(H)[0] - e0) < 1e-10


def test_2d_generator_probabilities():
    sysd = inputs.hubbard_lattice_system(TILTED8, 3, 2, U=2.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets = B.determinants(8, 3, 2)
    rng = np.random.default_rng(8)
    pick = [dets[i] for i in rng.choice(len(dets), 5, replace=False)]
    _check_generator(orc, 1, pick, nsamples=20000)
    for d in pick:
        _connected_reachable(orc, 1, d, dets)


def test_2d_fciqmc_meets_exact_diagonalisation():
    """Half-filled tilted 8-site cluster at U/t = 4, real weights: E_proj within
    two blocking errors of the dense ground state (4900 determinants)."""
    dets, H = _hubbard_brute(TILTED8, 4, 4, 1.0, 4.0)
    E0 = np.linalg.eigvalsh(H)[0]
    sysd = inputs.hubbard_lattice_system(TILTED8, 4, 4, t=1.0, U=4.0)
    q = inputs.qmc_params(tau=0.01, target_population=4000, real_amplitudes=1, spawn_cutoff=0.01, init_pop=100,
                          seed=12)
    orc = oracle.Oracle(sysd, q)
    orc.iterate(3000)
    r = orc.records()
    m, err = S.ratio_estimate(r["num"][1000:], r["n0"][1000:])
    assert abs(orc.e_ref + m - E0) < 2.0 * err, (orc.e_ref + m, err, E0)
    # the shift estimator agrees too (+ a population-control bias allowance)
    ms, es = S.optimal_error(r["shift"][1000:])
    assert abs(orc.e_ref + ms - E0) < 2.0 * es + 0.01, (orc.e_ref + ms, es, E0)


def test_invalid_lattices_are_rejected():
    with pytest.raises(ValueError):
        oracle.Oracle(inputs.hubbard_lattice_system([[2, 0], [0, 2]], 2, 2), inputs.qmc_params())  # +-x coincide
    bad = inputs.hubbard_lattice_system(TILTED8, 4, 4)
    bad["norb"] = 9
    with pytest.raises(ValueError):
        oracle.Oracle(bad, inputs.qmc_params())
