"""Pins of the CPU oracle against things other than itself: numpy's Philox,
published known-answer vectors, math.log, exact rational arithmetic, brute-force
second quantisation, closed forms and exact probability sums."""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import inputs
import _brute as B

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers():
    """Random123 known-answer vectors for Philox4x64-10 (Salmon et al. SC'11)."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x64_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = oracle.philox(v[:4], v[4:6])
        assert [int(x) for x in out] == v[6:]
        n += 1
    assert n == 3


def test_philox_matches_numpy():
    """numpy.random.Philox (4x64-10) increments its counter before each block,
    so its first block for counter c is the oracle's block for c + 1."""
    rng = np.random.default_rng(123)
    for _ in range(200):
        key = rng.integers(0, 2**63, size=2, dtype=np.uint64)
        ctr = rng.integers(0, 2**63, size=4, dtype=np.uint64)
        g = np.random.Philox(key=key, counter=ctr)
        raw = g.random_raw(4)
        c1 = ctr.copy()
        c1[0] += np.uint64(1)
        assert np.array_equal(oracle.philox(c1, key), raw)


# --------------------------------------------------------------------------- ln
def _ulp_diff(a: float, b: float) -> int:
    ia = np.float64(a).view(np.int64)
    ib = np.float64(b).view(np.int64)
    return abs(int(ia) - int(ib))


def test_own_log_against_math_log():
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(0.5, 2.0, 5000), np.exp(rng.uniform(-700, 700, 5000)),
                         1.0 + rng.uniform(-1e-3, 1e-3, 2000), [1.0, 2.0, 0.5, 10.0, 1e-300]])
    worst = 0
    for x in xs:
        ref = math.log(float(x))
        got = oracle.log(float(x))
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, _ulp_diff(got, ref))
    assert worst <= 4, worst


def test_own_log_special_values():
    assert oracle.log(1.0) == 0.0
    assert oracle.log(0.0) == -math.inf
    assert abs(oracle.log(math.e) - 1.0) < 4e-16


# --------------------------------------------------------------------------- fixed point
def test_fixed_point_term_is_round_half_even_of_the_exact_product():
    """Each estimator / deterministic-space term is round_half_even(n h 2^16) of
    the exact product of an int64 population and a double (checked with Fractions)."""
    rng = np.random.default_rng(3)
    ns = [int(x) for x in rng.integers(-(2 ** 62), 2 ** 62, 2000)]
    ns += [int(x) for x in rng.integers(-(2 ** 33), 2 ** 33, 2000)]
    hs = list(rng.normal(0, 1, 4000) * 10.0 ** rng.integers(-12, 4, 4000))
    # exact ties (n h 2^16 = k + 1/2), subnormal and tiny h, zero, extremes
    ns += [1, 3, -1, -3, 5, 7, 2 ** 62 - 1, -(2 ** 62), 1, 123456789, 0, 1]
    hs += [2.0 ** -17, 2.0 ** -17, 2.0 ** -17, 2.0 ** -17, 0.1, 2.5 * 2.0 ** -16, 3.75, -0.001,
           5e-324, 2.2e-308, 1.0, 0.0]
    for n, h in zip(ns, hs):
        exact = Fraction(n) * Fraction(float(h)) * 65536
        fl = math.floor(exact)
        rem = exact - fl
        if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
            fl += 1
        assert oracle.fixed_term(n, float(h)) == fl, (n, h)


def test_spawn_amount_is_one_rounding_of_the_exact_product():
    """The spawned amount is floor(a b 2^32) or floor(a b 2^32 + 1/2) of the
    exact rational product, saturated at 2^62 (checked with Fractions)."""
    rng = np.random.default_rng(5)
    a = list(np.abs(rng.normal(0, 1, 3000)) * 10.0 ** rng.integers(-12, 6, 3000))
    b = list(np.abs(rng.normal(0, 1, 3000)) * 10.0 ** rng.integers(-4, 9, 3000))
    # exact ties, subnormals, saturation, zero
    a += [1.5 * 2.0 ** -32, 2.5 * 2.0 ** -32, 3.0 * 2.0 ** -40, 5e-324, 2.2e-308, 1.0, 2.0 ** 29, 0.0, 0.3]
    b += [1.0, 1.0, 2.0 ** 7, 2.0 ** 1000, 3.0, 2.0 ** 30 - 1, 2.0 ** 33, 5.0, 0.0]
    cap = 2 ** 62
    for x, y in zip(a, b):
        exact = Fraction(float(x)) * Fraction(float(y)) * 2 ** 32
        fl = math.floor(exact)
        rd = math.floor(exact + Fraction(1, 2))
        assert oracle.fixed_product(x, y, False) == min(fl, cap), (x, y)
        assert oracle.fixed_product(x, y, True) == min(rd, cap), (x, y)


# --------------------------------------------------------------------------- Hamiltonians
def _oracle_matrix(orc: oracle.Oracle, dets, W):
    n = len(dets)
    H = np.zeros((n, n))
    keys = [B.bits_to_words(d, W) for d in dets]
    for j in range(n):
        for i in range(n):
            H[i, j] = orc.hij(keys[j], keys[i])
    return H


def test_slater_condon_hubbard_vs_brute_force():
    sysd = inputs.hubbard_system(L=4, nalpha=2, nbeta=2, t=1.0, U=4.0, periodic=True)
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets, Hb = B.hubbard_hamiltonian(4, 2, 2, 1.0, 4.0, True)
    Ho = _oracle_matrix(orc, dets, 1)
    assert np.array_equal(Ho, Ho.T)
    assert np.max(np.abs(Ho - Hb)) < 1e-13


def test_slater_condon_molecule_vs_brute_force():
    h1, eri = inputs.molecule_integrals(5, seed=5)
    sysd = {"kind": "molecule", "key_words": 1, "norb": 5, "nalpha": 2, "nbeta": 2,
            "h1": h1, "eri": eri, "ecore": 0.0}
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets, Hb = B.molecule_hamiltonian(h1, eri, 2, 2)
    Ho = _oracle_matrix(orc, dets, 1)
    assert np.array_equal(Ho, Ho.T), "H must be exactly symmetric"
    assert np.max(np.abs(Ho - Hb)) < 1e-12


def test_slater_condon_ueg_vs_brute_force():
    sysd = inputs.ueg_system(nel=4, norb=7, rs=1.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    kv_o, box = orc.ueg_basis()
    dets, Hb, kv, L = B.ueg_hamiltonian(7, 2, 2, 1.0)
    assert np.array_equal(kv_o, kv)
    assert abs(box - L) < 1e-13 * L
    Ho = _oracle_matrix(orc, dets, 1)
    assert np.array_equal(Ho, Ho.T)
    assert np.max(np.abs(Ho - Hb)) < 1e-12


def test_ueg_momentum_and_spin_conservation():
    """Every nonzero off-diagonal element (all singles and doubles of sampled
    determinants) conserves total momentum and each spin population."""
    import itertools
    sysd = inputs.ueg_system(nel=6, norb=19, rs=2.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    kv, _ = orc.ueg_basis()
    dets = B.determinants(19, 3, 3)
    rng = np.random.default_rng(0)
    nonzero = 0
    for i in rng.choice(len(dets), 6, replace=False):
        a = dets[i]
        src = B.bits_to_words(a, 1)
        occ = [p for p in range(38) if (a >> p) & 1]
        vir = [p for p in range(38) if not (a >> p) & 1]
        targets = [a ^ (1 << p) ^ (1 << q) for p in occ for q in vir]
        targets += [a ^ (1 << p) ^ (1 << q) ^ (1 << r) ^ (1 << s)
                    for p, q in itertools.combinations(occ, 2)
                    for r, s in itertools.combinations(vir, 2)]
        ka = sum(kv[p >> 1] for p in occ)
        for b in targets:
            h = orc.hij(src, B.bits_to_words(b, 1))
            kb = sum(kv[p >> 1] for p in range(38) if (b >> p) & 1)
            spin_a = [bin(a & int("01" * 19, 2)).count("1"), bin(a & int("10" * 19, 2)).count("1")]
            spin_b = [bin(b & int("01" * 19, 2)).count("1"), bin(b & int("10" * 19, 2)).count("1")]
            if h != 0.0:
                nonzero += 1
                assert np.array_equal(ka, kb)
                assert spin_a == spin_b
            elif np.array_equal(ka, kb) and spin_a == spin_b and bin(a ^ b).count("1") == 4:
                # momentum-conserving doubles vanish only by direct/exchange cancellation
                pass
    assert nonzero > 0


def test_hubbard_two_site_closed_form():
    """Open 2-site chain, one up and one down: E0 = U/2 - sqrt(U^2/4 + 4t^2)."""
    for U in (0.5, 2.0, 4.0, 8.0):
        sysd = inputs.hubbard_system(L=2, nalpha=1, nbeta=1, t=1.0, U=U, periodic=False)
        orc = oracle.Oracle(sysd, inputs.qmc_params())
        dets = B.determinants(2, 1, 1)
        H = _oracle_matrix(orc, dets, 1)
        e0 = np.linalg.eigvalsh(H)[0]
        assert abs(e0 - (U / 2 - math.sqrt(U * U / 4 + 4.0))) < 1e-13


def test_hubbard_8site_spectrum_two_constructions():
    """8-site ring (4900 determinants): ground state of the oracle's H equals
    that of the brute-force operator construction."""
    sysd = inputs.hubbard_system()
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets, Hb = B.hubbard_hamiltonian(8, 4, 4, 1.0, 4.0, True)
    # oracle matrix only over connected pairs (single hops) to keep it cheap
    n = len(dets)
    idx = {d: i for i, d in enumerate(dets)}
    Ho = np.zeros((n, n))
    for j, d in enumerate(dets):
        k = B.bits_to_words(d, 1)
        Ho[j, j] = orc.hdiag(k)
        for p in range(16):
            if not (d >> p) & 1:
                continue
            for q in range(16):
                if (d >> q) & 1 or (p & 1) != (q & 1):
                    continue
                d2 = d ^ (1 << p) ^ (1 << q)
                Ho[idx[d2], j] = orc.hij(k, B.bits_to_words(d2, 1))
    assert np.max(np.abs(Ho - Hb)) < 1e-13
    e_o = np.linalg.eigvalsh(Ho)[0]
    e_b = np.linalg.eigvalsh(Hb)[0]
    assert abs(e_o - e_b) < 1e-11


# --------------------------------------------------------------------------- generators
def _check_generator(orc, W, dets, nsamples=0, seed=0):
    rng = np.random.default_rng(seed)
    for d in dets:
        key = B.bits_to_words(d, W)
        children, probs = orc.enumerate(key)
        assert abs(probs.sum() - 1.0) < 1e-12
        tot = {}
        for ch, p in zip(children, probs):
            cb = B.words_to_bits(ch)
            tot[cb] = tot.get(cb, 0.0) + p
        # every connected determinant is reachable (ergodicity)
        nspin = 64 * W
        for cb, p in tot.items():
            if cb == 0:
                continue
            assert p > 0.0
        # sampled excitations report the exact summed path probability
        for _ in range(200):
            w = rng.integers(0, 2**64 - 1, size=4, dtype=np.uint64, endpoint=True)
            r = orc.generate(key, w)
            if r is None:
                continue
            child, pg, h = r
            cb = B.words_to_bits(child)
            assert abs(pg - tot[cb]) <= 1e-14 * tot[cb]
            # the spawn weight uses 1/p_gen as two reciprocal factors
            ia, ib = orc.last_inv
            assert abs(ia * ib * pg - 1.0) < 1e-15
            assert h == orc.hij(key, child)
        if nsamples:
            # chi^2 of the empirical child distribution against the exact one
            counts = {}
            words = rng.integers(0, 2**64 - 1, size=(nsamples, 4), dtype=np.uint64, endpoint=True)
            for w in words:
                r = orc.generate(key, w)
                cb = 0 if r is None else B.words_to_bits(r[0])
                counts[cb] = counts.get(cb, 0) + 1
            keys = sorted(tot)
            exp = np.array([tot[k] * nsamples for k in keys])
            obs = np.array([counts.get(k, 0) for k in keys])
            m = exp > 5
            chi2 = float(((obs[m] - exp[m]) ** 2 / exp[m]).sum())
            dof = int(m.sum()) - 1
            # 6-sigma bound on a chi^2 variable with `dof` degrees of freedom
            assert chi2 < dof + 6.0 * math.sqrt(2.0 * dof), (chi2, dof)
        del nspin


def _connected_reachable(orc, W, d, dets):
    key = B.bits_to_words(d, W)
    children, probs = orc.enumerate(key)
    reach = {}
    for ch, p in zip(children, probs):
        cb = B.words_to_bits(ch)
        reach[cb] = reach.get(cb, 0.0) + p
    for d2 in dets:
        if d2 == d:
            continue
        h = orc.hij(key, B.bits_to_words(d2, W))
        if h != 0.0:
            assert reach.get(d2, 0.0) > 0.0, "nonzero H_ij with zero generation probability"


def test_hubbard_generator_probabilities():
    sysd = inputs.hubbard_system()
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets = B.determinants(8, 4, 4)
    rng = np.random.default_rng(1)
    pick = [dets[i] for i in rng.choice(len(dets), 5, replace=False)]
    _check_generator(orc, 1, pick, nsamples=20000)
    for d in pick:
        _connected_reachable(orc, 1, d, dets)


def test_ueg_generator_probabilities():
    sysd = inputs.ueg_system(nel=4, norb=7, rs=1.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets = B.determinants(7, 2, 2)
    rng = np.random.default_rng(2)
    pick = [dets[i] for i in rng.choice(len(dets), 5, replace=False)]
    _check_generator(orc, 1, pick, nsamples=20000)
    for d in pick:
        _connected_reachable(orc, 1, d, dets)


def test_heat_bath_generator_probabilities():
    h1, eri = inputs.molecule_integrals(6, seed=4)
    sysd = {"kind": "molecule", "key_words": 1, "norb": 6, "nalpha": 2, "nbeta": 2,
            "h1": h1, "eri": eri, "ecore": 0.0}
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    dets = B.determinants(6, 2, 2)
    rng = np.random.default_rng(3)
    pick = [dets[i] for i in rng.choice(len(dets), 5, replace=False)]
    _check_generator(orc, 1, pick, nsamples=20000)
    for d in pick:
        _connected_reachable(orc, 1, d, dets)


def test_generator_uses_128_bit_keys():
    """UEG 14e / 38 orbitals: 76 spin orbitals need two key words."""
    sysd = inputs.ueg_system(14, 38, 1.0)
    assert sysd["key_words"] == 2
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    d0 = orc.reference()
    children, probs = orc.enumerate(d0)
    assert abs(probs.sum() - 1.0) < 1e-12
    rng = np.random.default_rng(5)
    seen = 0
    for _ in range(300):
        w = rng.integers(0, 2**64 - 1, size=4, dtype=np.uint64, endpoint=True)
        r = orc.generate(d0, w)
        if r is None:
            continue
        seen += 1
        assert orc.hij(d0, r[0]) == r[2]
    assert seen > 0


def _spin_eri(eri, p, q, r, s):
    """(pq|rs) over spin orbitals (spin orbital = 2 * spatial + spin)."""
    if (p & 1) != (q & 1) or (r & 1) != (s & 1):
        return 0.0
    return float(eri[p >> 1, q >> 1, r >> 1, s >> 1])


@pytest.mark.parametrize("norb,seed,pairs", [(6, 4, None), (28, 11, 40)])
def test_heat_bath_table_weights_are_antisymmetrised_integrals(norb, seed, pairs):
    """The heat-bath reading: the table of an occupied pair (p < q) lists every
    spin-allowed (a < b) outside {p, q} with w = |(pa|qb) - (pb|qa)| > 0 in
    ascending (a, b) order, and entry k is drawn with probability w_k / sum w.
    The weights are recomputed here from the integrals alone (a swapped index
    or a dropped exchange term changes them), and the drawn probabilities are
    the widths of the oracle's cumulative 64-bit thresholds."""
    h1, eri = inputs.molecule_integrals(norb, seed=seed)
    sysd = {"kind": "molecule", "key_words": 1, "norb": norb, "nalpha": 3, "nbeta": 2,
            "h1": h1, "eri": eri, "ecore": 0.0}
    orc = oracle.Oracle(sysd, inputs.qmc_params())
    ns = 2 * norb
    allp = [(p, q) for q in range(1, ns) for p in range(q)]
    if pairs is not None:
        rng = np.random.default_rng(seed)
        allp = [allp[i] for i in rng.choice(len(allp), pairs, replace=False)]
    two64 = 2.0 ** 64
    for p, q in allp:
        want_ab, want_w = [], []
        for a in range(ns):
            for b in range(a + 1, ns):
                if a in (p, q) or b in (p, q):
                    continue
                ok = ((a & 1) == (p & 1) and (b & 1) == (q & 1)) or ((a & 1) == (q & 1) and (b & 1) == (p & 1))
                if not ok:
                    continue
                w = abs(_spin_eri(eri, p, a, q, b) - _spin_eri(eri, p, b, q, a))
                if w > 0.0:
                    want_ab.append((a, b))
                    want_w.append(w)
        ta, tb, cum = orc.heat_bath_table(p, q)
        assert list(zip(ta.tolist(), tb.tolist())) == want_ab, (p, q)
        m = len(want_w)
        if m == 0:
            continue
        if m == 1:
            continue   # a single entry is drawn with probability 1
        c = [int(x) for x in cum[:-1]]
        widths = [c[0]] + [c[k] - c[k - 1] for k in range(1, m - 1)] + [(1 << 64) - c[-1]]
        assert all(wd > 0 for wd in widths)
        got = np.array(widths, dtype=np.float64) / two64
        want = np.array(want_w) / np.sum(want_w)
        tol = (m + 4) * 2.0 ** -52
        assert np.max(np.abs(got - want)) <= tol, (p, q, np.max(np.abs(got - want)))
