"""The full oracle iteration pinned against exact diagonalisation (deterministic
limit and stochastic runs), the blocking analysis against an AR(1) closed form,
and invariants of the walker list."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import inputs
import _brute as B
import _stats as S

F = 2 ** 32


def test_blocking_reproduces_ar1_error():
    """AR(1) x_t = phi x_{t-1} + e_t: var(mean) = sigma^2/(1-phi^2)/n (1+phi)/(1-phi)."""
    rng = np.random.default_rng(0)
    phi, n = 0.9, 2 ** 16
    e = rng.normal(size=n)
    x = np.zeros(n)
    for i in range(1, n):
        x[i] = phi * x[i - 1] + e[i]
    true = np.sqrt(1.0 / (1.0 - phi ** 2) / n * (1.0 + phi) / (1.0 - phi))
    _, err = S.optimal_error(x)
    assert abs(err - true) < 0.1 * true


def _mol_small():
    h1, eri = inputs.molecule_integrals(6, seed=4)
    return {"kind": "molecule", "key_words": 1, "norb": 6, "nalpha": 2, "nbeta": 2, "h1": h1,
            "eri": eri, "ecore": 0.0}, h1, eri


def _deterministic_limit(sysd, dets, E0, tau, iters, W=1, seed=1):
    """Core = the whole space, taken from the initial list (start_iteration 0):
    the propagation 1 - tau (H - E_ref - S) is then applied exactly, so E_proj
    and E_ref + S converge to the ground-state energy."""
    rng = np.random.default_rng(seed)
    keys = np.array([B.bits_to_words(d, W) for d in dets], dtype=np.uint64)
    pops = (rng.integers(F // 10, F // 3, len(dets)) * rng.choice([-1, 1], len(dets))).astype(np.int64)
    q = inputs.qmc_params(tau=tau, target_population=0.5 * np.abs(pops).sum() / F,
                          real_amplitudes=1, spawn_cutoff=0.01, semi_stoch_size=len(dets),
                          semi_stoch_start=0, shift_damping=0.5, seed=seed)
    orc = oracle.Oracle(sysd, q)
    d0 = B.words_to_bits(orc.reference())
    pops[dets.index(d0)] = 5 * F
    orc.set_walkers(keys, pops)
    assert len(orc.core()) == len(dets)
    orc.iterate(iters)
    r = orc.records()
    eproj = orc.e_ref + r["num"][-1] / r["n0"][-1]
    return eproj, orc.e_ref + r["shift"][-1], orc


def test_deterministic_limit_hubbard8():
    dets, H = B.hubbard_hamiltonian(8, 4, 4, 1.0, 4.0, True)
    E0 = np.linalg.eigvalsh(H)[0]
    ep, es, _ = _deterministic_limit(inputs.hubbard_system(), dets, E0, 0.05, 2000)
    assert abs(ep - E0) < 1e-8
    assert abs(es - E0) < 1e-6


def test_deterministic_limit_molecule():
    sysd, h1, eri = _mol_small()
    dets, H = B.molecule_hamiltonian(h1, eri, 2, 2)
    E0 = np.linalg.eigvalsh(H)[0]
    ep, es, _ = _deterministic_limit(sysd, dets, E0, 0.3, 2500)
    assert abs(ep - E0) < 1e-8
    assert abs(es - E0) < 1e-6


def test_deterministic_limit_ueg():
    sysd = inputs.ueg_system(nel=2, norb=19, rs=1.0)
    dets, H, _, _ = B.ueg_hamiltonian(19, 1, 1, 1.0)
    # restrict to the zero-momentum sector connected to the reference
    kv = B.ueg_basis(19)
    zero = [d for d in dets if not np.any(sum(kv[p >> 1] for p in range(38) if (d >> p) & 1))]
    idx = [dets.index(d) for d in zero]
    Hs = H[np.ix_(idx, idx)]
    E0 = np.linalg.eigvalsh(Hs)[0]
    ep, es, _ = _deterministic_limit(sysd, zero, E0, 0.02, 3000)
    assert abs(ep - E0) < 1e-8
    assert abs(es - E0) < 1e-6


def _stochastic(sysd, q, iters, start):
    orc = oracle.Oracle(sysd, q)
    orc.iterate(iters)
    r = orc.records()
    m, err = S.ratio_estimate(r["num"][start:], r["n0"][start:])
    return orc.e_ref + m, err, orc, r


def test_stochastic_molecule_within_two_sigma():
    sysd, h1, eri = _mol_small()
    dets, H = B.molecule_hamiltonian(h1, eri, 2, 2)
    E0 = np.linalg.eigvalsh(H)[0]
    q = inputs.qmc_params(tau=0.02, target_population=2000, real_amplitudes=1,
                          spawn_cutoff=0.01, init_pop=50, seed=3)
    e, err, orc, r = _stochastic(sysd, q, 4000, 500)
    assert abs(e - E0) < 2.0 * err, (e, err, E0)
    assert err < 0.05


def test_stochastic_hubbard8_integer_walkers():
    """The Hubbard ring workload itself (integer walkers, tau 0.01, target 1e4)."""
    dets, H = B.hubbard_hamiltonian(8, 4, 4, 1.0, 4.0, True)
    E0 = np.linalg.eigvalsh(H)[0]
    sysd, q = inputs.workload("hubbard8")
    e, err, orc, r = _stochastic(sysd, q, 2000, 300)
    assert abs(e - E0) < 2.0 * err, (e, err, E0)
    # shift estimator: E_ref + <S>
    ms, es = S.optimal_error(r["shift"][300:])
    assert abs(orc.e_ref + ms - E0) < 2.0 * es + 0.01   # + population-control bias allowance
    # integer walkers: every population is a whole number of walkers
    _, pops, _, _ = orc.walkers()
    assert np.all(pops % F == 0)


def test_stochastic_ueg_initiator_converges():
    """UEG, 1 up + 1 down in 19 orbitals with the initiator rule: the initiator
    error vanishes once the population is large, so E_proj meets exact FCI."""
    sysd = inputs.ueg_system(nel=2, norb=19, rs=1.0)
    dets, H, _, _ = B.ueg_hamiltonian(19, 1, 1, 1.0)
    E0 = np.linalg.eigvalsh(H)[0]
    q = inputs.qmc_params(tau=0.01, target_population=3000, real_amplitudes=1,
                          spawn_cutoff=0.05, initiator=1, initiator_threshold=3.0, init_pop=50,
                          seed=5)
    e, err, orc, r = _stochastic(sysd, q, 3000, 500)
    assert abs(e - E0) < 2.0 * err, (e, err, E0)


def test_walker_list_invariants():
    sysd, q = inputs.workload("ueg14", target_population=3000)
    orc = oracle.Oracle(sysd, q)
    d0 = orc.reference()
    for _ in range(6):
        orc.iterate(10)
        keys, pops, hd, fl = orc.walkers()
        r = orc.records()
        # sorted strictly ascending as big integers (word 1 most significant)
        big = [B.words_to_bits(k) for k in keys]
        assert all(a < b for a, b in zip(big, big[1:]))
        # the reference stays in the list; every other entry is nonzero and >= 1 walker
        is0 = np.all(keys == d0, axis=1)
        assert is0.sum() == 1
        assert np.all(np.abs(pops[~is0]) >= F)
        # recorded population equals the list
        assert r["nw_post"][-1] == np.abs(pops).sum()
        assert r["ndet"][-1] == len(pops)
        # cached diagonal equals H_ii - E_ref
        for i in range(0, len(keys), max(1, len(keys) // 20)):
            assert hd[i] == orc.hdiag(keys[i]) - orc.e_ref


def test_runs_are_reproducible_and_seeded():
    sysd, q = inputs.workload("hubbard8")
    a = oracle.Oracle(sysd, q)
    b = oracle.Oracle(sysd, q)
    c = oracle.Oracle(sysd, dict(q, seed=9))
    for o in (a, b, c):
        o.iterate(50)
    ka, pa, _, _ = a.walkers()
    kb, pb, _, _ = b.walkers()
    kc, pc, _, _ = c.walkers()
    assert np.array_equal(ka, kb) and np.array_equal(pa, pb)
    assert not (len(ka) == len(kc) and np.array_equal(ka, kc) and np.array_equal(pa, pc))


def test_initiator_blocks_new_determinants_from_non_initiators():
    """With an unreachable threshold only D0 is an initiator: every determinant
    added in an iteration is either already occupied or connected to D0."""
    sysd, q = inputs.workload("ueg14", target_population=1e9, initiator_threshold=1e12)
    orc = oracle.Oracle(sysd, q)
    d0 = orc.reference()
    orc.iterate(5)
    for _ in range(5):
        k_before, _, _, _ = orc.walkers()
        before = {B.words_to_bits(k) for k in k_before}
        orc.iterate(1)
        k_after, _, _, _ = orc.walkers()
        for k in k_after:
            kb = B.words_to_bits(k)
            if kb in before:
                continue
            assert bin(kb ^ B.words_to_bits(d0)).count("1") <= 4


def test_shift_held_until_target_then_varies():
    sysd, q = inputs.workload("hubbard8", target_population=2000)
    orc = oracle.Oracle(sysd, q)
    orc.iterate(400)
    r = orc.records()
    over = np.nonzero(r["nw_post"] > 2000 * F)[0]
    assert len(over) > 0
    t0 = over[0]
    assert np.all(r["shift"][: t0 + 1] == 0.0)
    assert np.any(r["shift"][t0 + 1:] != 0.0)


def test_semi_stochastic_core_is_highest_population_space():
    sysd, q = inputs.workload("ueg14", target_population=5000, semi_stoch_size=50,
                              semi_stoch_start=60)
    orc = oracle.Oracle(sysd, q)
    orc.iterate(60)
    keys, pops, _, fl = orc.walkers()
    d0 = orc.reference()
    core = orc.core()
    assert len(core) == 50
    big = [B.words_to_bits(k) for k in keys]
    is0 = np.array([b == B.words_to_bits(d0) for b in big])
    order = sorted([i for i in range(len(big)) if not is0[i]], key=lambda i: (-abs(int(pops[i])), big[i]))
    want = sorted([big[i] for i in order[:49]] + [B.words_to_bits(d0)])
    assert [B.words_to_bits(k) for k in core] == want
    assert fl.sum() == 50
    # core determinants stay in the list from then on
    orc.iterate(30)
    keys2, _, _, fl2 = orc.walkers()
    s2 = {B.words_to_bits(k) for k, f in zip(keys2, fl2) if f & 1}
    assert s2 == set(want)
