"""Pins of the learned excitation proposal's oracle half (CPU).

The proposal-table generator (UEG doubles: uniform occupied pair, particle
orbital A from the integer weights of row (I, J, same spin), b by momentum
conservation) is pinned like the other generators: the probabilities of all
selection paths sum to one, the reported p_gen equals the summed path
probability, every nonzero H_ij is reachable, sampled frequencies pass a chi^2
test, and an FCIQMC run with it meets exact diagonalisation within two
blocking standard errors.  The FP64 MLP (oracle/mlp.py) is pinned by central
finite differences of its loss and by the closed form of a zero network."""
from __future__ import annotations

import numpy as np
import pytest

import _brute as B
import _stats as S
import oracle
from oracle import mlp
from paper_1811_11679_gb300 import inputs
from test_oracle_pins import _check_generator, _connected_reachable


def _random_table(orc, seed):
    mask = orc.proposal_mask()
    rng = np.random.Generator(np.random.Philox(seed))
    q = rng.integers(1, 1 << 24, size=mask.shape, endpoint=True).astype(np.uint32)
    return np.where(mask, q, 0).astype(np.uint32), mask


def test_table_generator_probabilities_and_ergodicity():
    sysd = inputs.ueg_system(nel=4, norb=7, rs=1.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params(excit_gen=1))
    q, _ = _random_table(orc, 4)
    orc.set_proposal(q)
    dets = B.determinants(7, 2, 2)
    rng = np.random.default_rng(6)
    pick = [dets[i] for i in rng.choice(len(dets), 5, replace=False)]
    _check_generator(orc, 1, pick, nsamples=20000)
    for d in pick:
        _connected_reachable(orc, 1, d, dets)


def test_table_generator_rejects_tables_that_break_ergodicity():
    sysd = inputs.ueg_system(nel=4, norb=7, rs=1.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params(excit_gen=1))
    q, mask = _random_table(orc, 5)
    bad = q.copy()
    r, a = np.argwhere(mask)[3]
    bad[r, a] = 0                      # a drawable orbital with weight 0
    with pytest.raises(ValueError):
        orc.set_proposal(bad)
    bad = q.copy()
    r, a = np.argwhere(~mask)[0]
    bad[r, a] = 1                      # weight on an orbital whose partner is outside the basis
    with pytest.raises(ValueError):
        orc.set_proposal(bad)


def test_table_generator_run_meets_exact_diagonalisation():
    """1 up + 1 down electron in 19 plane waves, a random table: E_proj within
    two blocking errors of the ground state of the zero-momentum sector."""
    sysd = inputs.ueg_system(nel=2, norb=19, rs=1.0)
    dets, H, _, _ = B.ueg_hamiltonian(19, 1, 1, 1.0)
    E0 = np.linalg.eigvalsh(H)[0]
    q = inputs.qmc_params(tau=0.01, target_population=2000, real_amplitudes=1, spawn_cutoff=0.05,
                          init_pop=50, seed=9, excit_gen=1)
    orc = oracle.Oracle(sysd, q)
    t, _ = _random_table(orc, 7)
    orc.set_proposal(t)
    orc.iterate(3000)
    r = orc.records()
    m, err = S.ratio_estimate(r["num"][500:], r["n0"][500:])
    assert abs(orc.e_ref + m - E0) < 2.0 * err, (orc.e_ref + m, err, E0)


def _tiny_problem(seed=1, M=7, width=16, n=40):
    sysd = inputs.ueg_system(nel=4, norb=M, rs=1.0)
    orc = oracle.Oracle(sysd, inputs.qmc_params(excit_gen=1))
    mask_all = orc.proposal_mask()
    rng = np.random.default_rng(seed)
    usable = np.nonzero(mask_all.any(axis=1))[0]
    rows = rng.choice(usable, n)
    mask = mask_all[rows]
    target = np.array([rng.choice(np.nonzero(mk)[0]) for mk in mask])
    weight = rng.uniform(0.1, 2.0, n)
    params = mlp.init_params(M, width, seed)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.normal(0, 0.1, params[k].shape)
    return params, mlp.features(rows, M), mask, target, weight


def test_mlp_backward_matches_finite_differences():
    params, X, mask, target, weight = _tiny_problem()
    _, g = mlp.loss_and_grads(params, X, mask, target, weight)
    rng = np.random.default_rng(2)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in params[k].shape)
            pp = {a: b.copy() for a, b in params.items()}
            pm = {a: b.copy() for a, b in params.items()}
            pp[k][idx] += h
            pm[k][idx] -= h
            fd = (mlp.loss_and_grads(pp, X, mask, target, weight)[0]
                  - mlp.loss_and_grads(pm, X, mask, target, weight)[0]) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 + 1e-5 * abs(fd), (k, idx, fd, g[k][idx])


def test_zero_network_is_uniform_over_drawable_orbitals():
    params, X, mask, target, weight = _tiny_problem()
    for k in params:
        params[k] = np.zeros_like(params[k])
    f = mlp.forward(params, X, mask)
    cnt = mask.sum(axis=1, keepdims=True)
    assert np.allclose(f["p"], mask / cnt, rtol=0, atol=1e-15)
    loss, g = mlp.loss_and_grads(params, X, mask, target, weight)
    c = weight / weight.sum()
    assert abs(loss - float(np.sum(c * np.log(cnt[:, 0])))) < 1e-12
    onehot = np.zeros_like(f["p"])
    onehot[np.arange(len(target)), target] = 1.0
    assert np.allclose(g["b3"], (c[:, None] * (mask / cnt - onehot)).sum(axis=0), atol=1e-15)
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0) and np.all(g["W3"] == 0)


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -2.5, 3.0e38, 1e-40])
    got = mlp.bf16(x)
    # BF16 keeps 7 fraction bits: next to 1 is 1 + 2^-7.  1 + 2^-8 is the tie ->
    # 1 (even); 1 + 2^-9 -> 1; 1 + 3 2^-9 is above the tie -> 1 + 2^-7; -2.5 exact
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 and got[3] == 1.0 + 2 ** -7
    assert got[4] == -2.5
    # relative error at most half a unit (2^-8), subnormals to half their spacing 2^-133
    assert np.all(np.abs(got - x) <= np.abs(x) * 2 ** -8 + 2.0 ** -134)
