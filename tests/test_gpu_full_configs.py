"""Parity at the full sizes of the learned-proposal and batched configurations.

* Learned proposal, full basis: UEG 54 electrons in 246 plane waves (492 spin
  orbitals, 512-bit keys).  Given the same integer proposal table, the GPU
  walker lists equal the oracle's bit for bit on a synthetic list; the table
  the GPU derives from the network (BF16 tensor-core forward over all
  2 x 246^2 rows) and the loss gradients agree with the oracle's FP64 MLP on
  sampled rows.
* Batched replicas, all 256 (`inputs.batched_replicas(256)`): a sample of the
  replicas (the largest and smallest targets, both key widths, seeded picks)
  equals the oracle's runs of the same (system, qmc) pairs bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1811_11679_gb300 import hande, inputs
from test_gpu_parity import _same_lists, _same_records

pytestmark = pytest.mark.gpu

M_FULL = 246


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _full_basis(**over):
    sysd = inputs.ueg_system(54, M_FULL, 1.0)
    assert sysd["key_words"] == 8
    q = inputs.qmc_params(tau=0.002, target_population=1e7, initiator=1, real_amplitudes=1, spawn_cutoff=0.1,
                          init_pop=1000, seed=7, excit_gen=1, state_capacity=4_000_000,
                          spawn_capacity=4_000_000)
    q.update(over)
    return sysd, q


def test_full_basis_table_generator_bit_parity():
    sysd, q = _full_basis()
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    mask = c.proposal_mask()
    assert mask.shape == (2 * M_FULL * M_FULL, M_FULL)
    table = inputs.random_proposal(mask, seed=31)
    g.set_proposal(table)
    c.set_proposal(table)
    keys, pops = inputs.synthetic_walkers(sysd, 20000, 2e5, seed=4)
    g.set_walkers(keys, pops)
    c.set_walkers(keys, pops)
    for it in range(3):
        g.iterate(1)
        c.iterate(1)
        _same_lists(g, c, it + 1)
    _same_records(g, c)
    assert g.diagnostics()["nspawn"] > 100_000
    g.close()


def _flat(params):
    return np.concatenate([params[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def _unflat(flat, M, H):
    out, o = {}, 0
    for k, shape in (("W1", (H, 2 * M + 1)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (M, H)),
                     ("b3", (M,))):
        n = int(np.prod(shape))
        out[k] = flat[o:o + n].astype(np.float64).reshape(shape)
        o += n
    assert o == len(flat)
    return out


def test_full_basis_network_table_and_gradients_on_sampled_rows():
    H = 256
    sysd, q = _full_basis()
    g = hande.Hande(sysd, q)
    g.learn_proposal(width=H, batch=512, period=0, seed=3)
    c = oracle.Oracle(sysd, q)
    mask_all = c.proposal_mask()
    params = mlp.init_params(M_FULL, H, seed=13)
    rng = np.random.default_rng(17)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.normal(0, 0.2, params[k].shape)
    flat = _flat(params)
    g.learn_params(flat)
    P = _unflat(flat, M_FULL, H)
    usable = np.nonzero(mask_all.any(axis=1))[0]
    rows = np.sort(rng.choice(usable, 2000, replace=False)).astype(np.int32)
    mask = mask_all[rows]
    X = mlp.features(rows, M_FULL)
    # the table over all rows, compared on the sampled ones
    g.learn_refresh()
    qg = g.proposal()
    assert qg.shape == mask_all.shape
    assert np.array_equal(qg > 0, mask_all)
    po = mlp.forward(P, X, mask, bf=True)["p"]
    qo = mlp.table_from_probabilities(po, mask).astype(np.float64)
    qs = qg[rows].astype(np.float64)
    assert np.all(qs <= 2 ** 24)
    rel = np.abs(qs - qo) / np.maximum(qo, 2 ** 14)
    assert np.max(rel[mask]) < 2e-2, np.max(rel[mask])
    # probabilities, loss and gradients on a sampled batch
    n = 300
    b = rows[:n]
    bm = mask_all[b]
    tgt = np.array([rng.choice(np.nonzero(m)[0]) for m in bm], dtype=np.int32)
    w = rng.uniform(0.05, 3.0, n).astype(np.float32)
    Xb = mlp.features(b, M_FULL)
    pg = g.learn_probabilities(b).astype(np.float64)
    pb = mlp.forward(P, Xb, bm, bf=True)["p"]
    assert np.max(np.abs(pg - pb)) < 2e-3, np.max(np.abs(pg - pb))
    assert np.all(pg[~bm] == 0.0)
    lg, gg = g.learn_gradients(b, tgt, w)
    lo, go = mlp.loss_and_grads(P, Xb, bm, tgt, w.astype(np.float64), bf=True)
    assert abs(lg - lo) <= 1e-3 * abs(lo), (lg, lo)
    G = _unflat(gg, M_FULL, H)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.linalg.norm(G[k] - go[k]) / max(np.linalg.norm(go[k]), 1e-30)
        assert err < 2e-2, (k, err)
    g.close()


def test_all_256_batched_replicas_sampled_against_the_oracle():
    systems, qmcs = inputs.batched_replicas(256)
    targets = np.array([q["target_population"] for q in qmcs])
    rng = np.random.default_rng(23)
    pick = sorted({int(np.argmax(targets)), int(np.argmin(targets)), 0, 1,
                   *[int(x) for x in rng.choice(256, 4, replace=False)]})
    assert {systems[r]["key_words"] for r in pick} == {2, 8}
    b = hande.HandeBatch(systems, qmcs)
    assert len(b) == 256
    cs = {r: oracle.Oracle(systems[r], qmcs[r]) for r in pick}
    for step in (1, 3):
        b.iterate(step)
        for r in pick:
            cs[r].iterate(step)
            _same_lists(b.replicas[r], cs[r], f"{b.replicas[r].iterations} (replica {r})")
    for r in pick:
        _same_records(b.replicas[r], cs[r])
    assert all(v.iterations == 4 for v in b.replicas)
    b.close()


def test_benchmark_state_two_iterations_against_the_oracle():
    """The headline workload as the bench times it (28-orbital molecule, 1e7
    target walkers, deterministic space of 1e4 chosen at iteration 2000, the
    bench's capacities and launch configuration): grown on the GPU to iteration
    2060, its list and run state handed to the oracle (all host cores), then two
    more iterations on both sides compared element by element."""
    import os
    sysd, q = inputs.workload("molecule28", target_population=1e7, semi_stoch_size=10000, semi_stoch_start=2000,
                              state_capacity=16_000_000, spawn_capacity=32_000_000)
    g = hande.Hande(sysd, q)
    while g.iterations < 2060:
        g.iterate(min(250, 2060 - g.iterations))
    keys, pops, _, _ = g.walkers()
    state, core = g.state()
    assert len(pops) > 2_000_000 and state["core_active"] == 1 and len(core) == 10000
    assert g.diagnostics()["nbuckets"] > 4096
    g.estimators()
    c = oracle.Oracle(sysd, q, threads=os.cpu_count())
    c.set_walkers(keys, pops)
    c.set_state(state, core)
    for it in range(2):
        g.iterate(1)
        c.iterate(1)
        _same_lists(g, c, 2061 + it)
    rg, rc = g.estimators(), c.records()
    n = len(rc["iter"])
    assert n == 2 and len(rg["iter"]) == 2
    for k in ("iter", "nw_pre", "n0", "num_hi", "num_lo", "nw_post", "ndet", "natt", "nspawn"):
        assert np.array_equal(rg[k], rc[k][-n:]), k
    assert np.array_equal(rg["shift"].view(np.int64), rc["shift"][-n:].view(np.int64))
    g.close()
