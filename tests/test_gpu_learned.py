"""The learned excitation proposal on the GPU (UEG).

* The proposal-table generator is the same arithmetic on both sides: given the
  same integer table, GPU walker lists equal the oracle's bit for bit.
* The MLP's BF16 tensor-core forward and backward (tcgen05 GEMMs) against the
  oracle's FP64 MLP with the same BF16 rounding points: probabilities, loss and
  every gradient tensor within the FP32-accumulation tolerance; the table the
  GPU derives from the network against the oracle's.
* Online training on the run's own spawning attempts moves the table toward
  the heat-bath distribution (proportional to |H|), computed here in closed form.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1811_11679_gb300 import hande, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _same_lists(g, c, it):
    kg, pg, hg, _ = g.walkers()
    kc, pc, hc, _ = c.walkers()
    assert kg.shape == kc.shape, f"iteration {it}: {len(kg)} vs {len(kc)}"
    assert np.array_equal(kg, kc), f"iteration {it}: keys differ"
    assert np.array_equal(pg, pc), f"iteration {it}: populations differ"
    assert np.array_equal(hg.view(np.int64), hc.view(np.int64))


@pytest.mark.parametrize("norb,kw", [(19, 1), (38, 2), (38, 8)])
def test_table_generator_bit_parity(norb, kw):
    sysd = inputs.ueg_system(14, norb, 1.0, key_words=kw)
    q = inputs.qmc_params(tau=0.002, target_population=20000, initiator=1, real_amplitudes=1, spawn_cutoff=0.1,
                          init_pop=1000, seed=7, excit_gen=1)
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    table = inputs.random_proposal(c.proposal_mask(), seed=norb + kw)
    g.set_proposal(table)
    c.set_proposal(table)
    assert np.array_equal(g.proposal(), table)
    for it in range(60):
        g.iterate(1)
        c.iterate(1)
        _same_lists(g, c, it + 1)
    eg, ec = g.estimators(), c.records()
    for k in ("nw_pre", "n0", "num_hi", "num_lo", "nw_post", "ndet", "natt", "nspawn"):
        assert np.array_equal(eg[k], ec[k]), k
    g.close()


def _oracle_params(flat, M, H):
    din = 2 * M + 1
    o = 0
    out = {}
    for k, shape in (("W1", (H, din)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (M, H)), ("b3", (M,))):
        n = int(np.prod(shape))
        out[k] = flat[o:o + n].astype(np.float64).reshape(shape)
        o += n
    assert o == len(flat)
    return out


def _learner(norb=38, width=256, batch=512, seed=3):
    sysd = inputs.ueg_system(14, norb, 1.0)
    q = inputs.qmc_params(tau=0.002, target_population=1e5, initiator=1, real_amplitudes=1, spawn_cutoff=0.1,
                          init_pop=1000, seed=7, excit_gen=1)
    g = hande.Hande(sysd, q)
    g.learn_proposal(width=width, batch=batch, period=0, seed=seed)
    c = oracle.Oracle(sysd, q)
    return g, c, sysd


def test_mlp_forward_and_gradients_match_the_oracle():
    M, H = 38, 256
    g, c, _ = _learner()
    mask_all = c.proposal_mask()
    params = mlp.init_params(M, H, seed=11)
    rng = np.random.default_rng(5)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.normal(0, 0.2, params[k].shape)
    flat = np.concatenate([params[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)
    back = g.learn_params(flat)
    assert np.array_equal(g.learn_params(), flat) and np.array_equal(back, flat)
    P = _oracle_params(flat, M, H)          # the float32 values both sides use
    usable = np.nonzero(mask_all.any(axis=1))[0]
    n = 300
    rows = rng.choice(usable, n).astype(np.int32)
    mask = mask_all[rows]
    tgt = np.array([rng.choice(np.nonzero(m)[0]) for m in mask], dtype=np.int32)
    w = rng.uniform(0.05, 3.0, n).astype(np.float32)
    X = mlp.features(rows, M)
    # forward: masked softmax probabilities
    pg = g.learn_probabilities(rows).astype(np.float64)
    po = mlp.forward(P, X, mask, bf=True)["p"]
    assert np.max(np.abs(pg - po)) < 2e-3, np.max(np.abs(pg - po))
    assert np.all(pg[~mask] == 0.0)
    assert np.allclose(pg.sum(axis=1), 1.0, atol=1e-5)
    # loss and gradients
    lg, gg = g.learn_gradients(rows, tgt, w)
    lo, go = mlp.loss_and_grads(P, X, mask, tgt, w.astype(np.float64), bf=True)
    assert abs(lg - lo) <= 1e-3 * abs(lo), (lg, lo)
    G = _oracle_params(gg, M, H)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.linalg.norm(G[k] - go[k]) / max(np.linalg.norm(go[k]), 1e-30)
        assert err < 2e-2, (k, err)
    # the same gradients without any BF16 rounding (plain FP64): close, not equal
    _, g64 = mlp.loss_and_grads(P, X, mask, tgt, w.astype(np.float64), bf=False)
    for k in ("W1", "W2", "W3"):
        err = np.linalg.norm(G[k] - g64[k]) / max(np.linalg.norm(g64[k]), 1e-30)
        assert err < 0.1, (k, err)
    g.close()


def test_table_from_the_network_matches_the_oracle():
    M, H = 38, 256
    g, c, _ = _learner()
    mask = c.proposal_mask()
    params = mlp.init_params(M, H, seed=12)
    flat = np.concatenate([params[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)
    g.learn_params(flat)
    g.learn_refresh()
    qg = g.proposal().astype(np.float64)
    P = _oracle_params(flat, M, H)
    po = mlp.forward(P, mlp.features(np.arange(2 * M * M), M), mask, bf=True)["p"]
    qo = mlp.table_from_probabilities(po, mask).astype(np.float64)
    assert np.array_equal(qg > 0, mask)                      # weight exactly on the drawable orbitals
    assert np.all(qg <= 2 ** 24)
    rel = np.abs(qg - qo) / np.maximum(qo, 2 ** 14)
    assert np.max(rel[mask]) < 2e-2, np.max(rel[mask])
    # the table is a valid proposal for the oracle's generator as well
    c.set_proposal(qg.astype(np.uint32))
    g.close()


def _heat_bath_rows(c, M):
    """|H| of every drawable (row, A): |v(k_I - k_A) - [same] v(k_I - k_B)|, v = 1/|dn|^2
    (the common factor 4 pi / Omega cancels in the normalised distribution)."""
    kv, _ = c.ueg_basis()
    index = {tuple(k): i for i, k in enumerate(kv.tolist())}
    mask = c.proposal_mask()
    Hm = np.zeros(mask.shape)
    for r in range(2 * M * M):
        same, IJ = r & 1, r >> 1
        I, J = IJ // M, IJ % M
        for A in np.nonzero(mask[r])[0]:
            B = index[tuple(kv[I] + kv[J] - kv[A])]
            dA = int(np.sum((kv[I] - kv[A]) ** 2))
            dB = int(np.sum((kv[I] - kv[B]) ** 2))
            d = 1.0 / dA if dA else 0.0
            e = (1.0 / dB if dB else 0.0) if same else 0.0
            Hm[r, A] = abs(d - e)
    return Hm, mask


def test_online_training_learns_the_heat_bath_distribution():
    """A run with online training (one Adam step every 2 iterations on the
    attempts it draws): the KL divergence from the heat-bath distribution to
    the table, averaged over the rows the run visits, falls well below that of
    the uniform starting table."""
    M = 38
    sysd = inputs.ueg_system(14, M, 1.0)
    q = inputs.qmc_params(tau=0.002, target_population=1e5, initiator=1, real_amplitudes=1, spawn_cutoff=0.1,
                          init_pop=20000, seed=7, excit_gen=1)
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    Hm, mask = _heat_bath_rows(c, M)
    target = Hm / np.maximum(Hm.sum(axis=1, keepdims=True), 1e-300)

    # rows of pairs among the reference's occupied orbitals (the run visits them most)
    occ = np.arange(7)
    visited = np.zeros(2 * M * M, dtype=bool)
    for I in occ:
        for J in occ:
            visited[(I * M + J) * 2:(I * M + J) * 2 + 2] = True

    def kl(table):
        p = table / np.maximum(table.sum(axis=1, keepdims=True), 1)
        keep = visited & (Hm.sum(axis=1) > 0) & mask.any(axis=1)
        t, pp = target[keep], p[keep]
        m = t > 0
        return float(np.sum(np.where(m, t * np.log(np.where(m, t, 1) / np.where(m, pp, 1)), 0)) / keep.sum())

    uniform = mask.astype(np.float64)
    g.learn_proposal(width=256, batch=4096, period=2, learning_rate=3e-3, seed=1)
    before = kl(g.proposal().astype(np.float64))
    g.iterate(400)
    g.synchronize()
    after = kl(g.proposal().astype(np.float64))
    assert after < 0.5 * kl(uniform), (kl(uniform), before, after)
    assert after < 0.5 * before, (before, after)
    g.close()
