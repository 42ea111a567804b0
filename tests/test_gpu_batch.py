"""Batched replicas (include/hande.h, batches) against the CPU oracle: every
replica of a mixed batch -- different systems, key widths, seeds, replica words,
walker modes and a deterministic space chosen mid-run -- gives, bit for bit, the
walker lists and estimator records of the oracle's run with its parameters."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import hande, inputs
from test_gpu_parity import _same_lists, _same_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _mixed_replicas():
    runs = []
    s, q = inputs.workload("hubbard8")
    runs.append((s, q))
    runs.append((s, dict(q, replica=1)))
    runs.append((s, dict(q, seed=9)))
    runs.append(inputs.workload("ueg14", target_population=20000, init_pop=1000))
    runs.append((inputs.ueg_system(14, 19, 2.0),
                 inputs.qmc_params(tau=0.005, target_population=5000, initiator=1, real_amplitudes=1,
                                   spawn_cutoff=0.1, init_pop=100, seed=11)))
    runs.append(inputs.workload("molecule28", target_population=30000, semi_stoch_size=300,
                                semi_stoch_start=40))
    return runs


def test_mixed_batch_equals_oracle_per_replica():
    runs = _mixed_replicas()
    b = hande.HandeBatch([s for s, _ in runs], [q for _, q in runs])
    assert len(b) == len(runs)
    cs = [oracle.Oracle(s, q) for s, q in runs]
    for g, c in zip(b.replicas, cs):
        e, k = g.reference()
        assert e == c.e_ref and np.array_equal(k, c.reference())
    done = 0
    for step in (1, 29, 30, 40):
        b.iterate(step)
        for c in cs:
            c.iterate(step)
        done += step
        for r, (g, c) in enumerate(zip(b.replicas, cs)):
            assert g.iterations == done
            _same_lists(g, c, f"{done} (replica {r})")
    for g, c in zip(b.replicas, cs):
        _same_records(g, c)
    assert 0 < b.replicas[-1].diagnostics()["ncore"] <= 300   # core flags already compared per list
    k0, p0 = b.replicas[0].walkers()[:2]
    k1, p1 = b.replicas[1].walkers()[:2]
    assert not (np.array_equal(k0, k1) and np.array_equal(p0, p1))
    b.synchronize()
    b.close()


def test_batch_replica_equals_single_run_and_advances_alone():
    """A replica advanced by itself (hande_iterate on its context) and then with
    the batch stays identical to a single run of the same length."""
    s, q = inputs.workload("ueg14", target_population=20000, init_pop=1000)
    b = hande.HandeBatch([s, s], [q, dict(q, seed=8)])
    one = hande.Hande(s, q)
    b.replicas[0].iterate(10)
    b.iterate(20)
    one.iterate(30)
    assert b.replicas[0].iterations == 30 and b.replicas[1].iterations == 20
    _same_lists(b.replicas[0], one, 30)
    e0, e1 = b.replicas[0].estimators(), one.estimators()
    for k in e1:
        assert np.array_equal(np.asarray(e0[k]).view(np.uint8), np.asarray(e1[k]).view(np.uint8)), k
    one.close()
    b.close()


def test_batch_stream_ordering_with_torch():
    """The caller's stream waits for the batch: a walker count read right after
    an iteration on the same stream sees every replica's finished iteration."""
    import torch
    s, q = inputs.workload("hubbard8")
    b = hande.HandeBatch([s] * 4, [dict(q, replica=r) for r in range(4)])
    b.iterate(50)
    torch.cuda.current_stream().synchronize()
    for g in b.replicas:
        rec = g.estimators()
        assert len(rec["iter"]) == 50 and rec["iter"][-1] == 50
    b.close()


def test_wide_key_batch_past_the_splitter_table():
    """Batched graphs with 512-bit replicas whose bucket counts pass the
    256-splitter on-chip table (UEG 14e in 66 orbitals from synthetic lists),
    beside 128-bit replicas: every replica equals the oracle bit for bit."""
    runs, lists = [], []
    for r, (norb, ndet) in enumerate([(66, 60000), (66, 20000), (38, 30000)]):
        s = inputs.ueg_system(14, norb, 1.0)
        q = inputs.qmc_params(tau=0.002, target_population=1e7, initiator=1, real_amplitudes=1, spawn_cutoff=0.1,
                              seed=5 + r, state_capacity=400_000, spawn_capacity=800_000)
        runs.append((s, q))
        lists.append(inputs.synthetic_walkers(s, ndet, 3.0 * ndet, seed=30 + r))
    b = hande.HandeBatch([s for s, _ in runs], [q for _, q in runs])
    cs = [oracle.Oracle(s, q) for s, q in runs]
    for g, c, (k, p) in zip(b.replicas, cs, lists):
        g.set_walkers(k, p)
        c.set_walkers(k, p)
    for it in range(3):
        b.iterate(1)
        for c in cs:
            c.iterate(1)
        for r, (g, c) in enumerate(zip(b.replicas, cs)):
            _same_lists(g, c, f"{it + 1} (replica {r})")
    assert b.replicas[0].diagnostics()["nbuckets"] > 256
    for g, c in zip(b.replicas, cs):
        _same_records(g, c)
    b.close()


def test_autotune_keeps_the_walker_lists():
    """The autotuner changes only the launch shape: a tuned batch and an
    untuned one give the same lists after the same number of iterations."""
    runs = [inputs.workload("ueg14", target_population=20000, init_pop=2000, seed=s) for s in (1, 2, 3, 4)]
    a = hande.HandeBatch([s for s, _ in runs], [q for _, q in runs])
    b = hande.HandeBatch([s for s, _ in runs], [q for _, q in runs])
    a.iterate(20)
    b.iterate(20)
    scale, ms = a.autotune(iterations=3)
    assert scale in (1.0, 2.0, 4.0, 8.0) and ms > 0.0
    groups, cap = a.layout()
    assert cap in (0, 4, 8, 16) and 1 <= groups <= len(runs)
    done = a.replicas[0].iterations
    b.iterate(done - 20)
    a.iterate(10)
    b.iterate(10)
    for ga, gb in zip(a.replicas, b.replicas):
        assert ga.iterations == gb.iterations
        ka, pa, _, _ = ga.walkers()
        kb, pb, _, _ = gb.walkers()
        assert np.array_equal(ka, kb) and np.array_equal(pa, pb)
    a.close()
    b.close()


def test_failing_replica_is_named():
    s, q = inputs.workload("hubbard8")
    b = hande.HandeBatch([s, s, s], [q, dict(q, spawn_capacity=64, replica=1), dict(q, replica=2)])
    b.iterate(5)
    with pytest.raises(hande.HandeError) as e:
        b.synchronize()
    assert e.value.status == -3 and e.value.replica == 1
    b.close()
