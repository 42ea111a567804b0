"""Multi-process host logic of the benchmark (gloo, two ranks on the CPU) and
the independence of replicas: each rank runs its own FCIQMC replica (Philox key
word 1 = rank), the job's figures are the slowest rank's time and the sum of
the attempts."""
from __future__ import annotations

import os
import socket

import numpy as np
import torch.multiprocessing as mp

import oracle
from paper_1811_11679_gb300 import inputs


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.aggregate_ranks(1.5 + rank, 100.0 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_rank_aggregation_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        got = dict(out)
    assert got[0] == got[1] == (2.5, 300.0)


def test_replicas_are_independent_and_reproducible():
    sysd, q = inputs.workload("hubbard8")
    runs = {}
    for rep, tag in ((0, "a"), (1, "b"), (1, "c")):
        o = oracle.Oracle(sysd, dict(q, replica=rep))
        o.iterate(30)
        runs[tag] = o.walkers()
    for x, y in zip(runs["b"], runs["c"]):
        assert np.array_equal(x, y)
    assert not all(np.array_equal(x, y) for x, y in zip(runs["a"], runs["b"]))


def test_batched_replica_recipe():
    """256 replicas: 2 bases x 4 r_s x 32 seeds, distinct Philox keys, targets in [1e4, 1e6]."""
    systems, qmcs = inputs.batched_replicas(256)
    assert len(systems) == len(qmcs) == 256
    combos = {}
    for s, q in zip(systems, qmcs):
        combos.setdefault((s["norb"], s["rs"]), []).append(q["seed"])
        assert s["key_words"] == (2 if s["norb"] == 38 else 8)
        assert 1e4 <= q["target_population"] <= 1e6
        assert q["state_capacity"] > 1.5 * q["target_population"]
    assert sorted(combos) == [(n, r) for n in (38, 66) for r in (0.5, 1.0, 2.0, 5.0)]
    assert all(sorted(v) == list(range(100, 132)) for v in combos.values())
    assert len({(q["seed"], q["replica"]) for q in qmcs}) == 256
    t = np.log10([q["target_population"] for q in qmcs])
    assert 4.8 < t.mean() < 5.2
