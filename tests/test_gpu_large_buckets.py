"""GPU = oracle parity at the bucket counts the benchmark runs.

The spawning kernel finds a spawn's annihilation bucket by a two-level search:
every r-th splitter key is staged in shared memory (r = 1 while the bucket
count fits the on-chip table: 4096, 2048 and 256 splitters for 64-, 128- and
512-bit keys), then at most r - 1 more in global memory.  The one-block scans
of the bucket counts and of the kept counts carry a running sum across chunks
of 4096 buckets.  The 1e7-walker benchmark runs about 13 000 buckets, so both
the second search level (r > 1) and the carried scan run there.  These tests
start from seeded synthetic lists large enough to pass those limits, assert
that the bucket count did, and compare every determinant, population,
diagonal element and core flag with the oracle after each iteration, and the
estimator records at the end (Sec. 2.4 and App. B: one annihilation per
iteration of the sorted main list with the spawned list)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import hande, inputs

pytestmark = pytest.mark.gpu

# on-chip splitter table of the spawning kernel and the scan chunk
SPLITTERS = {1: 4096, 2: 2048, 8: 256}
SCAN_CHUNK = 4096


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _same_lists(g, c, it):
    kg, pg, hg, fg = g.walkers()
    kc, pc, hc, fc = c.walkers()
    assert kg.shape == kc.shape, f"iteration {it}: {len(kg)} vs {len(kc)} determinants"
    assert np.array_equal(kg, kc), f"iteration {it}: keys differ"
    assert np.array_equal(pg, pc), f"iteration {it}: populations differ"
    assert np.array_equal(hg.view(np.int64), hc.view(np.int64)), f"iteration {it}: diagonal differs"
    assert np.array_equal(fg & 1, fc & 1), f"iteration {it}: core flags differ"
    return len(kg)


def _same_records(g, c):
    eg = g.estimators()
    ec = c.records()
    n = len(ec["iter"])
    for k in ("iter", "nw_pre", "n0", "num_hi", "nw_post", "ndet", "natt", "nspawn"):
        assert np.array_equal(eg[k][-n:], ec[k]), k
    assert np.array_equal(eg["num_lo"][-n:], ec["num_lo"])
    assert np.array_equal(eg["shift"][-n:].view(np.int64), ec["shift"].view(np.int64))


CASES = {
    # the benchmark's system and settings (heat-bath, initiator, real weights,
    # a 1e4 deterministic space chosen from the list), 64-bit keys
    "molecule28_w1": dict(system=lambda: inputs.molecule_system(),
                          qmc=dict(tau=0.01, target_population=1e7, initiator=1, real_amplitudes=1,
                                   spawn_cutoff=0.1, semi_stoch_size=10000, semi_stoch_start=0, seed=8,
                                   state_capacity=3_000_000, spawn_capacity=6_000_000),
                          ndet=1_000_000, walkers=2.5e6, iters=3),
    # UEG 14e / 38 spatial orbitals, 128-bit keys
    "ueg14_w2": dict(system=lambda: inputs.ueg_system(14, 38, 1.0),
                     qmc=dict(tau=0.002, target_population=1e7, initiator=1, real_amplitudes=1,
                              spawn_cutoff=0.1, seed=7, state_capacity=2_000_000, spawn_capacity=4_000_000),
                     ndet=500_000, walkers=1.2e6, iters=3),
    # UEG 14e / 66 spatial orbitals (132 spin orbitals), 512-bit keys
    "ueg66_w8": dict(system=lambda: inputs.ueg_system(14, 66, 1.0),
                     qmc=dict(tau=0.002, target_population=1e7, initiator=1, real_amplitudes=1,
                              spawn_cutoff=0.1, seed=5, state_capacity=600_000, spawn_capacity=1_500_000),
                     ndet=100_000, walkers=3e5, iters=3),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_bucket_counts_beyond_the_on_chip_splitter_table(case):
    spec = CASES[case]
    sysd = spec["system"]()
    q = inputs.qmc_params(**spec["qmc"])
    W = int(sysd["key_words"])
    keys, pops = inputs.synthetic_walkers(sysd, spec["ndet"], spec["walkers"])
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    g.set_walkers(keys, pops)
    c.set_walkers(keys, pops)
    counts = []
    for it in range(spec["iters"]):
        g.iterate(1)
        c.iterate(1)
        d = g.diagnostics()
        counts.append(int(d["nbuckets"]))
        # the second search level runs in every iteration
        assert d["nbuckets"] > SPLITTERS[W], (it + 1, d["nbuckets"])
        _same_lists(g, c, it + 1)
    if W in (1, 2):
        # the carried scans (more than one chunk of bucket counts) ran as well
        assert max(counts) > SCAN_CHUNK, counts
    _same_records(g, c)
    g.close()


@pytest.mark.parametrize("init_pop", [300, 3000])
def test_wide_key_oversized_and_deferred_buckets(init_pop):
    """512-bit keys on the warp path (tile: 96 segment entries, 64 staged new
    keys): a one-determinant start puts every spawn of the first iterations in
    few buckets, beyond the warp's staging (deferred to block tiles) or beyond
    8 x 64 spawns (taken by block tiles beside the warp kernel)."""
    sysd = inputs.ueg_system(14, 66, 1.0)
    assert sysd["key_words"] == 8
    q = inputs.qmc_params(tau=0.002, target_population=1e6, initiator=1, real_amplitudes=1,
                          spawn_cutoff=0.1, init_pop=init_pop, seed=7, annihilation=2)
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    deferred, biggest = 0, 0
    for it in range(25):
        g.iterate(1)
        c.iterate(1)
        d = g.diagnostics()
        deferred = max(deferred, int(d["deferred_buckets"]))
        biggest = max(biggest, int(d["max_bucket_spawns"]))
        _same_lists(g, c, it + 1)
    _same_records(g, c)
    assert deferred > 0
    if init_pop >= 3000:
        assert biggest > 8 * 64
    else:
        assert biggest > 64
    g.close()
