"""The oracle's hash-partitioned parallel iteration (the paper's parallel
layout, App. B: determinants owned by hash mod P, one all-to-all of the spawns,
annihilation per owner) against its serial iteration: bit-identical walker
lists and records for every thread count, because the random numbers are
counter-based and all population sums are exact integers."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import inputs

CASES = {
    "hubbard8_integer": lambda: inputs.workload("hubbard8", target_population=3000),
    "molecule_core": lambda: (inputs.molecule_system(norb=10, nalpha=3, nbeta=3),
                              inputs.qmc_params(tau=0.01, target_population=5000, initiator=1, real_amplitudes=1,
                                                spawn_cutoff=0.1, semi_stoch_size=80, semi_stoch_start=20,
                                                init_pop=100, seed=5)),
    "ueg_initiator": lambda: inputs.workload("ueg14", target_population=8000, init_pop=500),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_parallel_oracle_equals_serial(case, threads):
    sysd, q = CASES[case]()
    a = oracle.Oracle(sysd, q)
    b = oracle.Oracle(sysd, q, threads=threads)
    for _ in range(4):
        a.iterate(15)
        b.iterate(15)
        ka, pa, ha, fa = a.walkers()
        kb, pb, hb, fb = b.walkers()
        assert np.array_equal(ka, kb) and np.array_equal(pa, pb)
        assert np.array_equal(ha.view(np.int64), hb.view(np.int64)) and np.array_equal(fa, fb)
    ra, rb = a.records(), b.records()
    for k in ra:
        assert np.array_equal(np.asarray(ra[k]).view(np.int64), np.asarray(rb[k]).view(np.int64)), k
