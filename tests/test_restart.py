"""Restart (Sec. 3.1: restart files let a resumed calculation follow the same
Markov chain as one that ran uninterrupted).  A snapshot is the walker list
plus the run state (iteration, shift, its latch and reference population,
deterministic space); the random numbers are counter-based, so the iteration
number is their whole state.  A run stopped, snapshotted and resumed in a new
context must equal the uninterrupted run bit for bit: the oracle against
itself on the CPU, the GPU engine against itself and against the oracle, and
a GPU snapshot resumed by the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import inputs


def _equal_lists(a, b):
    ka, pa, ha, fa = a.walkers()
    kb, pb, hb, fb = b.walkers()
    assert np.array_equal(ka, kb)
    assert np.array_equal(pa, pb)
    assert np.array_equal(ha.view(np.int64), hb.view(np.int64))
    assert np.array_equal(fa & 1, fb & 1)


def _equal_records(ra, rb):
    n = len(rb["iter"])
    assert n > 0
    for k in ("iter", "nw_pre", "n0", "num_hi", "num_lo", "nw_post", "ndet", "natt", "nspawn"):
        assert np.array_equal(ra[k][-n:], rb[k]), k
    assert np.array_equal(ra["shift"][-n:].view(np.int64), rb["shift"].view(np.int64))


CASES = {
    # integer walkers, the shift varying before the snapshot
    "hubbard8": (lambda: inputs.workload("hubbard8", target_population=2000), 300, 60),
    # time-step search still running at the snapshot
    "ueg_tau_search": (lambda: inputs.workload("ueg14", target_population=5000, init_pop=200, tau=0.05,
                                               tau_search=1), 8, 40),
    # heat-bath, initiator, real weights, deterministic space chosen at 30
    "molecule": (lambda: (inputs.molecule_system(norb=10, nalpha=3, nbeta=3),
                          inputs.qmc_params(tau=0.01, target_population=3000, initiator=1, real_amplitudes=1,
                                            spawn_cutoff=0.1, semi_stoch_size=60, semi_stoch_start=30,
                                            init_pop=50, seed=5)), 60, 40),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_oracle_restart_follows_the_same_chain(case):
    make, before, after = CASES[case]
    sysd, q = make()
    a = oracle.Oracle(sysd, q)
    a.iterate(before)
    keys, pops, _, _ = a.walkers()
    state, core = a.state()
    if case == "hubbard8":
        assert state["vary"] == 1
    elif case == "molecule":
        assert state["core_active"] == 1 and state["ncore"] > 1
    else:
        assert state["vary"] == 0 and state["rmax"] > 0.0
    b = oracle.Oracle(sysd, q)
    b.set_walkers(keys, pops)
    b.set_state(state, core)
    _equal_lists(a, b)
    a.iterate(after)
    b.iterate(after)
    _equal_lists(a, b)
    _equal_records(a.records(), b.records())


def test_oracle_restart_before_the_space_is_chosen():
    """A snapshot taken before semi_stoch_start: the resumed run chooses the
    deterministic space at the same iteration."""
    sysd, q = CASES["molecule"][0]()
    a = oracle.Oracle(sysd, q)
    a.iterate(20)
    keys, pops, _, _ = a.walkers()
    state, core = a.state()
    assert state["core_active"] == 0
    b = oracle.Oracle(sysd, q)
    b.set_walkers(keys, pops)
    b.set_state(state, core)
    a.iterate(30)
    b.iterate(30)
    _equal_lists(a, b)
    assert np.array_equal(a.core(), b.core()) and len(b.core()) > 1


@pytest.fixture
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(CASES))
def test_gpu_restart_equals_uninterrupted_run(_cuda, case):
    from paper_1811_11679_gb300 import hande
    make, before, after = CASES[case]
    sysd, q = make()
    a = hande.Hande(sysd, q)
    ref = oracle.Oracle(sysd, q)
    a.iterate(before)
    ref.iterate(before)
    keys, pops, hd, _ = a.walkers()
    state, core = a.state()
    ostate, ocore = ref.state()
    for k in ("iter", "nw_ref", "vary", "core_active", "ncore", "tau", "rmax"):
        assert state[k] == ostate[k], k
    assert np.float64(state["shift"]).view(np.int64) == np.float64(ostate["shift"]).view(np.int64)
    assert np.array_equal(core, ocore)
    b = hande.Hande(sysd, q)
    b.set_walkers(keys, pops)
    b.set_state(state, core)
    assert b.iterations == before
    a.iterate(after)
    b.iterate(after)
    ref.iterate(after)
    _equal_lists(a, b)
    _equal_lists(b, ref)
    rb = b.estimators()
    assert len(rb["iter"]) == after and rb["iter"][0] == before + 1
    _equal_records(rb, {k: v[-after:] for k, v in ref.records().items()})
    # the GPU snapshot resumed by the oracle follows the same chain too
    c = oracle.Oracle(sysd, q)
    k2, p2, _, _ = b.walkers()
    s2, core2 = b.state()
    c.set_walkers(k2, p2)
    c.set_state(s2, core2)
    b.iterate(10)
    c.iterate(10)
    _equal_lists(b, c)
    a.close()
    b.close()


@pytest.mark.gpu
def test_gpu_set_state_rejects_inconsistent_snapshots(_cuda):
    from paper_1811_11679_gb300 import hande
    sysd, q = CASES["molecule"][0]()
    a = hande.Hande(sysd, q)
    a.iterate(40)
    keys, pops, _, _ = a.walkers()
    state, core = a.state()
    assert state["core_active"] == 1
    _, ref = a.reference()
    b = hande.Hande(sysd, q)
    with pytest.raises(hande.HandeError) as e:
        b.set_state(dict(state, ncore=q["semi_stoch_size"] + 1), core)     # more than the space's size
    assert e.value.status == -1
    # a list without one (non-reference) core determinant
    drop = next(i for i in range(len(core)) if not np.array_equal(core[i], ref))
    keep = ~np.all(keys == core[drop][None, :], axis=1)
    b.set_walkers(keys[keep], pops[keep])
    with pytest.raises(hande.HandeError) as e:
        b.set_state(state, core)
    assert e.value.status == -1
    b.iterate(3)                                   # still usable
    b.synchronize()
    a.close()
    b.close()
