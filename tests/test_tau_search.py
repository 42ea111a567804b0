"""Time-step search (the tutorial's `tau_search`; the reading: until the
population first exceeds the target, after each iteration
tau <- min(tau, 1 / R), R = the largest |H_ij| / p_gen = (|H_ij| inv_a) inv_b
over every spawning attempt so far; tau is fixed afterwards).

Pins: on the Hubbard ring every hop has |H| = t and p_gen = 1 / (2N), so R is
2 N t exactly and the search lands on 1 / (2 N t); the time step never grows
and stops changing once the shift varies; on the GPU the walker lists and the
recorded time steps equal the oracle's bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import inputs


def test_hubbard_ring_search_lands_on_the_closed_form():
    sysd, q = inputs.workload("hubbard8", tau=0.2, tau_search=1, target_population=3000)
    o = oracle.Oracle(sysd, q)
    o.iterate(20)
    r = o.records()
    n = sysd["nalpha"] + sysd["nbeta"]
    assert r["tau"][0] == 0.2                       # the first iteration uses the given step
    assert r["tau"][1] == 1.0 / (2.0 * n * sysd["t"])
    assert np.all(np.diff(r["tau"]) <= 0.0)


def test_search_only_shrinks_and_freezes_with_the_shift():
    sysd, q = inputs.workload("ueg14", target_population=2500, init_pop=200, tau=0.05, tau_search=1)
    o = oracle.Oracle(sysd, q)
    o.iterate(120)
    r = o.records()
    tau, shift = r["tau"], r["shift"]
    assert np.all(np.diff(tau) <= 0.0) and tau[-1] < 0.05
    varying = np.nonzero(shift != 0.0)[0]
    assert len(varying) > 0
    first = varying[0]
    assert np.all(tau[first + 1:] == tau[first + 1])
    st, _ = o.state()
    assert st["tau"] == tau[-1] and st["rmax"] > 0.0 and st["tau"] <= 1.0 / st["rmax"]


def _equal(g, c):
    kg, pg, hg, _ = g.walkers()
    kc, pc, hc, _ = c.walkers()
    assert np.array_equal(kg, kc) and np.array_equal(pg, pc)
    assert np.array_equal(hg.view(np.int64), hc.view(np.int64))


CASES = {
    "hubbard8": lambda: inputs.workload("hubbard8", tau=0.2, tau_search=1, target_population=3000, init_pop=50),
    "ueg14": lambda: inputs.workload("ueg14", target_population=5000, init_pop=200, tau=0.05, tau_search=1),
    "molecule": lambda: inputs.workload("molecule28", target_population=20000, tau=0.05, tau_search=1,
                                        semi_stoch_size=200, semi_stoch_start=40),
}


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(CASES))
def test_gpu_time_step_search_parity(case):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1811_11679_gb300 import hande
    sysd, q = CASES[case]()
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    for _ in range(6 if case == "hubbard8" else 12):
        g.iterate(10)
        c.iterate(10)
        _equal(g, c)
    eg, ec = g.estimators(), c.records()
    assert np.array_equal(eg["tau"].view(np.int64), ec["tau"].view(np.int64))
    assert np.array_equal(eg["shift"].view(np.int64), ec["shift"].view(np.int64))
    for k in ("nw_pre", "n0", "num_hi", "num_lo", "nw_post", "ndet", "natt", "nspawn"):
        assert np.array_equal(eg[k], ec[k]), k
    assert ec["tau"][-1] < q["tau"]
    sg, _ = g.state()
    so, _ = c.state()
    assert np.float64(sg["tau"]).view(np.int64) == np.float64(so["tau"]).view(np.int64)
    assert np.float64(sg["rmax"]).view(np.int64) == np.float64(so["rmax"]).view(np.int64)
    g.close()
