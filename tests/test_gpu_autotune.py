"""Single-context autotuner (include/hande.h, hande_autotune): it changes the
bucket sizes and the spawning grid only, so a tuned run keeps the walker lists
of an untuned run of the same length bit for bit, and both equal the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import hande, inputs
from test_gpu_parity import _same_lists

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name", ["ueg14", "molecule28"])
def test_autotune_keeps_the_lists(name):
    s, q = inputs.workload(name, target_population=20000, init_pop=2000, semi_stoch_size=0)
    a, b = hande.Hande(s, q), hande.Hande(s, q)
    a.iterate(30)
    b.iterate(30)
    t = a.autotune(iterations=2)
    assert t["bucket_spawns"] >= 1 and t["attempt_blocks"] >= 1 and t["ms_per_iteration"] > 0.0
    assert a.iterations == 30 + 16 * 3
    b.iterate(a.iterations - 30)
    a.iterate(5)
    b.iterate(5)
    ka, pa, _, _ = a.walkers()
    kb, pb, _, _ = b.walkers()
    assert np.array_equal(ka, kb) and np.array_equal(pa, pb)
    ra, rb = a.estimators(), b.estimators()
    for k in rb:
        assert np.array_equal(np.asarray(ra[k]).view(np.uint8), np.asarray(rb[k]).view(np.uint8)), k
    c = oracle.Oracle(s, q)
    c.iterate(a.iterations)
    _same_lists(a, c, a.iterations)
    a.close()
    b.close()
