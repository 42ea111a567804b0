"""hande_estimate_noalloc, the entry point for callers that may not allocate
device memory (an application that reserved its whole device budget up front,
a memory pool that owns every free byte, a latency-critical loop that must not
call cudaMalloc because it can synchronise the device): its projected-energy
sums must equal those the regular iteration records for the same walker list,
call after call, although its partial sums live in one fixed device array
shared by all calls.  Collected last on purpose."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1811_11679_gb300 import hande, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _device_list(torch, keys, pops):
    dk = torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()
    dp = torch.from_numpy(np.ascontiguousarray(pops)).cuda()
    return dk, dp


@pytest.mark.parametrize("workload,kw", [
    ("ueg14", dict(target_population=20000, init_pop=1000)),
    ("molecule28", dict(target_population=30000)),
])
def test_noalloc_estimator_equals_iteration_records(torch_cuda, workload, kw):
    torch = torch_cuda
    sysd, q = inputs.workload(workload, **kw)
    g = hande.Hande(sysd, q)
    g.iterate(40)
    g.estimators()
    out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    for call in range(2):                       # two calls in a row share the scratch array
        keys, pops, _, _ = g.walkers()
        dk, dp = _device_list(torch, keys, pops)
        torch.cuda.synchronize()
        g.estimate_noalloc(dk.data_ptr(), dp.data_ptr(), len(pops), out.data_ptr())
        g.synchronize()
        got = out.cpu().numpy()
        g.iterate(1)                            # its record is evaluated on the same list
        rec = g.estimators()
        assert got[0] == rec["nw_pre"][-1]
        assert got[1] == rec["n0"][-1]
        assert np.uint64(got[2].view(np.uint64)) == rec["num_lo"][-1]
        assert got[3] == rec["num_hi"][-1]
        g.iterate(5)
        g.estimators()
    g.close()


def test_noalloc_allocates_nothing_and_handles_an_empty_list(torch_cuda):
    """A call changes neither PyTorch's device-memory statistics (the library's
    own buffers are routed through PyTorch's allocator) nor needs a list: n = 0
    writes zeros."""
    torch = torch_cuda
    sysd, q = inputs.workload("ueg14", target_population=20000, init_pop=1000)
    g = hande.Hande(sysd, q)
    g.iterate(30)
    keys, pops, _, _ = g.walkers()
    dk, dp = _device_list(torch, keys, pops)
    out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    g.estimate_noalloc(dk.data_ptr(), dp.data_ptr(), len(pops), out.data_ptr())   # first call: set-up
    g.synchronize()
    first = out.cpu().numpy().copy()
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats()
    g.estimate_noalloc(dk.data_ptr(), dp.data_ptr(), len(pops), out.data_ptr())
    g.synchronize()
    after = torch.cuda.memory_stats()
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert before.get(k) == after.get(k), k
    assert np.array_equal(out.cpu().numpy(), first)
    g.estimate_noalloc(0, 0, 0, out.data_ptr())
    g.synchronize()
    assert out.cpu().numpy().tolist() == [0, 0, 0, 0]
    g.close()


def test_noalloc_rejects_lists_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    sysd, q = inputs.workload("ueg14", target_population=1000, init_pop=100)
    g = hande.Hande(sysd, q)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    small = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(hande.HandeError) as e:
        g.estimate_noalloc(small.data_ptr(), small.data_ptr(), 4096 * 4096 + 1, out.data_ptr())
    assert e.value.status == -3
    # the context is still usable afterwards
    g.iterate(2)
    g.synchronize()
    g.close()
