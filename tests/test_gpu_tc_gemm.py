"""The tensor-core GEMM (tcgen05 MMAs, TMA tile loads, accumulators in tensor
memory) behind the learned proposal's dense layers: D = A B^T with BF16
operands and FP32 accumulation, against the same product of the same BF16
values in FP64.  Products of BF16 values are exact in FP32, so the only error
is the FP32 accumulation over K terms: |D - D_exact| <= 4 K 2^-24 (|A| |B|^T)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1811_11679_gb300 import hande

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _check(torch, m, n, k, lda=None, ldb=None, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    lda = lda or k
    ldb = ldb or k
    a_full = torch.randn((m, lda), generator=g).to(torch.bfloat16)
    b_full = torch.randn((n, ldb), generator=g).to(torch.bfloat16)
    a = a_full.cuda()[:, :k]
    b = b_full.cuda()[:, :k]
    d = hande.gemm_bf16(a, b)
    torch.cuda.synchronize()
    a64 = a_full[:, :k].double()
    b64 = b_full[:, :k].double()
    exact = a64 @ b64.T
    bound = 4.0 * k * 2.0 ** -24 * (a64.abs() @ b64.abs().T) + 1e-30
    err = (d.cpu().double() - exact).abs()
    assert torch.all(err <= bound), (m, n, k, float((err / bound).max()))
    return d


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (128, 128, 16), (256, 384, 1024), (200, 72, 100),
                                   (1, 1, 1), (129, 257, 65), (4096, 256, 256), (2944, 64, 256)])
def test_gemm_matches_fp64(torch_cuda, m, n, k):
    _check(torch_cuda, m, n, k, lda=(k + 7) // 8 * 8, ldb=(k + 7) // 8 * 8)


def test_gemm_strided_operands_and_repeat(torch_cuda):
    """Leading dimensions larger than K (views into wider rows); two calls in a
    row give the same bits."""
    d1 = _check(torch_cuda, 384, 192, 136, lda=200, ldb=144, seed=3)
    d2 = _check(torch_cuda, 384, 192, 136, lda=200, ldb=144, seed=3)
    assert torch_cuda.equal(d1, d2)


def test_gemm_rejects_misaligned_rows(torch_cuda):
    torch = torch_cuda
    a = torch.zeros((128, 70), dtype=torch.bfloat16, device="cuda")[:, :68]
    b = torch.zeros((128, 68), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(hande.HandeError) as e:
        hande.gemm_bf16(a, b)   # lda = 70 is not a multiple of 8
    assert e.value.status == -1
