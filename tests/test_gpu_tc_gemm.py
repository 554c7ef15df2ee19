"""The tensor-core product (tcgen05, TMA, TMEM) against numpy.

C = alpha A B^T (+ C) with bf16 A, B and fp32 accumulation: the products of
two bf16 values are exact in fp32, so the only difference from the float64
product of the same bf16 values is the fp32 summation, bounded here by
K * 2^-24 * sum |a||b| per element.  Shapes cover every tile width (32, 64,
128, 256), ragged edges in m, n and k, batches and accumulation."""

import numpy as np
import pytest

from paper_1102_3069_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()
    return t, t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m,n,k,batch", [(128, 128, 64, 1), (200, 72, 40, 1), (256, 256, 1024, 1), (64, 32, 16, 3),
                                         (1000, 300, 136, 2), (33, 17, 8, 1), (130, 250, 200, 1),
                                         (2048, 1024, 2048, 1), (64, 64, 64, 512)])
def test_product_matches_float64(m, n, k, batch):
    import torch
    g = np.random.default_rng(m * 7 + n * 3 + k)
    a, a64 = _bf16(g.standard_normal((batch, m, k)))
    b, b64 = _bf16(g.standard_normal((batch, n, k)))
    c = torch.full((batch, m, n), float("nan"), dtype=torch.float32, device="cuda")
    B.mm_gemm_bf16(a, k, m * k, b, k, n * k, c, n, m * n, m, n, k, batch)
    assert B.mm_gemm_status() == B.MM_OK
    ref = np.einsum("bmk,bnk->bmn", a64, b64)
    bound = k * 2.0 ** -24 * np.einsum("bmk,bnk->bmn", np.abs(a64), np.abs(b64))
    got = c.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= bound + 1e-30), float(np.max(np.abs(got - ref) / (bound + 1e-30)))
    # and on average like a random walk of fp32 roundings: sqrt(K) * 2^-24 relative
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 4.0 * np.sqrt(k) * 2.0 ** -24, rel


def test_alpha_beta_and_strided_rows():
    import torch
    g = np.random.default_rng(9)
    m, n, k, lda = 150, 96, 80, 96          # A rows padded to 96 elements
    a_full, a64f = _bf16(g.standard_normal((m, lda)))
    b, b64 = _bf16(g.standard_normal((n, k)))
    c0 = g.standard_normal((m, n)).astype(np.float32)
    c = torch.from_numpy(c0.copy()).cuda()
    B.mm_gemm_bf16(a_full, lda, 0, b, k, 0, c, n, 0, m, n, k, 1, alpha=-0.5, beta=1)
    assert B.mm_gemm_status() == B.MM_OK
    ref = c0.astype(np.float64) - 0.5 * a64f[:, :k] @ b64.T
    got = c.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_bad_strides_are_refused():
    import torch
    a = torch.zeros((4, 12), dtype=torch.bfloat16, device="cuda")
    c = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(B.MMError):
        B.mm_gemm_bf16(a, 12, 0, a, 12, 0, c, 4, 0, 4, 4, 12, 1)     # row stride of 24 bytes
