"""tcgen05 bf16 product (lrr_gemm_bf16) against a float64 CPU product of the
same bf16 values: the only difference is float32 accumulation order."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K,pad", [(128, 128, 64, 0), (200, 300, 100, 4), (96, 40, 8, 0),
                                       (1000, 1500, 1000, 0), (257, 129, 200, 8)])
def test_tc_gemm_matches_float64_product(lib, M, N, K, pad):
    import torch
    from paper_1304_5583_gb300 import binding
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    lda = ((K + pad + 7) // 8) * 8
    A = torch.randn(M, lda, generator=g).to(torch.bfloat16)
    B = torch.randn(N, lda, generator=g).to(torch.bfloat16)
    C = binding.gemm_bf16(A.cuda(), B.cuda(), M, N, K).cpu().numpy()
    ref = A[:, :K].double().numpy() @ B[:, :K].double().numpy().T
    err = np.abs(C - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err
