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


@pytest.mark.parametrize("M,N,K,pad", [(128, 128, 32, 0), (200, 300, 100, 4), (96, 40, 8, 0),
                                       (1000, 1500, 1000, 0), (257, 129, 203, 4)])
def test_split_tf32_gemm_is_float32_accurate(lib, M, N, K, pad):
    """lrr_gemm_f32 (three TF32 tensor-core products per term) against the
    float64 product of the same float32 values: the error is that of a
    float32 product, well below what a single TF32 or bf16 pass gives."""
    import torch
    from paper_1304_5583_gb300 import binding
    g = torch.Generator().manual_seed(M * 5 + N * 3 + K)
    lda = ((K + pad + 3) // 4) * 4
    A = torch.randn(M, lda, generator=g, dtype=torch.float32)
    B = torch.randn(N, lda, generator=g, dtype=torch.float32)
    C = binding.gemm_f32(A.cuda(), B.cuda(), M, N, K).cpu().numpy()
    ref = A[:, :K].double().numpy() @ B[:, :K].double().numpy().T
    # per entry against sum_k |a_ik b_kj| (the scale of its rounding)
    scale = np.abs(A[:, :K].double().numpy()) @ np.abs(B[:, :K].double().numpy()).T
    err = float(np.max(np.abs(C - ref) / scale))
    # a float32 product (OpenBLAS sgemm) of the same operands, for scale
    c32 = (A[:, :K].numpy() @ B[:, :K].numpy().T).astype(np.float64)
    err32 = float(np.max(np.abs(c32 - ref) / scale))
    print(f"3xTF32 {M}x{N}x{K}: max error / sum|ab| = {err:.2e} (float32 sgemm {err32:.2e})")
    assert err < max(4 * err32, 2e-7), (err, err32)
