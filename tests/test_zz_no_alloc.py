"""lrr_svt_noalloc -- the SVT entry point that allocates nothing, for callers
that cannot allocate device memory while they call it (stream capture, foreign
allocators, latency-bound loops) -- gives the same result as lrr_svt, call
after call, through the C ABI.  Collected last on purpose: it runs after every
other test, and also passes on its own in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _case(seed, rows, cols, lo, hi):
    rng = np.random.default_rng(seed)
    k = min(rows, cols)
    U = np.linalg.qr(rng.standard_normal((rows, k)))[0]
    V = np.linalg.qr(rng.standard_normal((cols, k)))[0]
    return (U * np.geomspace(hi, lo, k)) @ V.T


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_no_alloc_svt_matches_allocating_svt_on_consecutive_calls(lib, dtype):
    import torch
    from paper_1304_5583_gb300 import binding
    dt = np.float32 if dtype == "f32" else np.float64
    tol = 5e-6 if dtype == "f32" else 1e-12
    # two calls in a row with different shapes: the second must not see the first's leftovers
    for seed, (rows, cols, tau) in enumerate([(300, 150, 1e-2), (120, 260, 5e-2)]):
        A = torch.from_numpy(np.asfortranarray(_case(seed, rows, cols, 1e-4, 1.0).astype(dt))).cuda()
        J_ref, rk_ref = binding.svt(A, tau)
        J, rk = binding.svt(A, tau, no_alloc=True)
        assert rk == rk_ref
        Jr = J_ref.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(J.cpu().numpy() - Jr) / np.linalg.norm(Jr) < tol


def test_no_alloc_svt_rejects_oversized_problem(lib):
    import ctypes
    import torch
    from paper_1304_5583_gb300 import binding
    cap = lib.lrr_svt_noalloc_capacity()
    assert cap == 32 << 20
    n = 2048                      # float32 2048 x 2048 needs ~64 MiB of scratch
    A = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    J = torch.empty_like(A)
    rk = ctypes.c_int32(0)
    code = lib.lrr_svt_noalloc(ctypes.c_void_p(A.data_ptr()), n, n, n, 0.1, ctypes.c_void_p(J.data_ptr()), n,
                               binding.LRR_PREC_F32, ctypes.byref(rk),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == -7
