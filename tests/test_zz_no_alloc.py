"""lrr_svt_noalloc -- the SVT entry point that allocates nothing, for callers
that cannot allocate device memory at the point where they need it (memory
owned by another allocator, fixed arenas, latency-critical paths) -- gives the
same result as lrr_svt and as the oracle's closed-form SVT, call after call,
through the C ABI.  Collected last on purpose: it runs after every other test,
and also passes on its own in a fresh process."""
import numpy as np
import pytest

from oracle import lrr as olrr

pytestmark = pytest.mark.gpu


def _case(seed, rows, cols, lo, hi):
    rng = np.random.default_rng(seed)
    k = min(rows, cols)
    U = np.linalg.qr(rng.standard_normal((rows, k)))[0]
    V = np.linalg.qr(rng.standard_normal((cols, k)))[0]
    return (U * np.geomspace(hi, lo, k)) @ V.T


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_no_alloc_svt_matches_allocating_svt_on_consecutive_calls(lib, dtype):
    import torch
    from paper_1304_5583_gb300 import binding
    dt = np.float32 if dtype == "f32" else np.float64
    tol = 5e-6 if dtype == "f32" else 1e-12
    # two calls in a row with different shapes: the second must not see the first's leftovers
    for seed, (rows, cols, tau) in enumerate([(300, 150, 1e-2), (120, 260, 5e-2)]):
        Ah = _case(seed, rows, cols, 1e-4, 1.0).astype(dt)
        A = torch.from_numpy(np.asfortranarray(Ah)).cuda()
        J_ref, rk_ref = binding.svt(A, tau)
        J, rk = binding.svt(A, tau, no_alloc=True)
        assert rk == rk_ref
        Jr = J_ref.cpu().numpy().astype(np.float64)
        Jn = J.cpu().numpy().astype(np.float64)
        assert _rel(Jn, Jr) < tol
        # and against the closed form (full SVD in float64) on the same input
        Jo, Uo, _, _ = olrr.svt(Ah.astype(np.float64), tau)
        assert rk == Uo.shape[1]
        assert _rel(Jn, Jo) < tol


def test_no_alloc_svt_near_capacity(lib):
    """The largest float64 square problem that fits the fixed array."""
    import torch
    from paper_1304_5583_gb300 import binding
    n, tau = 1000, 3e-2
    Ah = _case(7, n, n, 1e-3, 1.0)
    A = torch.from_numpy(np.asfortranarray(Ah)).cuda()
    J, rk = binding.svt(A, tau, no_alloc=True)
    Jo, Uo, _, _ = olrr.svt(Ah, tau)
    assert rk == Uo.shape[1]
    assert _rel(J.cpu().numpy(), Jo) < 1e-12


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
