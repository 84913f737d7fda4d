"""ctypes binding of libdfc_lrr.so (declared in include/dfc_lrr.h).

Argument marshalling only: torch tensors become device pointers, the current
torch stream becomes the library's stream, and the workspace is a torch
allocation.  Every step of the solve runs in the library's CUDA kernels; if
the library is missing or cannot load, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdfc_lrr.so")

LRR_OK, LRR_NOT_CONVERGED = 0, 1
LRR_PREC_F64, LRR_PREC_F32, LRR_PREC_MIXED = 0, 1, 2
PRECISIONS = {"f64": LRR_PREC_F64, "f32": LRR_PREC_F32, "mixed": LRR_PREC_MIXED}

# every symbol include/dfc_lrr.h declares
EXPORTS = ("dfc_partition", "lrr_workspace_bytes", "lrr_solve", "dfc_lrr_solve", "lrr_svt", "lrr_svt_noalloc",
           "lrr_svt_noalloc_capacity", "lrr_gemm_bf16", "lrr_default_options", "lrr_status_string",
           "lrr_factor_max_rank", "lrr_gemm_f32", "lrr_unrolled_workspace_bytes", "lrr_unrolled_forward",
           "lrr_unrolled_backward", "lrr_gemm_timing", "lrr_segment_workspace_bytes", "lrr_segment",
           "lrr_solve_batch", "dfc_lrr_solve_local")


class LrrProblem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("ldm", ctypes.c_int64),
                ("t", ctypes.c_int32), ("perm", ctypes.POINTER(ctypes.c_int64)),
                ("offsets", ctypes.POINTER(ctypes.c_int64)), ("seed", ctypes.c_uint64)]


class LrrOptions(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("rho", ctypes.c_double), ("mu0", ctypes.c_double),
                ("mu_max", ctypes.c_double), ("eps", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("batched", ctypes.c_int32), ("jacobi_sweeps", ctypes.c_int32),
                ("rank_tol", ctypes.c_double), ("mixed_switch", ctypes.c_double), ("profile", ctypes.c_int32),
                ("tc_products", ctypes.c_int32), ("autotune", ctypes.c_int32)]

NPHASE = 12
PHASES = ("setup", "gram", "warm", "jacobi", "svt_apply", "zgemm", "zupdate", "mzgemm", "eupdate", "stop",
          "combine", "host")


class LrrUnrolledOptions(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("rho", ctypes.c_double), ("mu0", ctypes.c_double),
                ("mu_max", ctypes.c_double), ("rank_tol", ctypes.c_double), ("K", ctypes.c_int32),
                ("checkpoint", ctypes.c_int32), ("precision", ctypes.c_int32)]


class LrrStats(ctypes.Structure):
    _fields_ = [("phase_ms", ctypes.c_double * NPHASE), ("phase_launches", ctypes.c_int64 * NPHASE),
                ("launches", ctypes.c_int64), ("iterations", ctypes.c_int64), ("svt_sweeps", ctypes.c_int64),
                ("svt_calls", ctypes.c_int64)]


class LrrResult(ctypes.Structure):
    _fields_ = [("Z", ctypes.c_void_p), ("S", ctypes.c_void_p), ("iters", ctypes.POINTER(ctypes.c_int32)),
                ("resid", ctypes.POINTER(ctypes.c_double)), ("ranks", ctypes.POINTER(ctypes.c_int32)),
                ("timings_ms", ctypes.POINTER(ctypes.c_double)), ("stats", ctypes.POINTER(LrrStats)),
                ("F", ctypes.c_void_p), ("G", ctypes.c_void_p), ("factor_k", ctypes.POINTER(ctypes.c_int32)),
                ("sweeps", ctypes.POINTER(ctypes.c_int32))]


_LIB = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (raises OSError if it is not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise OSError(f"{path} is not built; run paper_1304_5583_gb300/build.py")
    lib = ctypes.CDLL(path)
    lib.dfc_partition.restype = ctypes.c_int
    lib.dfc_partition.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int64)]
    lib.lrr_workspace_bytes.restype = ctypes.c_size_t
    lib.lrr_workspace_bytes.argtypes = [ctypes.POINTER(LrrProblem), ctypes.POINTER(LrrOptions)]
    for fn in (lib.lrr_solve, lib.dfc_lrr_solve):
        fn.restype = ctypes.c_int
        fn.argtypes = [ctypes.POINTER(LrrProblem), ctypes.POINTER(LrrOptions), ctypes.c_void_p, ctypes.c_size_t,
                       ctypes.POINTER(LrrResult), ctypes.c_void_p]
    lib.lrr_svt.restype = ctypes.c_int
    lib.lrr_svt.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                            ctypes.c_void_p]
    lib.lrr_svt_noalloc.restype = ctypes.c_int
    lib.lrr_svt_noalloc.argtypes = lib.lrr_svt.argtypes
    lib.lrr_svt_noalloc_capacity.restype = ctypes.c_size_t
    lib.lrr_svt_noalloc_capacity.argtypes = []
    lib.lrr_gemm_bf16.restype = ctypes.c_int
    lib.lrr_gemm_bf16.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    lib.lrr_gemm_f32.restype = ctypes.c_int
    lib.lrr_gemm_f32.argtypes = lib.lrr_gemm_bf16.argtypes
    lib.lrr_unrolled_workspace_bytes.restype = ctypes.c_size_t
    lib.lrr_unrolled_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(LrrUnrolledOptions),
                                                 ctypes.c_int32]
    lib.lrr_unrolled_forward.restype = ctypes.c_int
    lib.lrr_unrolled_forward.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(LrrUnrolledOptions), ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    lib.lrr_unrolled_backward.restype = ctypes.c_int
    lib.lrr_unrolled_backward.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.POINTER(LrrUnrolledOptions), ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    lib.lrr_gemm_timing.restype = ctypes.c_int
    lib.lrr_gemm_timing.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.lrr_segment_workspace_bytes.restype = ctypes.c_size_t
    lib.lrr_segment_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
    lib.lrr_segment.restype = ctypes.c_int
    lib.lrr_segment.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.c_void_p]
    lib.lrr_solve_batch.restype = ctypes.c_int
    lib.lrr_solve_batch.argtypes = [ctypes.POINTER(LrrProblem), ctypes.c_int32, ctypes.POINTER(LrrOptions),
                                    ctypes.POINTER(LrrResult), ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                    ctypes.c_void_p]
    lib.dfc_lrr_solve_local.restype = ctypes.c_int
    lib.dfc_lrr_solve_local.argtypes = [ctypes.POINTER(LrrProblem), ctypes.POINTER(LrrOptions), ctypes.c_int64,
                                        ctypes.POINTER(LrrResult), ctypes.c_int32, ctypes.c_void_p]
    lib.lrr_factor_max_rank.restype = ctypes.c_int64
    lib.lrr_factor_max_rank.argtypes = [ctypes.POINTER(LrrProblem)]
    lib.lrr_default_options.restype = None
    lib.lrr_default_options.argtypes = [ctypes.POINTER(LrrOptions)]
    lib.lrr_status_string.restype = ctypes.c_char_p
    lib.lrr_status_string.argtypes = [ctypes.c_int]
    _LIB = lib
    return lib


def status_string(code: int) -> str:
    return load().lrr_status_string(int(code)).decode()


class LrrError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"lrr status {code}: {status_string(code)}")
        self.code = code


@dataclass
class SolveResult:
    Z: object            # torch (n, n), column-major storage, original column order
    S: object            # torch (m, n)
    iters: np.ndarray    # (t,)
    resid: np.ndarray    # (t, 2)
    rank_M: int
    k1: int
    block_ranks: np.ndarray
    timings_ms: np.ndarray
    status: int
    stats: dict
    F: object = None         # torch (n, kmax) or None: Z = F[:, :factor_k] @ G[:factor_k]
    G: object = None         # torch (kmax, n) or None
    factor_k: int = 0
    sweeps: np.ndarray = None   # (t,) Jacobi sweeps per block


def column_major(x):
    """(rows, cols) tensor with unit row stride (a column-major matrix); copies if needed."""
    if x.dim() == 2 and x.stride(0) == 1 and (x.stride(1) >= max(1, x.shape[0]) or x.shape[1] == 1):
        return x
    return x.t().contiguous().t()


def leading_dim(x):
    """Leading dimension of a column-major (rows, cols) tensor (a single
    column's stride is arbitrary in torch: use rows)."""
    return x.stride(1) if x.shape[1] > 1 else max(1, x.shape[0])


def options(lam: float, rho: float = 1.1, mu0: float = 1e-6, mu_max: float = 1e10, eps: float = 1e-6,
            max_iter: int = 1000, precision: str = "f32", batched: bool = True, jacobi_sweeps: int = 0,
            rank_tol: float = 0.0, mixed_switch: float = 0.0, profile: bool = False, tc_products: bool = False,
            autotune: bool = False) -> LrrOptions:
    o = LrrOptions()
    load().lrr_default_options(ctypes.byref(o))
    o.lambda_, o.rho, o.mu0, o.mu_max, o.eps = lam, rho, mu0, mu_max, eps
    o.max_iter, o.precision, o.batched = int(max_iter), PRECISIONS[precision], int(bool(batched))
    o.jacobi_sweeps, o.rank_tol, o.mixed_switch = int(jacobi_sweeps), float(rank_tol), float(mixed_switch)
    o.profile = int(bool(profile))
    o.tc_products, o.autotune = int(bool(tc_products)), int(bool(autotune))
    return o


def partition(n: int, t: int, seed: int):
    """The D step's random partition (dfc_partition): (perm, offsets)."""
    perm = np.zeros(n, np.int64)
    offsets = np.zeros(t + 1, np.int64)
    code = load().dfc_partition(ctypes.c_int64(n), ctypes.c_int32(t), ctypes.c_uint64(seed),
                                perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if code < 0:
        raise LrrError(code)
    return perm, offsets


def _problem(M, perm, offsets, t=None, seed=0):
    """perm / offsets may be None (the library then draws the D step from
    `seed`); t is required when offsets is None."""
    p = LrrProblem()
    p.M = ctypes.c_void_p(M.data_ptr())
    p.m, p.n, p.ldm = M.shape[0], M.shape[1], leading_dim(M)
    keep = []
    if offsets is not None:
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        p.t = len(offsets) - 1
        p.offsets = offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        keep.append(offsets)
    else:
        if t is None:
            raise ValueError("t is required when offsets is None")
        p.t = int(t)
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.int64)
        p.perm = perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        keep.append(perm)
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return p, keep


def workspace_bytes(M, perm, offsets, opts: LrrOptions, t=None, seed=0) -> int:
    p, keep = _problem(M, perm, offsets, t, seed)
    return int(load().lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(opts)))


def factor_max_rank(M, perm, offsets, t=None, seed=0) -> int:
    p, keep = _problem(M, perm, offsets, t, seed)
    return int(load().lrr_factor_max_rank(ctypes.byref(p)))


def _solve(entry: str, M, perm, offsets, opts: LrrOptions, want_Z=True, want_S=True, workspace=None,
           raise_on_error=True, t=None, seed=0, want_factors=False) -> SolveResult:
    import torch
    lib = load()
    if not M.is_cuda:
        raise ValueError("M must be a CUDA tensor")
    M = column_major(M)
    m, n = M.shape
    p, keep = _problem(M, perm, offsets, t, seed)
    t = p.t
    need = int(lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(opts)))
    if need == 0:
        if raise_on_error:
            raise LrrError(-1)
        return SolveResult(Z=None, S=None, iters=np.zeros(t, np.int32), resid=np.zeros((t, 2)), rank_M=0, k1=0,
                           block_ranks=np.zeros(t, np.int32), timings_ms=np.zeros(3), status=-1, stats={})
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=M.device)
    Z = torch.empty((n, n), dtype=M.dtype, device=M.device).t() if want_Z else None
    S = torch.empty((n, m), dtype=M.dtype, device=M.device).t() if want_S else None
    kmax = int(lib.lrr_factor_max_rank(ctypes.byref(p))) if want_factors else 0
    F = torch.empty((kmax, n), dtype=M.dtype, device=M.device).t() if want_factors else None
    G = torch.empty((n, kmax), dtype=M.dtype, device=M.device).t() if want_factors else None
    fk = ctypes.c_int32(0)
    sweeps = np.zeros(t, np.int32)
    iters = np.zeros(t, np.int32)
    resid = np.zeros((t, 2), np.float64)
    ranks = np.zeros(t + 2, np.int32)
    tim = np.zeros(3, np.float64)
    r = LrrResult()
    r.Z = ctypes.c_void_p(Z.data_ptr()) if Z is not None else None
    r.S = ctypes.c_void_p(S.data_ptr()) if S is not None else None
    r.iters = iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    r.resid = resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    r.ranks = ranks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    r.timings_ms = tim.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = LrrStats()
    r.stats = ctypes.pointer(st)
    r.F = ctypes.c_void_p(F.data_ptr()) if F is not None else None
    r.G = ctypes.c_void_p(G.data_ptr()) if G is not None else None
    r.factor_k = ctypes.pointer(fk)
    r.sweeps = sweeps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    stream = torch.cuda.current_stream(M.device).cuda_stream
    code = getattr(lib, entry)(ctypes.byref(p), ctypes.byref(opts), ctypes.c_void_p(workspace.data_ptr()),
                               ctypes.c_size_t(workspace.numel()), ctypes.byref(r), ctypes.c_void_p(stream))
    if code < 0 and raise_on_error:
        raise LrrError(code)
    return SolveResult(Z=Z, S=S, iters=iters, resid=resid, rank_M=int(ranks[0]), k1=int(ranks[1]),
                       block_ranks=ranks[2:].copy(), timings_ms=tim, status=int(code),
                       stats={"phase_ms": dict(zip(PHASES, list(st.phase_ms))),
                              "phase_launches": dict(zip(PHASES, list(st.phase_launches))),
                              "launches": int(st.launches), "iterations": int(st.iterations),
                              "svt_sweeps": int(st.svt_sweeps), "svt_calls": int(st.svt_calls)},
                       F=F, G=G, factor_k=int(fk.value), sweeps=sweeps)


def dfc_lrr_solve(M, perm, offsets, opts: LrrOptions, **kw) -> SolveResult:
    """Algorithm 1 through the C ABI (see include/dfc_lrr.h).  perm and/or
    offsets may be None: pass t= (and seed=) and the library draws them."""
    return _solve("dfc_lrr_solve", M, perm, offsets, opts, **kw)


def lrr_solve(M, perm, opts: LrrOptions, **kw) -> SolveResult:
    """Eq. (1) through the C ABI: one block holding every column in `perm` order."""
    n = M.shape[1]
    return _solve("lrr_solve", M, perm, np.array([0, n], np.int64), opts, **kw)


def svt(A, tau: float, no_alloc: bool = False):
    """Singular-value thresholding through the C ABI: returns (J, rank).
    no_alloc=True calls lrr_svt_noalloc (fixed device scratch, no allocation)."""
    import torch
    lib = load()
    A = column_major(A)
    rows, cols = A.shape
    J = torch.empty((cols, rows), dtype=A.dtype, device=A.device).t()
    prec = LRR_PREC_F64 if A.dtype == torch.float64 else LRR_PREC_F32
    rk = ctypes.c_int32(0)
    fn = lib.lrr_svt_noalloc if no_alloc else lib.lrr_svt
    code = fn(ctypes.c_void_p(A.data_ptr()), rows, cols, leading_dim(A), float(tau),
                       ctypes.c_void_p(J.data_ptr()), leading_dim(J), prec, ctypes.byref(rk), ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream))
    if code < 0:
        raise LrrError(code)
    return J, int(rk.value)


def gemm_bf16(A_km, B_km, M: int, N: int, K: int):
    """C = A B on the tensor cores through the C ABI.  A_km: bf16 tensor of
    shape (M, lda) holding A K-major (row m = A[m, :K]); B_km: bf16 tensor of
    shape (N, ldb) holding B K-major (column n = B_km[n, :K]).  Returns C as a
    float32 (M, N) tensor with column-major storage."""
    import torch
    lib = load()
    C = torch.empty((N, M), dtype=torch.float32, device=A_km.device).t()
    code = lib.lrr_gemm_bf16(ctypes.c_void_p(A_km.data_ptr()), A_km.stride(0), ctypes.c_void_p(B_km.data_ptr()),
                             B_km.stride(0), ctypes.c_void_p(C.data_ptr()), C.stride(1), M, N, K,
                             ctypes.c_void_p(torch.cuda.current_stream(A_km.device).cuda_stream))
    if code < 0:
        raise LrrError(code)
    return C


def gemm_f32(A_km, B_km, M: int, N: int, K: int):
    """C = A B on the tensor cores in split TF32 through the C ABI.  A_km:
    float32 tensor of shape (M, lda) holding A K-major; B_km: float32 (N, ldb)
    holding B K-major.  Returns C as a float32 (M, N) column-major tensor."""
    import torch
    lib = load()
    C = torch.empty((N, M), dtype=torch.float32, device=A_km.device).t()
    code = lib.lrr_gemm_f32(ctypes.c_void_p(A_km.data_ptr()), A_km.stride(0), ctypes.c_void_p(B_km.data_ptr()),
                            B_km.stride(0), ctypes.c_void_p(C.data_ptr()), C.stride(1), M, N, K,
                            ctypes.c_void_p(torch.cuda.current_stream(A_km.device).cuda_stream))
    if code < 0:
        raise LrrError(code)
    return C


def unrolled_options(lam: float, K: int, mu0: float = 1e-6, rho: float = 1.1, mu_max: float = 1e10,
                     checkpoint: int = 5, precision: str = "f32", rank_tol: float = 0.0) -> LrrUnrolledOptions:
    o = LrrUnrolledOptions()
    o.lambda_, o.rho, o.mu0, o.mu_max, o.rank_tol = float(lam), float(rho), float(mu0), float(mu_max), rank_tol
    o.K, o.checkpoint, o.precision = int(K), int(checkpoint), PRECISIONS[precision]
    return o


def unrolled_forward(M, opts: LrrUnrolledOptions):
    """Z_K (n x n, column-major) of K unrolled ALM iterations through the C ABI."""
    import torch
    lib = load()
    M = column_major(M)
    m, n = M.shape
    Z = torch.empty((n, n), dtype=M.dtype, device=M.device).t()
    code = lib.lrr_unrolled_forward(ctypes.c_void_p(M.data_ptr()), m, n, leading_dim(M), ctypes.byref(opts),
                                    ctypes.c_void_p(Z.data_ptr()), n, None, 0,
                                    ctypes.c_void_p(torch.cuda.current_stream(M.device).cuda_stream))
    if code < 0:
        raise LrrError(code)
    return Z


def unrolled_backward(M, opts: LrrUnrolledOptions, Zbar):
    """(dL/dM, dL/dlambda) for Zbar = dL/dZ_K through the C ABI."""
    import torch
    lib = load()
    M = column_major(M)
    Zbar = column_major(Zbar.to(M.dtype))
    m, n = M.shape
    Mb = torch.empty((n, m), dtype=M.dtype, device=M.device).t()
    lb = ctypes.c_double(0.0)
    code = lib.lrr_unrolled_backward(ctypes.c_void_p(M.data_ptr()), m, n, leading_dim(M), ctypes.byref(opts),
                                     ctypes.c_void_p(Zbar.data_ptr()), leading_dim(Zbar),
                                     ctypes.c_void_p(Mb.data_ptr()), m, ctypes.byref(lb), None, 0,
                                     ctypes.c_void_p(torch.cuda.current_stream(M.device).cuda_stream))
    if code < 0:
        raise LrrError(code)
    return Mb, lb.value


def _unrolled_function():
    import torch

    class UnrolledLRR(torch.autograd.Function):
        """Z_K(M, lambda) of K unrolled ALM iterations; backward by the
        library's hand-written reverse pass (checkpointed recompute)."""

        @staticmethod
        def forward(ctx, M, lam, K, mu0, rho, mu_max, checkpoint):
            prec = "f64" if M.dtype == torch.float64 else "f32"
            opts = unrolled_options(float(lam), K, mu0=mu0, rho=rho, mu_max=mu_max, checkpoint=checkpoint,
                                    precision=prec)
            ctx.save_for_backward(M)
            ctx.opts = opts
            return unrolled_forward(M, opts)

        @staticmethod
        def backward(ctx, gZ):
            (M,) = ctx.saved_tensors
            Mb, lb = unrolled_backward(M, ctx.opts, gZ)
            return Mb, torch.tensor(lb, dtype=M.dtype, device=M.device), None, None, None, None, None

    return UnrolledLRR


def unrolled_lrr(M, lam, K: int, mu0: float = 1e-6, rho: float = 1.1, mu_max: float = 1e10, checkpoint: int = 5):
    """Differentiable Z_K(M, lam) (torch.autograd): gradients reach M and lam
    (a 0-d tensor) through lrr_unrolled_backward."""
    import torch
    if not torch.is_tensor(lam):
        lam = torch.tensor(float(lam), dtype=M.dtype, device=M.device)
    return _unrolled_function().apply(M, lam, K, mu0, rho, mu_max, checkpoint)


def gemm_timing(kind: str, M: int, N: int, K: int, repeat: int = 20) -> float:
    """Mean device time (ms) of one launch of the bf16 ("bf16"), split-bf16
    ("bf16x3") or split-TF32 ("3xtf32") tensor-core product at M x N x K
    (lrr_gemm_timing)."""
    import torch
    ms = ctypes.c_double(0.0)
    code = load().lrr_gemm_timing({"bf16": 0, "3xtf32": 1, "bf16x3": 2}[kind], M, N, K, repeat, ctypes.byref(ms),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if code < 0:
        raise LrrError(code)
    return ms.value


def segment(F, G, k: int, clusters: int, rel_tol: float = 1e-6, seed: int = 0, restarts: int = 20,
            power_iters: int = 100):
    """Cluster labels (numpy int32, n) of the estimate Z = F[:, :k] G[:k] on the
    GPU (lrr_segment); F, G as returned by a solve with want_factors=True."""
    import torch
    lib = load()
    F = column_major(F.float())
    G = column_major(G.float())
    n = F.shape[0]
    labels = np.zeros(n, np.int32)
    code = lib.lrr_segment(ctypes.c_void_p(F.data_ptr()), leading_dim(F), ctypes.c_void_p(G.data_ptr()),
                           leading_dim(G), n, int(k), int(clusters), float(rel_tol), int(seed) & 0xFFFFFFFFFFFFFFFF,
                           int(restarts), int(power_iters), labels.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           None, 0, ctypes.c_void_p(torch.cuda.current_stream(F.device).cuda_stream))
    if code < 0:
        raise LrrError(code)
    return labels


def dfc_lrr_solve_local(M, perm, offsets, opts: LrrOptions, rank: int = 0, streams: int = 8):
    """The footnote variant (dictionary C_i per block, C step = truncated SVD of
    diag(Z_1..Z_t)) through the C ABI.  Returns a SolveResult (no factors)."""
    import torch
    lib = load()
    M = column_major(M)
    m, n = M.shape
    p, keep = _problem(M, perm, offsets)
    t = p.t
    Z = torch.empty((n, n), dtype=M.dtype, device=M.device).t()
    S = torch.empty((n, m), dtype=M.dtype, device=M.device).t()
    iters = np.zeros(t, np.int32)
    resid = np.zeros((t, 2), np.float64)
    ranks = np.zeros(t + 2, np.int32)
    sweeps = np.zeros(t, np.int32)
    r = LrrResult()
    r.Z, r.S = ctypes.c_void_p(Z.data_ptr()), ctypes.c_void_p(S.data_ptr())
    r.iters = iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    r.resid = resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    r.ranks = ranks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    r.sweeps = sweeps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    code = lib.dfc_lrr_solve_local(ctypes.byref(p), ctypes.byref(opts), int(rank), ctypes.byref(r), int(streams),
                                   ctypes.c_void_p(torch.cuda.current_stream(M.device).cuda_stream))
    if code < 0:
        raise LrrError(code)
    return SolveResult(Z=Z, S=S, iters=iters, resid=resid, rank_M=int(ranks[0]), k1=int(ranks[1]),
                       block_ranks=ranks[2:].copy(), timings_ms=np.zeros(3), status=int(code), stats={},
                       sweeps=sweeps)


def solve_batch(Ms, opts: LrrOptions, streams: int = 8, want_Z=True, want_S=True, parts=None):
    """Independent problems (a list of column-major CUDA tensors, each solved
    as plain LRR unless `parts` gives (perm, offsets) per problem) on
    concurrent streams (lrr_solve_batch).  Returns (list of (Z, S, iters),
    per-problem status)."""
    import torch
    lib = load()
    cnt = len(Ms)
    probs = (LrrProblem * cnt)()
    res = (LrrResult * cnt)()
    keep, outs = [], []
    for i, M in enumerate(Ms):
        M = column_major(M)
        m, n = M.shape
        perm, off = parts[i] if parts is not None else (np.arange(n, dtype=np.int64), np.array([0, n], np.int64))
        p, kp = _problem(M, perm, off)
        keep += kp + [M]
        probs[i] = p
        Z = torch.empty((n, n), dtype=M.dtype, device=M.device).t() if want_Z else None
        S = torch.empty((n, m), dtype=M.dtype, device=M.device).t() if want_S else None
        it = np.zeros(p.t, np.int32)
        keep.append(it)
        res[i].Z = ctypes.c_void_p(Z.data_ptr()) if Z is not None else None
        res[i].S = ctypes.c_void_p(S.data_ptr()) if S is not None else None
        res[i].iters = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        outs.append((Z, S, it))
    st = np.zeros(cnt, np.int32)
    code = lib.lrr_solve_batch(probs, cnt, ctypes.byref(opts), res, st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               int(streams), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if code < 0:
        raise LrrError(code)
    return outs, st
