"""CPU float64 oracle for LRR and DFC-LRR.  TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg use
this module.  It shares no code with the CUDA library: plain numpy/LAPACK in
float64, written for readability, with every step in the order the method
states it.

What it computes
----------------
LRR, eq. (1): min ||Z||_* + lam ||S||_{2,1} s.t. M = M Z + S, with ||.||_* the
nuclear norm and ||.||_{2,1} the sum of column 2-norms (Section 1).

DFC-LRR, Algorithm 1 (Section 2.2):
  D step  -- columns of M split at random into t blocks C_i (the permutation
             and block sizes are inputs: they are random draws);
  F step  -- each block solves eq. (2):
             min ||Z_i||_* + lam ||S_i||_{2,1} s.t. C_i = M Z_i + S_i
             with M, the whole input, as the dictionary;
  C step  -- column projection of [Z_1 ... Z_t] onto the column space of Z_1.

Base solver (Section 4: the inexact augmented Lagrange multiplier method is
the base LRR algorithm; the paper cites it without writing it out).  Restated
here from the augmented Lagrangian of eq. (2) with the splitting Z = J:

  L = ||J||_* + lam||E||_{2,1} + <Y1, C - M Z - E> + <Y2, Z - J>
      + mu/2 (||C - M Z - E||_F^2 + ||Z - J||_F^2)

  each iteration minimises L over J, then Z, then E, then takes a dual ascent
  step:
    J <- argmin_J 1/mu ||J||_* + 1/2 ||J - (Z + Y2/mu)||^2
         = singular-value thresholding of Z + Y2/mu at 1/mu
    Z <- (I + M^T M)^{-1} (M^T (C - E) + J + (M^T Y1 - Y2)/mu)
    E <- argmin_E lam/mu ||E||_{2,1} + 1/2 ||E - (C - M Z + Y1/mu)||^2
         = column shrinkage of C - M Z + Y1/mu at lam/mu
    stop if max(||C - M Z - E||_inf, ||Z - J||_inf) < eps
    Y1 <- Y1 + mu (C - M Z - E);  Y2 <- Y2 + mu (Z - J);  mu <- min(rho mu, mu_max)
  starting from Z = J = E = Y1 = Y2 = 0, mu = mu0.

Readings where the paper is silent:
  * the iteration above, its zero start and its stopping rule (absolute
    infinity-norm residuals, checked before the dual step; no dual step is
    taken on the stopping iteration);
  * the returned block estimate is Z_i; the column space of Z_1 used by the
    C step is the column space of the factored SVT output J_1 of the final
    iteration (rank k1 = number of singular values above the final 1/mu),
    orthonormalised by a QR that drops columns with |R_jj| < 1e-10 max|R_jj|;
  * for t = 1 the C step is the identity (Z_1 projected on its own column
    space) and is skipped;
  * the Z-update solves with a Cholesky factor of I + M^T M when n <= 2432,
    otherwise through the Woodbury identity
      (I_n + M^T M)^{-1} = I_n - M^T (I_m + M M^T)^{-1} M
    with a Cholesky factor of I_m + M M^T;
  * the residual C - M Z uses a directly computed product M Z.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


# --------------------------------------------------------------------------
# proximal operators (closed forms of the two norms' proximal maps)
# --------------------------------------------------------------------------

def svt(A: np.ndarray, tau: float):
    """Singular-value thresholding: argmin_J tau||J||_* + 1/2||J - A||_F^2.

    Closed form U diag(max(s - tau, 0)) V^T from a full (thin) SVD of A.
    Returns (J, U_k, s_k - tau, Vt_k) where k = #{s > tau}; the last three are
    the factored form of J."""
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    k = int(np.count_nonzero(s > tau))
    sk = s[:k] - tau
    J = (U[:, :k] * sk) @ Vt[:k]
    return J, U[:, :k], sk, Vt[:k]


def col_shrink(X: np.ndarray, tau: float) -> np.ndarray:
    """Column-wise shrinkage: argmin_E tau||E||_{2,1} + 1/2||E - X||_F^2.

    Column j becomes max(0, 1 - tau/||x_j||) x_j (zero when x_j = 0)."""
    norms = np.linalg.norm(X, axis=0)
    scale = np.zeros_like(norms)
    nz = norms > tau
    scale[nz] = 1.0 - tau / norms[nz]
    return X * scale


def nuclear_norm(Z: np.ndarray) -> float:
    return float(np.linalg.svd(Z, compute_uv=False).sum())


def l21_norm(S: np.ndarray) -> float:
    return float(np.linalg.norm(S, axis=0).sum())


def lrr_objective(Z: np.ndarray, S: np.ndarray, lam: float) -> float:
    """Objective of eq. (1)/(2): ||Z||_* + lam ||S||_{2,1}."""
    return nuclear_norm(Z) + lam * l21_norm(S)


# --------------------------------------------------------------------------
# Z-update system (I + M^T M) Z = R
# --------------------------------------------------------------------------

class ZSolve:
    """Solves (I_n + M^T M) Z = R.  Direct Cholesky of the n x n matrix when
    n <= direct_max, else the Woodbury identity with the m x m Cholesky factor
    of I_m + M M^T."""

    def __init__(self, M: np.ndarray, direct_max: int = 2432):
        self.M = M
        m, n = M.shape
        self.direct = n <= direct_max
        if self.direct:
            self.cf = sla.cho_factor(np.eye(n) + M.T @ M, lower=True)
        else:
            self.cf = sla.cho_factor(np.eye(m) + M @ M.T, lower=True)

    def __call__(self, R: np.ndarray) -> np.ndarray:
        if self.direct:
            return sla.cho_solve(self.cf, R)
        W = sla.cho_solve(self.cf, self.M @ R)
        return R - self.M.T @ W


# --------------------------------------------------------------------------
# inexact ALM for one LRR subproblem, eq. (2)
# --------------------------------------------------------------------------

@dataclass
class LRRResult:
    Z: np.ndarray
    E: np.ndarray
    J: np.ndarray
    Y1: np.ndarray
    Y2: np.ndarray
    mu: float            # mu used in the final iteration
    iters: int
    resid_primal: float  # ||C - M Z - E||_inf at the final iteration
    resid_zj: float      # ||Z - J||_inf at the final iteration
    rank: int            # SVT rank of J at the final iteration
    J_U: np.ndarray      # left factor of J (n x rank)
    J_s: np.ndarray      # thresholded singular values (rank)
    J_Vt: np.ndarray     # right factor of J (rank x l)
    converged: bool
    trace: list


def lrr_alm(C: np.ndarray, M: np.ndarray, lam: float, rho: float = 1.1, mu0: float = 1e-6,
            mu_max: float = 1e10, eps: float = 1e-8, max_iter: int = 1000,
            fixed_iters: int | None = None, zsolve: ZSolve | None = None,
            keep_trace: bool = False) -> LRRResult:
    """Inexact ALM for min ||Z||_* + lam||E||_{2,1} s.t. C = M Z + E (eq. (2);
    eq. (1) when C = M).  With ``fixed_iters`` the stopping test is ignored and
    exactly that many iterations run (used to compare two implementations
    iteration for iteration)."""
    C = np.asarray(C, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    l = C.shape[1]
    zs = zsolve if zsolve is not None else ZSolve(M)
    Z = np.zeros((n, l)); J = np.zeros((n, l)); E = np.zeros((m, l))
    Y1 = np.zeros((m, l)); Y2 = np.zeros((n, l))
    mu = mu0
    trace = []
    n_iter = fixed_iters if fixed_iters is not None else max_iter
    converged = False
    it = 0
    for it in range(1, n_iter + 1):
        mu_it = mu
        # J: proximal step of (1/mu)||.||_* at Z + Y2/mu
        A = Z + Y2 / mu
        J, JU, Js, JVt = svt(A, 1.0 / mu)
        # Z: stationary point of the quadratic part
        R = M.T @ (C - E) + J + (M.T @ Y1 - Y2) / mu
        Z = zs(R)
        # E: proximal step of (lam/mu)||.||_{2,1}
        MZ = M @ Z
        E = col_shrink(C - MZ + Y1 / mu, lam / mu)
        # residuals of the two constraints
        leq1 = C - MZ - E
        leq2 = Z - J
        r1 = float(np.abs(leq1).max()) if leq1.size else 0.0
        r2 = float(np.abs(leq2).max()) if leq2.size else 0.0
        if keep_trace:
            # (mu, primal residual, ||Z - J||_inf, SVT rank, ||SVT input||_F)
            trace.append((mu, r1, r2, JU.shape[1], float(np.linalg.norm(A))))
        if fixed_iters is None and max(r1, r2) < eps:
            converged = True
            break
        if fixed_iters is not None and it == fixed_iters:
            converged = max(r1, r2) < eps
            break
        # dual ascent and penalty growth
        Y1 = Y1 + mu * leq1
        Y2 = Y2 + mu * leq2
        mu = min(rho * mu, mu_max)
    return LRRResult(Z=Z, E=E, J=J, Y1=Y1, Y2=Y2, mu=mu_it, iters=it, resid_primal=r1,
                     resid_zj=r2, rank=JU.shape[1], J_U=JU, J_s=Js, J_Vt=JVt,
                     converged=converged, trace=trace)


# --------------------------------------------------------------------------
# C step: column projection (Section 2.2, Algorithm 1 ColProj)
# --------------------------------------------------------------------------

def orth_basis(U: np.ndarray, drop_tol: float = 1e-10) -> np.ndarray:
    """Orthonormal basis of span(U) by Householder QR; columns whose |R_jj| is
    below drop_tol * max|R_jj| are dropped."""
    if U.shape[1] == 0:
        return U.copy()
    Q, R = np.linalg.qr(U)
    d = np.abs(np.diag(R))
    keep = d >= drop_tol * d.max()
    return Q[:, keep]


def col_proj(Z_blocks: list, basis: np.ndarray) -> np.ndarray:
    """[Z_1 ... Z_t] projected onto span(basis): Q Q^T [Z_1 ... Z_t] with Q an
    orthonormal basis of span(basis)."""
    Q = orth_basis(basis)
    Zc = np.concatenate(Z_blocks, axis=1)
    return Q @ (Q.T @ Zc)


# --------------------------------------------------------------------------
# DFC-LRR driver (Algorithm 1)
# --------------------------------------------------------------------------

@dataclass
class DFCResult:
    Z: np.ndarray         # n x n, columns in the original order
    S: np.ndarray         # m x n, columns in the original order
    iters: np.ndarray     # t
    resid: np.ndarray     # t x 2 (primal, Z - J)
    k1: int               # rank of the C-step basis
    blocks: list          # per-block LRRResult


_WORKER = {}


def _worker_init(M):
    _WORKER["M"] = M
    _WORKER["zs"] = ZSolve(M)


def _worker_block(args):
    cols, lam, rho, mu0, mu_max, eps, max_iter, fi = args
    M = _WORKER["M"]
    return lrr_alm(M[:, cols], M, lam, rho, mu0, mu_max, eps, max_iter, fixed_iters=fi, zsolve=_WORKER["zs"])


def dfc_lrr(M: np.ndarray, perm: np.ndarray, offsets: np.ndarray, lam: float, rho: float = 1.1,
            mu0: float = 1e-6, mu_max: float = 1e10, eps: float = 1e-6, max_iter: int = 1000,
            fixed_iters=None, blocks_only=None, workers: int = 0) -> DFCResult:
    """Algorithm 1.  ``perm``/``offsets`` are the D step's random draw: block i
    observes the original columns perm[offsets[i]:offsets[i+1]].  ``fixed_iters``
    may be an int or a per-block sequence.  ``blocks_only`` restricts the F
    step to the listed block indices (then no C step is taken).  With
    ``workers`` > 1 the independent block problems of the F step ("do in
    parallel") run in that many spawned processes; the arithmetic is the same."""
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    t = len(offsets) - 1
    which = list(range(t) if blocks_only is None else blocks_only)

    def fixed(i):
        return fixed_iters[i] if isinstance(fixed_iters, (list, tuple, np.ndarray)) else fixed_iters

    res = {}
    if workers > 1 and len(which) > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        jobs = [(perm[offsets[i]:offsets[i + 1]], lam, rho, mu0, mu_max, eps, max_iter, fixed(i)) for i in which]
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                 initializer=_worker_init, initargs=(M,)) as ex:
            for i, r in zip(which, ex.map(_worker_block, jobs)):
                res[i] = r
    else:
        zs = ZSolve(M)
        for i in which:
            cols = perm[offsets[i]:offsets[i + 1]]
            res[i] = lrr_alm(M[:, cols], M, lam, rho, mu0, mu_max, eps, max_iter, fixed_iters=fixed(i), zsolve=zs)
    iters = np.array([res[i].iters if i in res else 0 for i in range(t)], dtype=np.int64)
    resid = np.array([[res[i].resid_primal, res[i].resid_zj] if i in res else [0.0, 0.0]
                      for i in range(t)])
    if blocks_only is not None:
        return DFCResult(Z=None, S=None, iters=iters, resid=resid, k1=res[min(res)].rank if res else 0,
                         blocks=[res.get(i) for i in range(t)])
    blocks = [res[i] for i in range(t)]
    if t == 1:
        Zc = blocks[0].Z
        k1 = blocks[0].rank
    else:
        Q = orth_basis(blocks[0].J_U)
        k1 = Q.shape[1]
        Zc = col_proj([b.Z for b in blocks], Q)
    Ec = np.concatenate([b.E for b in blocks], axis=1)
    Z = np.empty((n, n)); S = np.empty((m, n))
    Z[:, perm] = Zc
    S[:, perm] = Ec
    return DFCResult(Z=Z, S=S, iters=iters, resid=resid, k1=k1, blocks=blocks)


# --------------------------------------------------------------------------
# Footnote variant of the F and C steps (Section 2.2, footnote to eq. (2))
# --------------------------------------------------------------------------

def lowrank_blockdiag(Z_blocks: list, k: int):
    """Best rank-k approximation (truncated SVD) of the block-diagonal matrix
    diag(Z_1, ..., Z_t).  Its singular triplets are the union of the blocks'
    triplets, so the k largest singular values over all blocks are kept, each
    block keeping its own.  Ties are broken by block order, then by position.
    Returns the list of truncated blocks."""
    svds = [np.linalg.svd(Zb, full_matrices=False) for Zb in Z_blocks]
    allv = [(-s[j], b, j) for b, (_, s, _) in enumerate(svds) for j in range(len(s))]
    allv.sort()
    keep = {(b, j) for _, b, j in allv[:max(0, int(k))]}
    out = []
    for b, (U, s, Vt) in enumerate(svds):
        idx = [j for j in range(len(s)) if (b, j) in keep]
        out.append((U[:, idx] * s[idx]) @ Vt[idx] if idx else np.zeros_like(Z_blocks[b]))
    return out


def dfc_lrr_local(M: np.ndarray, perm: np.ndarray, offsets: np.ndarray, lam: float, rho: float = 1.1,
                  mu0: float = 1e-6, mu_max: float = 1e10, eps: float = 1e-6, max_iter: int = 1000,
                  fixed_iters=None, k=None) -> DFCResult:
    """The alternative formulation of the footnote to eq. (2): both instances
    of M in the block problem become C_i,
        min ||Z_i||_* + lam ||S_i||_{2,1}  s.t.  C_i = C_i Z_i + S_i   (Z_i: l_i x l_i),
    and the C step is a low-rank approximation of diag(Z_1, ..., Z_t), here
    the truncated SVD at rank k (reading: the footnote leaves the rank open;
    by default k = k1, the SVT rank of block 1 at its final iteration, the
    same rank the column projection keeps).  Z is n x n with block i's
    rows and columns at the original columns perm[offsets[i]:offsets[i+1]]."""
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    t = len(offsets) - 1
    blocks = []
    for i in range(t):
        cols = perm[offsets[i]:offsets[i + 1]]
        C = M[:, cols]
        fi = fixed_iters[i] if isinstance(fixed_iters, (list, tuple, np.ndarray)) else fixed_iters
        blocks.append(lrr_alm(C, C, lam, rho, mu0, mu_max, eps, max_iter, fixed_iters=fi))
    k1 = blocks[0].rank if k is None else int(k)
    approx = lowrank_blockdiag([b.Z for b in blocks], k1)
    Z = np.zeros((n, n))
    S = np.empty((m, n))
    for i in range(t):
        cols = perm[offsets[i]:offsets[i + 1]]
        Z[np.ix_(cols, cols)] = approx[i]
        S[:, cols] = blocks[i].E
    iters = np.array([b.iters for b in blocks], dtype=np.int64)
    resid = np.array([[b.resid_primal, b.resid_zj] for b in blocks])
    return DFCResult(Z=Z, S=S, iters=iters, resid=resid, k1=k1, blocks=blocks)
