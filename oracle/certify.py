"""Optimality certificates and an independent brute-force solver for eq. (2).
TEST INFRASTRUCTURE ONLY.

Duality (derived from the Lagrangian of eq. (2)):
  primal  p* = min ||Z||_* + lam ||S||_{2,1}  s.t.  C = M Z + S
  dual    d* = max <C, Y>  s.t.  ||M^T Y||_2 <= 1  and  max_j ||Y_j||_2 <= lam
(the conjugates of ||.||_* and lam||.||_{2,1} are the indicators of the
spectral-norm unit ball and of the column-norm ball of radius lam).  Any
primal-feasible pair bounds p* from above and any dual-feasible Y bounds it
from below, so a small gap certifies a solution without trusting the solver
that produced it.

The optimality conditions of Theorem 6 (Appendix, "Conditions for
Optimality") in the form used here: with Q the dual variable,
M^T Q is a subgradient of ||.||_* at Z and Q is lam times a subgradient of
||.||_{2,1} at S.
"""
from __future__ import annotations

import numpy as np


def primal_value(C, M, Z, lam):
    """Objective at the feasible pair (Z, S = C - M Z)."""
    S = C - M @ Z
    return float(np.linalg.svd(Z, compute_uv=False).sum() + lam * np.linalg.norm(S, axis=0).sum())


def dual_value(C, M, Y, lam):
    """<C, Y> after scaling Y into the dual feasible set; returns (value, scale)."""
    spec = float(np.linalg.norm(M.T @ Y, 2))
    colmax = float(np.linalg.norm(Y, axis=0).max()) if Y.size else 0.0
    s = max(spec, colmax / lam, 1e-300)
    return float(np.sum(C * Y) / s), s


def duality_gap(C, M, Z, Y, lam):
    """(primal, dual, relative gap) for a primal estimate Z and dual estimate Y."""
    p = primal_value(C, M, Z, lam)
    d, _ = dual_value(C, M, Y, lam)
    return p, d, (p - d) / max(abs(p), 1e-300)


def subgradient_solve(C, M, lam, f_lower, iters=10000):
    """Brute force: subgradient descent on the unconstrained equivalent
    min_Z f(Z) = ||Z||_* + lam ||C - M Z||_{2,1} with Polyak's step
    (f(Z) - f_lower)/||g||^2, where f_lower is any certified lower bound (a
    dual value), keeping the best iterate.  A subgradient of f is
    U V^T - lam M^T N, with U V^T from the SVD of Z (nonzero part only) and N
    the column-normalised residual (zero columns give zero).  Slow and simple;
    for tiny inputs only."""
    n = M.shape[1]
    Z = np.zeros((n, C.shape[1]))
    best, bestZ = np.inf, Z.copy()
    for _ in range(iters):
        U, s, Vt = np.linalg.svd(Z, full_matrices=False)
        nz = s > 1e-12
        R = C - M @ Z
        nr = np.linalg.norm(R, axis=0)
        N = np.where(nr > 1e-12, R / np.where(nr > 1e-12, nr, 1.0), 0.0)
        f = s.sum() + lam * nr.sum()
        if f < best:
            best, bestZ = f, Z.copy()
        g = U[:, nz] @ Vt[nz] - lam * (M.T @ N)
        Z = Z - (f - f_lower) / max(float((g * g).sum()), 1e-300) * g
    return bestZ, best
