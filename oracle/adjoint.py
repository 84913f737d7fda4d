"""Reverse-mode derivative of K unrolled inexact-ALM iterations of LRR, in
float64.  TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline).

The map differentiated is plain LRR (eq. (1), t = 1, the observations are the
dictionary: C = M) run for exactly K iterations of the inexact ALM that
oracle.lrr states (J-step, Z-step, E-step, then the dual step; the K-th
iteration stops before its dual step), from the zero start:

    Z_K(M, lam) = ALM^K(M, lam)

The penalty schedule mu_k = min(rho^(k-1) mu0, mu_max) does not depend on M or
lam and is held fixed.  The backward pass visits the iterations in reverse and
the steps of each in reverse, with these adjoints (bar = d loss / d value):

  dual step      Y1' = Y1 + mu (C - M Z - E),  Y2' = Y2 + mu (Z - J)
  E-step         E = shrink(X, lam/mu), X = C - M Z + Y1/mu; on a column with
                 ||x|| > theta:  e = (1 - theta/||x||) x, so
                 xbar = (1 - theta/||x||) ebar + theta (x.ebar) x / ||x||^3 and
                 d/dtheta = -(x/||x||).ebar;  zero columns pass nothing back
  product        M Z:  Mbar += (MZ)bar Z^T,  Zbar += M^T (MZ)bar
  Z-step         Z = S^-1 R with S = I + M^T M:  Q = S^-1 Zbar,  Rbar = Q,
                 Mbar -= (M Z) Q^T + (M Q) Z^T
  right side     R = M^T (C - E) + J + (M^T Y1 - Y2)/mu
  J-step         J = SVT_tau(A), A = Z + Y2/mu, tau = 1/mu: the derivative of
                 the singular-value function f(s) = max(s - tau, 0) (below)
and C = M adds the observation path's adjoint to the dictionary's.

SVT derivative (derived): for A = U diag(s) V^T (thin, square or tall) and
P = U^T dA V,
  U^T dJ V = diag(f'(s_i) P_ii) + G+ o sym(P) + G- o skew(P)  (off-diagonal)
  G+_ij = (f(s_i) - f(s_j)) / (s_i - s_j),  G-_ij = (f(s_i) + f(s_j)) / (s_i + s_j)
plus, for a tall A, (I - U U^T) dA V diag(f(s)/s) V^T.  The map is
self-adjoint in this form, so the adjoint applies it to Jbar.

Checkpointing: the forward pass keeps the state (Z, E, Y1, Y2) every
`checkpoint` iterations and the backward pass recomputes each segment from its
checkpoint before reversing it.
"""
from __future__ import annotations

import numpy as np

from oracle import lrr


def _mu_schedule(K, mu0, rho, mu_max):
    mus, mu = [], mu0
    for _ in range(K):
        mus.append(mu)
        mu = min(rho * mu, mu_max)
    return mus


def _step(M, Ms, state, mu, lam, last):
    """One iteration from state (Z, E, Y1, Y2); returns the new state and the
    intermediate values the backward pass needs."""
    Z, E, Y1, Y2 = state
    C = M
    A = Z + Y2 / mu
    J = lrr.svt(A, 1.0 / mu)[0]
    R = M.T @ (C - E) + J + (M.T @ Y1 - Y2) / mu
    Zn = Ms(R)
    MZ = M @ Zn
    X = C - MZ + Y1 / mu
    En = lrr.col_shrink(X, lam / mu)
    if last:
        Y1n, Y2n = Y1, Y2
    else:
        Y1n = Y1 + mu * (C - MZ - En)
        Y2n = Y2 + mu * (Zn - J)
    return (Zn, En, Y1n, Y2n), dict(A=A, J=J, Z=Zn, MZ=MZ, X=X, E_in=E, Y1_in=Y1, Y2_in=Y2)


def unrolled_forward(M, lam, K, mu0=1e-6, rho=1.1, mu_max=1e10, checkpoint=0):
    """Z_K after K iterations from the zero start; with checkpoint > 0 also the
    states at iterations 0, checkpoint, 2 checkpoint, ... (list of tuples)."""
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    Ms = lrr.ZSolve(M)
    state = (np.zeros((n, n)), np.zeros((m, n)), np.zeros((m, n)), np.zeros((n, n)))
    cps = []
    for k, mu in enumerate(_mu_schedule(K, mu0, rho, mu_max)):
        if checkpoint and k % checkpoint == 0:
            cps.append(state)
        state, _ = _step(M, Ms, state, mu, lam, k == K - 1)
    return (state[0], cps) if checkpoint else state[0]


def svt_adjoint(A, tau, Jbar):
    """Adjoint of J = SVT_tau(A) at A applied to Jbar (see the module docstring)."""
    A = np.asarray(A, dtype=np.float64)
    if A.shape[0] < A.shape[1]:
        return svt_adjoint(A.T, tau, Jbar.T).T
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    V = Vt.T
    f = np.maximum(s - tau, 0.0)
    fp = (s > tau).astype(np.float64)
    si, sj = s[:, None], s[None, :]
    fi, fj = f[:, None], f[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        gp = np.where(np.abs(si - sj) > 0, (fi - fj) / (si - sj), fp[:, None] * np.ones_like(sj))
        gm = np.where(si + sj > 0, (fi + fj) / (si + sj), 0.0)
        fs = np.where(s > 0, f / s, 0.0)
    P = U.T @ Jbar @ V
    Ps, Pa = 0.5 * (P + P.T), 0.5 * (P - P.T)
    core = gp * Ps + gm * Pa
    np.fill_diagonal(core, fp * np.diag(P))
    out = U @ core @ Vt
    # left complement of a tall A
    out += (Jbar @ V - U @ (U.T @ Jbar @ V)) * fs @ Vt
    return out


def shrink_adjoint(X, theta, Ebar):
    """Adjoint of E = col_shrink(X, theta): returns (Xbar, dL/dtheta)."""
    nrm = np.linalg.norm(X, axis=0)
    act = nrm > theta
    Xbar = np.zeros_like(X)
    dth = 0.0
    if act.any():
        x, e, r = X[:, act], Ebar[:, act], nrm[act]
        xe = np.sum(x * e, axis=0)
        Xbar[:, act] = (1.0 - theta / r) * e + theta * xe / r ** 3 * x
        dth = float(-np.sum(xe / r))
    return Xbar, dth


def unrolled_grad(M, lam, K, Zbar, mu0=1e-6, rho=1.1, mu_max=1e10, checkpoint=5):
    """Gradients (dL/dM, dL/dlam) of a loss L(Z_K) given Zbar = dL/dZ_K."""
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    Ms = lrr.ZSolve(M)
    mus = _mu_schedule(K, mu0, rho, mu_max)
    cp = max(1, int(checkpoint))
    _, cps = unrolled_forward(M, lam, K, mu0, rho, mu_max, checkpoint=cp)
    Mbar = np.zeros_like(M)
    lbar = 0.0
    # adjoints of the state leaving the current iteration
    Zb, Eb, Y1b, Y2b = np.array(Zbar, dtype=np.float64), np.zeros((m, n)), np.zeros((m, n)), np.zeros((n, n))
    for seg in reversed(range(len(cps))):
        k0, k1 = seg * cp, min(K, (seg + 1) * cp)
        # recompute the segment's intermediates from its checkpoint
        state, saved = cps[seg], []
        for k in range(k0, k1):
            state, sv = _step(M, Ms, state, mus[k], lam, k == K - 1)
            saved.append(sv)
        for k in reversed(range(k0, k1)):
            sv, mu = saved[k - k0], mus[k]
            Cb = np.zeros_like(M)
            MZb = np.zeros_like(M)
            Jb = np.zeros((n, n))
            # dual step (not taken at the K-th iteration)
            if k != K - 1:
                Cb += mu * Y1b
                MZb -= mu * Y1b
                Eb = Eb - mu * Y1b
                Zb = Zb + mu * Y2b
                Jb -= mu * Y2b
            Y1_in_b, Y2_in_b = Y1b.copy(), Y2b.copy()
            # E-step
            Xb, dth = shrink_adjoint(sv["X"], lam / mu, Eb)
            lbar += dth / mu
            Cb += Xb
            MZb -= Xb
            Y1_in_b += Xb / mu
            # M Z
            Mbar += MZb @ sv["Z"].T
            Zb = Zb + M.T @ MZb
            # Z-step
            Q = Ms(Zb)
            Mbar -= sv["MZ"] @ Q.T + (M @ Q) @ sv["Z"].T
            Rb = Q
            # right side R = M^T (C - E) + J + (M^T Y1 - Y2)/mu
            Mbar += (M - sv["E_in"] + sv["Y1_in"] / mu) @ Rb.T
            Cb += M @ Rb
            E_in_b = -(M @ Rb)
            Jb += Rb
            Y1_in_b += (M @ Rb) / mu
            Y2_in_b -= Rb / mu
            # J-step
            Ab = svt_adjoint(sv["A"], 1.0 / mu, Jb)
            Z_in_b = Ab
            Y2_in_b += Ab / mu
            # observations are the dictionary
            Mbar += Cb
            Zb, Eb, Y1b, Y2b = Z_in_b, E_in_b, Y1_in_b, Y2_in_b
    return Mbar, lbar


def weighted_loss(Z, W):
    """L = ||Z o W||_F^2 (the loss of the differentiable configuration)."""
    return float(np.sum((Z * W) ** 2))
