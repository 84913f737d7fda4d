"""Phase-transition sweep of Section 4.1.1 (the paper's first simulation) on
the GPU: for each outlier fraction, independent trials of the paper's
generator (k subspaces of dimension r in R^m, n_s points each with U[0,1]
coefficients, n_o = gamma/(1-gamma) k n_s appended N(0, s^2) outlier columns,
a random column permutation), solved by LRR and by DFC-LRR with t blocks, all
problems of a sweep at once on concurrent streams (lrr_solve_batch).

Success is the paper's criterion: the oracle constraints of the Appendix hold
within 1e-4 -- the columns of Z lie in the row space of L0 (the inlier
columns, outliers zeroed) and S is supported on the outlier columns.  Read as
max |P Z - Z| <= tol and max |S on inlier columns| <= tol, P the projector
onto the row space of L0.  The check runs on the host on the returned
estimates (it evaluates the method, it is not part of it).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import binding, synth


@dataclass
class Trial:
    gamma: float
    seed: int
    data: synth.SubspaceData
    V0: np.ndarray                  # n x rank(L0): row space of the inlier part
    perm: np.ndarray = None
    offsets: np.ndarray = None


def row_space_of_inliers(d: synth.SubspaceData, tol: float = 1e-10) -> np.ndarray:
    L0 = d.M.copy()
    L0[:, d.outlier] = 0.0
    _, s, Vt = np.linalg.svd(L0, full_matrices=False)
    k = int((s > tol * s[0]).sum())
    return Vt[:k].T


def oracle_constraints_hold(Z: np.ndarray, S: np.ndarray, V0: np.ndarray, outlier: np.ndarray,
                            tol: float = 1e-4) -> bool:
    """The Appendix's oracle constraints within tol (max-abs): P_{L0^T} Z = Z and
    S supported on the outlier columns."""
    Z = np.asarray(Z, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    zres = np.abs(V0 @ (V0.T @ Z) - Z).max() if Z.size else 0.0
    sres = np.abs(S[:, ~outlier]).max() if (~outlier).any() else 0.0
    return bool(zres <= tol and sres <= tol)


def make_trials(gammas, trials: int, m: int, k: int, r: int, n_s: int, t: int, seed: int = 0):
    out = []
    for gi, g in enumerate(gammas):
        for j in range(trials):
            sd = seed + 1000 * gi + j
            d = synth.union_of_subspaces(sd, m, k, r, n_s, g, recipe="paper")
            tr = Trial(gamma=g, seed=sd, data=d, V0=row_space_of_inliers(d))
            if t > 1:
                tr.perm, tr.offsets = synth.column_partition(sd + 7, d.M.shape[1], t)
            out.append(tr)
    return out


@dataclass
class SweepResult:
    gammas: list
    success: dict = field(default_factory=dict)   # gamma -> fraction of trials
    per_trial: list = field(default_factory=list)  # (gamma, seed, ok, iters)
    seconds: float = 0.0
    problems: int = 0


def sweep(gammas, trials: int = 10, m: int = 1500, k: int = 3, r: int = 5, n_s: int = 200, lam: float = 0.2,
          t: int = 1, precision: str = "f32", eps: float = 1e-6, streams: int = 8, seed: int = 0) -> SweepResult:
    """Success frequency of LRR (t = 1) or DFC-LRR (t > 1) per outlier fraction."""
    import torch
    trs = make_trials(gammas, trials, m, k, r, n_s, t, seed)
    dt = torch.float64 if precision == "f64" else torch.float32
    Ms = [torch.from_numpy(np.asfortranarray(tr.data.M)).to(dt).cuda() for tr in trs]
    parts = [(tr.perm, tr.offsets) for tr in trs] if t > 1 else None
    o = binding.options(lam, eps=eps, precision=precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs, st = binding.solve_batch(Ms, o, streams=streams, parts=parts)
    torch.cuda.synchronize()
    res = SweepResult(gammas=list(gammas), seconds=time.perf_counter() - t0, problems=len(trs))
    for tr, (Z, S, it), code in zip(trs, outs, st):
        ok = code >= 0 and oracle_constraints_hold(Z.cpu().numpy(), S.cpu().numpy(), tr.V0, tr.data.outlier)
        res.per_trial.append((tr.gamma, tr.seed, bool(ok), it.tolist()))
    for g in gammas:
        oks = [p[2] for p in res.per_trial if p[0] == g]
        res.success[g] = float(np.mean(oks)) if oks else 0.0
    return res
