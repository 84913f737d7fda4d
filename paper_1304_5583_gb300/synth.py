"""Seeded synthetic inputs for DFC-LRR (union-of-subspaces data with outliers).

This module draws random numbers only: data matrices, the random column
partition of the D step and its block sizes.  It holds none of the solver's
arithmetic, so both the CUDA path and the CPU oracle can consume its output.

Data model (Section 4.1.1, "Simulations"): k independent r-dimensional
subspaces of R^m, each with an orthonormal basis U_i drawn uniformly (Haar),
n_s points per subspace X_i = U_i T_i, and a fraction of outlier columns.
The workload recipes below vary that model as follows (stated per recipe):

* ``gaussian``: T_i ~ N(0,1); a fraction of the columns is *replaced* by
  N(0,1) columns rescaled to the median inlier column norm.
* ``faces``: T_i ~ N(0,1), the whole matrix is shifted to be nonnegative and
  scaled into [0,1]; in a fraction of the columns a fraction of the entries is
  overwritten by U[0,1] values (a stand-in for shadowed face images, Sec. 4.1.2).
* ``paper``: the paper's own generator: T_i ~ U[0,1], n_o = g/(1-g) k n_s
  appended N(0, s^2) outlier columns with s the mean absolute inlier entry,
  then a random column permutation.

The D step (Section 2.2, Algorithm 1 SampleCols) is a uniformly random
partition of the columns into t blocks; ``column_partition`` draws the
permutation and block sizes (even, or an uneven Dirichlet split with bounds).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def haar_orthonormal(rng: np.random.Generator, m: int, r: int) -> np.ndarray:
    """m x r matrix with orthonormal columns drawn from the Haar measure
    (QR of a Gaussian matrix with the signs of R's diagonal folded into Q)."""
    g = rng.standard_normal((m, r))
    q, rr = np.linalg.qr(g)
    d = np.sign(np.diag(rr))
    d[d == 0] = 1.0
    return q * d


@dataclass
class SubspaceData:
    M: np.ndarray                 # m x n, float64, column-major semantics (columns = points)
    labels: np.ndarray            # n, subspace index of each column, -1 for outliers
    outlier: np.ndarray           # n, bool
    k: int                        # number of subspaces
    rank: int                     # rank of each subspace
    bases: list = field(default_factory=list)   # U_i, m x r each


def union_of_subspaces(seed: int, m: int, k: int, r: int, n_s: int, outlier_frac: float,
                       recipe: str = "gaussian", corrupt_entry_frac: float = 0.1) -> SubspaceData:
    """Draw an m x n union-of-subspaces matrix (see the module docstring)."""
    rng = np.random.default_rng(seed)
    bases = [haar_orthonormal(rng, m, r) for _ in range(k)]
    if recipe == "paper":
        X0 = np.concatenate([U @ rng.uniform(0.0, 1.0, (r, n_s)) for U in bases], axis=1)
        n_o = int(round(outlier_frac / (1.0 - outlier_frac) * k * n_s))
        sigma = float(np.mean(np.abs(X0)))
        S = rng.normal(0.0, sigma, (m, n_o))
        labels = np.concatenate([np.repeat(np.arange(k), n_s), -np.ones(n_o, dtype=np.int64)])
        M = np.concatenate([X0, S], axis=1)
        p = rng.permutation(M.shape[1])
        M = M[:, p]
        labels = labels[p]
        return SubspaceData(M=np.ascontiguousarray(M), labels=labels, outlier=labels < 0,
                            k=k, rank=r, bases=bases)

    X0 = np.concatenate([U @ rng.standard_normal((r, n_s)) for U in bases], axis=1)
    n = k * n_s
    labels = np.repeat(np.arange(k), n_s).astype(np.int64)
    if recipe == "gaussian":
        n_out = int(round(outlier_frac * n))
        idx = np.sort(rng.choice(n, n_out, replace=False))
        med = float(np.median(np.linalg.norm(X0, axis=0)))
        G = rng.standard_normal((m, n_out))
        G *= med / np.linalg.norm(G, axis=0)
        M = X0.copy()
        M[:, idx] = G
        labels[idx] = -1
        return SubspaceData(M=M, labels=labels, outlier=labels < 0, k=k, rank=r, bases=bases)
    if recipe == "faces":
        M = X0 - X0.min()
        M /= M.max()
        n_cor = int(round(outlier_frac * n))
        cols = np.sort(rng.choice(n, n_cor, replace=False))
        n_ent = int(round(corrupt_entry_frac * m))
        for j in cols:
            rows = rng.choice(m, n_ent, replace=False)
            M[rows, j] = rng.uniform(0.0, 1.0, n_ent)
        outlier = np.zeros(n, dtype=bool)
        outlier[cols] = True
        return SubspaceData(M=M, labels=labels, outlier=outlier, k=k, rank=r, bases=bases)
    raise ValueError(f"unknown recipe {recipe!r}")


def column_partition(seed: int, n: int, t: int, min_cols: int | None = None,
                     max_cols: int | None = None, alpha: float = 1.0):
    """D step draw: a uniformly random permutation of the n columns and t block
    sizes.  With no bounds the split is even (the paper's t | n case; the last
    block takes the remainder).  With bounds, the sizes are min_cols plus a
    multinomial share of the rest under Dirichlet(alpha) weights, redrawn until
    every size is <= max_cols.  Returns (perm int64[n], offsets int64[t+1]);
    block i holds the original columns perm[offsets[i]:offsets[i+1]]."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n).astype(np.int64)
    if min_cols is None and max_cols is None:
        base = n // t
        sizes = np.full(t, base, dtype=np.int64)
        sizes[: n - base * t] += 1
    else:
        lo = int(min_cols or 1)
        hi = int(max_cols or n)
        extra = n - lo * t
        if extra < 0 or hi * t < n:
            raise ValueError("infeasible block-size bounds")
        for _ in range(10000):
            w = rng.dirichlet(np.full(t, alpha))
            sizes = lo + rng.multinomial(extra, w).astype(np.int64)
            if sizes.max() <= hi:
                break
        else:
            raise RuntimeError("could not draw block sizes within bounds")
    offsets = np.zeros(t + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    assert offsets[-1] == n
    return perm, offsets


@dataclass
class Workload:
    name: str
    data: SubspaceData
    perm: np.ndarray
    offsets: np.ndarray
    lam: float
    rho: float = 1.1
    mu0: float = 1e-6
    mu_max: float = 1e10
    eps: float = 1e-6
    max_iter: int = 1000

    @property
    def M(self):
        return self.data.M

    @property
    def t(self):
        return len(self.offsets) - 1


def workload(name: str, seed: int = 0) -> Workload:
    """The named synthetic workloads used by the tests and the benchmark.

    plain_lrr_100x500      : 5 rank-5 subspaces in R^100, 100 points each, 10% outlier
                             columns replaced; t=1; lambda=0.1, eps=1e-8 (float64 solve)
    dfc_500x5000           : 10 rank-10 subspaces in R^500, 500 points each, 5% outliers;
                             t=10 Dirichlet blocks of >= 200 columns; lambda=0.1
    dfc_faces_2016x2432    : 38 rank-9 subspaces in R^2016, 64 points each, face-like
                             nonnegative data, 10% of the entries of 20% of the columns
                             corrupted; t=8 uneven blocks (>= 200); lambda=0.15
    dfc_1000x20000         : 20 rank-20 subspaces in R^1000, 1000 points each, 5% outliers;
                             t=40 blocks of 400-600 columns; lambda=0.1, eps=1e-6
    diff_200x1000          : 5 rank-8 subspaces in R^200, 200 points each, 5% outliers; t=1
    tiny_20x30             : 3 rank-2 subspaces in R^20, 10 points each, 10% outliers; t=1
    small_dfc_60x240       : 4 rank-3 subspaces in R^60, 60 points each, 5% outliers; t=3
                             uneven blocks (>= 64)
    """
    if name == "plain_lrr_100x500":
        d = union_of_subspaces(seed, 100, 5, 5, 100, 0.10)
        perm, off = column_partition(seed + 1, d.M.shape[1], 1)
        return Workload(name, d, perm, off, lam=0.1, eps=1e-8)
    if name == "dfc_500x5000":
        d = union_of_subspaces(seed, 500, 10, 10, 500, 0.05)
        perm, off = column_partition(seed + 1, d.M.shape[1], 10, min_cols=200)
        return Workload(name, d, perm, off, lam=0.1, eps=1e-6)
    if name == "dfc_faces_2016x2432":
        d = union_of_subspaces(seed, 2016, 38, 9, 64, 0.20, recipe="faces", corrupt_entry_frac=0.10)
        perm, off = column_partition(seed + 1, d.M.shape[1], 8, min_cols=200)
        return Workload(name, d, perm, off, lam=0.15, eps=1e-6)
    if name == "dfc_1000x20000":
        d = union_of_subspaces(seed, 1000, 20, 20, 1000, 0.05)
        perm, off = column_partition(seed + 1, d.M.shape[1], 40, min_cols=400, max_cols=600, alpha=4.0)
        return Workload(name, d, perm, off, lam=0.1, eps=1e-6)
    if name == "diff_200x1000":
        d = union_of_subspaces(seed, 200, 5, 8, 200, 0.05)
        perm, off = column_partition(seed + 1, d.M.shape[1], 1)
        return Workload(name, d, perm, off, lam=0.1, eps=1e-6)
    if name == "tiny_20x30":
        d = union_of_subspaces(seed, 20, 3, 2, 10, 0.10)
        perm, off = column_partition(seed + 1, d.M.shape[1], 1)
        return Workload(name, d, perm, off, lam=0.5, eps=1e-8)
    if name == "small_dfc_60x240":
        d = union_of_subspaces(seed, 60, 4, 3, 60, 0.05)
        perm, off = column_partition(seed + 1, d.M.shape[1], 3, min_cols=64)
        return Workload(name, d, perm, off, lam=0.2, eps=1e-6)
    raise KeyError(name)


WORKLOADS = ("plain_lrr_100x500", "dfc_500x5000", "dfc_faces_2016x2432", "dfc_1000x20000",
             "diff_200x1000", "tiny_20x30", "small_dfc_60x240")
