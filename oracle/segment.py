"""Segmentation post-processing of an LRR estimate.  TEST INFRASTRUCTURE ONLY.

Section 4.1.2: the affinity U_Z U_Z^T is built from the top left singular
vectors of the estimate Z, the points are embedded spectrally in k
dimensions and clustered by k-means; each cluster is labelled by majority
vote of the ground truth, and the segmentation accuracy is the per-class
percentage of correctly labelled points, averaged over the classes.

Readings (the paper leaves these open): "top" singular vectors are those with
sigma > rel_tol * sigma_max; the affinity is the entrywise absolute value
|U U^T|; the embedding is the k eigenvectors of the normalised Laplacian
I - D^-1/2 A D^-1/2 with the smallest eigenvalues, rows scaled to unit norm;
k-means is Lloyd's method from k-means++ seeds with a fixed seed, best of
``restarts`` runs.  Everything is deterministic for a fixed seed, so two
estimates can be compared label for label.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment


def affinity(Z: np.ndarray, rel_tol: float = 1e-6, basis: np.ndarray = None) -> np.ndarray:
    """|U U^T| from the left singular vectors U of Z with s > rel_tol * s_max.
    ``basis``: an orthonormal Q whose span holds every column of Z (Z = Q Q^T Z,
    as for the C step's output, Q = Q1); then Z = Q (Q^T Z) and the left
    singular vectors of Z are Q times those of the small matrix Q^T Z, with
    the same singular values -- the same U without an SVD of the n x n Z."""
    if basis is None:
        U, s, _ = np.linalg.svd(Z, full_matrices=False)
    else:
        Ub, s, _ = np.linalg.svd(basis.T @ Z, full_matrices=False)
        U = basis @ Ub
    k = int(np.count_nonzero(s > rel_tol * s[0])) if s.size and s[0] > 0 else 0
    Uk = U[:, :k]
    return np.abs(Uk @ Uk.T)


def spectral_embedding(A: np.ndarray, k: int, subset: bool = None) -> np.ndarray:
    """``subset`` (default: n > 5000): compute only the k eigenpairs with the
    smallest eigenvalues (LAPACK's subset driver) instead of all n."""
    d = A.sum(axis=1)
    dinv = np.where(d > 0, 1.0 / np.sqrt(np.maximum(d, 1e-300)), 0.0)
    L = np.eye(A.shape[0]) - (dinv[:, None] * A) * dinv[None, :]
    if subset is None:
        subset = A.shape[0] > 5000
    if subset:
        from scipy.linalg import eigh as sp_eigh
        w, V = sp_eigh(L, subset_by_index=[0, k - 1], overwrite_a=True, check_finite=False)
    else:
        w, V = np.linalg.eigh(L)
    Y = V[:, :k]
    nrm = np.linalg.norm(Y, axis=1, keepdims=True)
    return Y / np.where(nrm > 0, nrm, 1.0)


def kmeans(Y: np.ndarray, k: int, seed: int = 0, restarts: int = 20, iters: int = 300) -> np.ndarray:
    rng = np.random.default_rng(seed)
    best_lab, best_cost = None, np.inf
    n = Y.shape[0]
    for _ in range(restarts):
        # k-means++ seeding
        centers = [Y[rng.integers(n)]]
        for _c in range(1, k):
            d2 = np.min(((Y[:, None, :] - np.array(centers)[None]) ** 2).sum(-1), axis=1)
            p = d2 / d2.sum() if d2.sum() > 0 else np.full(n, 1.0 / n)
            centers.append(Y[rng.choice(n, p=p)])
        C = np.array(centers)
        lab = None
        for _it in range(iters):
            d2 = ((Y[:, None, :] - C[None]) ** 2).sum(-1)
            new = d2.argmin(axis=1)
            if lab is not None and np.array_equal(new, lab):
                break
            lab = new
            for j in range(k):
                pts = Y[lab == j]
                if len(pts):
                    C[j] = pts.mean(axis=0)
        cost = float(((Y - C[lab]) ** 2).sum())
        if cost < best_cost - 1e-12:
            best_cost, best_lab = cost, lab.copy()
    return best_lab


def segment(Z: np.ndarray, k: int, seed: int = 0, basis: np.ndarray = None) -> np.ndarray:
    """Cluster labels (0..k-1) of the n points from an n x n estimate Z
    (``basis`` as for affinity)."""
    return kmeans(spectral_embedding(affinity(Z, basis=basis), k), k, seed=seed)


def matched_accuracy(labels: np.ndarray, truth: np.ndarray) -> float:
    """Fraction of points labelled correctly under the best one-to-one
    matching of clusters to classes (Hungarian matching)."""
    ks = int(max(labels.max(), truth.max())) + 1
    W = np.zeros((ks, ks))
    for a, b in zip(labels, truth):
        W[a, b] += 1
    r, c = linear_sum_assignment(-W)
    return float(W[r, c].sum() / len(labels))


def majority_vote_accuracy(labels: np.ndarray, truth: np.ndarray) -> float:
    """Section 4.1.2's measure: every cluster takes the majority ground-truth
    label of its members; accuracy is averaged over the classes."""
    pred = np.empty_like(truth)
    for c in np.unique(labels):
        members = labels == c
        vals, cnt = np.unique(truth[members], return_counts=True)
        pred[members] = vals[cnt.argmax()]
    accs = [float(np.mean(pred[truth == c] == c)) for c in np.unique(truth)]
    return float(np.mean(accs))


def same_partition(a: np.ndarray, b: np.ndarray) -> bool:
    """True if two labelings define the same partition (equal up to renaming)."""
    if a.shape != b.shape:
        return False
    pairs = {}
    back = {}
    for x, y in zip(a.tolist(), b.tolist()):
        if pairs.setdefault(x, y) != y or back.setdefault(y, x) != x:
            return False
    return True
