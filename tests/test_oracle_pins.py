"""Pins for the CPU oracle: closed forms, a hand-worked example, optimality
certificates, a brute-force solver and the paper's structural facts.  None of
these compares the oracle with itself."""
import json
import os

import numpy as np
import pytest

from oracle import certify, lrr, segment
from paper_1304_5583_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- closed forms

def test_svt_closed_form_on_diagonal_input():
    """SVT of P1 diag(d) P2 (signed permutations) is P1 diag(sign(d) max(|d|-tau,0)) P2."""
    rng = np.random.default_rng(3)
    d = np.array([3.0, -0.5, 1.25, -2.0, 0.1])
    tau = 0.7
    P1 = np.eye(7)[:, rng.permutation(7)][:, :5]          # 7 x 5 partial permutation
    P2 = np.eye(5)[rng.permutation(5)] * rng.choice([-1.0, 1.0], 5)[:, None]
    A = P1 @ np.diag(d) @ P2
    J, U, s, Vt = lrr.svt(A, tau)
    expect = P1 @ np.diag(np.sign(d) * np.maximum(np.abs(d) - tau, 0.0)) @ P2
    assert np.allclose(J, expect, atol=1e-14)
    assert U.shape[1] == 3
    assert np.allclose(np.sort(s)[::-1], [2.3, 1.3, 0.55])


def test_svt_is_the_proximal_point():
    """A - J = tau (U_k V_k^T + W) with ||W||_2 <= 1, W orthogonal to U_k and V_k."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((9, 6)) @ np.diag([5, 3, 1, 0.5, 0.2, 0.05])
    tau = 0.4
    J, U, s, Vt = lrr.svt(A, tau)
    G = (A - J) / tau
    assert np.linalg.norm(G, 2) <= 1 + 1e-12
    W = G - U @ Vt
    assert np.allclose(U.T @ W, 0, atol=1e-12) and np.allclose(W @ Vt.T, 0, atol=1e-12)
    obj = lambda X: tau * np.linalg.svd(X, compute_uv=False).sum() + 0.5 * np.sum((X - A) ** 2)
    f0 = obj(J)
    for _ in range(50):
        assert obj(J + 1e-3 * rng.standard_normal(J.shape)) >= f0 - 1e-12


def test_col_shrink_closed_form():
    X = np.array([[3.0, 0.3, 0.0], [4.0, 0.4, 0.0]])
    E = lrr.col_shrink(X, 1.0)
    assert np.allclose(E, [[2.4, 0.0, 0.0], [3.2, 0.0, 0.0]], atol=1e-15)
    # boundary: a column whose norm equals tau is zeroed
    assert np.all(lrr.col_shrink(np.array([[0.6], [0.8]]), 1.0) == 0.0)


# ------------------------------------------------------------ hand-worked ALM

@pytest.mark.parametrize("n_iter", [1, 2])
def test_two_alm_iterations_match_hand_derivation(n_iter):
    g = json.load(open(os.path.join(GOLDEN, "alm_diag_2x3.json")))
    M = np.array(g["M"])
    r = lrr.lrr_alm(M, M, g["lam"], rho=g["rho"], mu0=g["mu0"], fixed_iters=n_iter)
    e = g[f"after_iter_{n_iter}"]
    assert np.allclose(r.Z, np.diag(e["Z_diag"]), atol=1e-14)
    assert np.allclose(r.J, np.diag(e["J_diag"]), atol=1e-14)
    E = np.zeros((2, 3)); E[0, 0] = e["E11"]; E[1, 1] = e["E22"]
    assert np.allclose(r.E, E, atol=1e-14)
    assert r.resid_primal == pytest.approx(e["resid_primal"], abs=1e-14)
    assert r.resid_zj == pytest.approx(e["resid_zj"], abs=1e-14)
    assert r.rank == e["rank"]


# ----------------------------------------------------- solutions and certificates

def _small_problem(seed=5, m=30, k=3, rdim=2, n_s=15, frac=0.1):
    d = synth.union_of_subspaces(seed, m, k, rdim, n_s, frac)
    return d


def test_converged_solution_has_small_duality_gap_and_kkt():
    """The duality gap certifies the ALM point.  With the geometric penalty
    growth rho = 1.1 the inexact ALM stops slightly short of the optimum (the
    sum of 1/mu_k is finite), so the certified gap there is ~1e-5; a slower
    schedule (rho = 1.02) must close it to 1e-8, which it could not do if a
    term of the iteration were wrong."""
    d = _small_problem()
    M = d.M
    lam = 0.3
    r = lrr.lrr_alm(M, M, lam, eps=1e-9, max_iter=2000)
    assert r.converged
    assert max(r.resid_primal, r.resid_zj) < 1e-9
    p, dv, gap = certify.duality_gap(M, M, r.Z, r.Y1, lam)
    assert 0 <= gap < 2e-5, (p, dv, gap)
    slow = lrr.lrr_alm(M, M, lam, rho=1.02, eps=1e-9, max_iter=5000)
    _, _, gap_slow = certify.duality_gap(M, M, slow.Z, slow.Y1, lam)
    assert 0 <= gap_slow < 1e-8, gap_slow
    # KKT (Theorem 6 form, Q = Y1) at the slow-schedule point: M^T Y1 ~ Y2,
    # ||Y2||_2 <= 1, ||Y1_j|| <= lam and Y1_j = lam E_j/||E_j|| on E's support
    r = slow
    assert np.linalg.norm(M.T @ r.Y1 - r.Y2) / np.linalg.norm(r.Y2) < 1e-6
    assert np.linalg.norm(r.Y2, 2) <= 1 + 1e-6
    cn = np.linalg.norm(r.Y1, axis=0)
    assert cn.max() <= lam * (1 + 1e-9)
    sup = np.linalg.norm(r.E, axis=0) > 1e-8
    assert sup.any()
    dirs = r.E[:, sup] / np.linalg.norm(r.E[:, sup], axis=0)
    assert np.allclose(r.Y1[:, sup], lam * dirs, atol=1e-6)


def test_brute_force_subgradient_agrees_on_tiny_problem():
    """On a 20 x 30 input, subgradient descent on the unconstrained form of
    eq. (1) and the ALM agree on the optimal value.  The slow-schedule ALM is
    certified optimal by its duality gap; the rho = 1.1 ALM is within the
    inexact-ALM shortfall of it; the subgradient search approaches it from
    above and never beats the certified lower bound."""
    w = synth.workload("tiny_20x30")
    M = w.M
    slow = lrr.lrr_alm(M, M, w.lam, rho=1.02, eps=1e-10, max_iter=5000)
    p_slow, d_slow, gap_slow = certify.duality_gap(M, M, slow.Z, slow.Y1, w.lam)
    assert 0 <= gap_slow < 1e-7
    fast = lrr.lrr_alm(M, M, w.lam, eps=1e-10, max_iter=3000)
    f_fast = certify.primal_value(M, M, fast.Z, w.lam)
    assert d_slow <= f_fast and (f_fast - p_slow) / p_slow < 5e-4
    Zb, f_bf = certify.subgradient_solve(M, M, w.lam, d_slow, iters=10000)
    assert f_bf >= d_slow
    assert (f_bf - p_slow) / p_slow < 5e-4, (p_slow, f_bf)
    assert np.linalg.norm(Zb - slow.Z) / np.linalg.norm(slow.Z) < 0.05


def test_noiseless_independent_subspaces_give_shape_interaction_matrix():
    """Clean data from independent subspaces: Z = V V^T (the shape interaction
    matrix, block diagonal after sorting by subspace), S = 0 (Section 2.1),
    when lam exceeds max_j ||(M^+)^T e_j|| (derived sufficient condition)."""
    d = synth.union_of_subspaces(11, 40, 3, 3, 20, 0.0)
    M = d.M
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    r = int((s > 1e-10 * s[0]).sum())
    V = Vt[:r].T
    pinvT_cols = np.linalg.norm((U[:, :r] / s[:r]) @ Vt[:r], axis=0)
    lam = 1.5 * pinvT_cols.max()
    res = lrr.lrr_alm(M, M, lam, eps=1e-10, max_iter=3000)
    assert np.allclose(res.Z, V @ V.T, atol=1e-7)
    assert np.abs(res.E).max() < 1e-7
    lab = d.labels
    off = lab[:, None] != lab[None, :]
    assert np.abs(res.Z[off]).max() < 1e-7


def test_column_projection_is_exact_when_block_one_spans():
    """Cor. 4: if Z_1 spans the column space of [Z_1..Z_t], ColProj returns it."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((50, 4))
    blocks = [A @ rng.standard_normal((4, l)) for l in (12, 9, 15)]
    out = lrr.col_proj(blocks, blocks[0])
    assert np.allclose(out, np.concatenate(blocks, axis=1), atol=1e-12)
    # a block outside the span is changed
    blocks[1] = rng.standard_normal((50, 9))
    out = lrr.col_proj(blocks, blocks[0])
    assert not np.allclose(out[:, 12:21], blocks[1])
    # rank-deficient basis: duplicated columns are dropped
    Q = lrr.orth_basis(np.concatenate([A, A[:, :2]], axis=1))
    assert Q.shape[1] == 4 and np.allclose(Q.T @ Q, np.eye(4), atol=1e-12)


def test_dfc_with_one_block_is_lrr():
    w = synth.workload("tiny_20x30")
    M = w.M
    perm = np.random.default_rng(2).permutation(M.shape[1])
    dfc = lrr.dfc_lrr(M, perm, np.array([0, M.shape[1]]), w.lam, eps=1e-8)
    ref = lrr.lrr_alm(M, M, w.lam, eps=1e-8)
    assert dfc.iters[0] == ref.iters
    assert np.allclose(dfc.Z, ref.Z, atol=1e-10)
    assert np.allclose(dfc.S, ref.E, atol=1e-10)


def test_woodbury_and_direct_z_solves_agree():
    rng = np.random.default_rng(9)
    M = rng.standard_normal((12, 40))
    R = rng.standard_normal((40, 7))
    a = lrr.ZSolve(M, direct_max=10_000)(R)
    b = lrr.ZSolve(M, direct_max=10)(R)
    assert np.allclose((np.eye(40) + M.T @ M) @ a, R, atol=1e-10)
    assert np.allclose(a, b, atol=1e-10)


def test_oracle_constraints_on_paper_generator():
    """Section 4.1.1 success criterion: the oracle constraints (Appendix,
    eq. oracle-constraints) hold within 1e-4: Z lies in the row space of L0
    and S is supported on the outlier columns."""
    d = synth.union_of_subspaces(1, 60, 3, 3, 30, 0.1, recipe="paper")
    M = d.M
    r = lrr.lrr_alm(M, M, 0.5, eps=1e-8, max_iter=2000)
    L0 = M.copy(); L0[:, d.outlier] = 0.0
    U0, s0, Vt0 = np.linalg.svd(L0, full_matrices=False)
    k = int((s0 > 1e-10 * s0[0]).sum())
    V0 = Vt0[:k].T
    assert np.abs(V0 @ (V0.T @ r.Z) - r.Z).max() < 1e-4
    assert np.abs(r.E[:, ~d.outlier]).max() < 1e-4
    assert np.linalg.norm(r.E[:, d.outlier], axis=0).min() > 0.1   # outliers identified


def test_segmentation_of_clean_data_is_perfect():
    d = synth.union_of_subspaces(12, 50, 4, 3, 25, 0.0)
    M = d.M
    r = lrr.lrr_alm(M, M, 0.5, eps=1e-8)
    lab = segment.segment(r.Z, d.k, seed=0)
    assert segment.matched_accuracy(lab, d.labels) == 1.0
    assert segment.majority_vote_accuracy(lab, d.labels) == 1.0
    assert segment.same_partition(lab, d.labels)


# ------------------------------------------------ planted mistakes are caught

def _pins_hold():
    """The hand-worked two-iteration pin and the shape-interaction pin, as one
    boolean (used to show that planted mistakes are caught)."""
    try:
        g = json.load(open(os.path.join(GOLDEN, "alm_diag_2x3.json")))
        M = np.array(g["M"])
        e = g["after_iter_2"]
        r = lrr.lrr_alm(M, M, g["lam"], rho=g["rho"], mu0=g["mu0"], fixed_iters=2)
        hand = (np.allclose(np.diag(r.Z), e["Z_diag"], atol=1e-12)
                and np.allclose(np.diag(r.J), e["J_diag"], atol=1e-12)
                and abs(r.E[0, 0] - e["E11"]) < 1e-12)
        d = synth.union_of_subspaces(11, 40, 3, 3, 20, 0.0)
        U, s_, Vt = np.linalg.svd(d.M, full_matrices=False)
        k = int((s_ > 1e-10 * s_[0]).sum())
        lam = 1.5 * np.linalg.norm((U[:, :k] / s_[:k]) @ Vt[:k], axis=0).max()
        res = lrr.lrr_alm(d.M, d.M, lam, eps=1e-10, max_iter=3000)
        shape = np.allclose(res.Z, Vt[:k].T @ Vt[:k], atol=1e-7)
        return hand and shape
    except (ValueError, np.linalg.LinAlgError):
        return False


def test_planted_mistakes_are_caught(monkeypatch):
    """A halved shrink threshold, a doubled SVT threshold and a transposed
    operand in the Z-update system each break at least one pin."""
    assert _pins_hold()
    orig_shrink, orig_svt, orig_zs = lrr.col_shrink, lrr.svt, lrr.ZSolve

    monkeypatch.setattr(lrr, "col_shrink", lambda X, tau: orig_shrink(X, 0.5 * tau))
    assert not _pins_hold()
    monkeypatch.setattr(lrr, "col_shrink", orig_shrink)

    monkeypatch.setattr(lrr, "svt", lambda A, tau: orig_svt(A, 2 * tau))
    assert not _pins_hold()
    monkeypatch.setattr(lrr, "svt", orig_svt)

    class Transposed(orig_zs):
        """Solves with I + M M^T (zero-padded) where I + M^T M is meant."""
        def __init__(self, M_, direct_max=2432):
            super().__init__(M_, direct_max)
            import scipy.linalg as sla
            K = np.zeros((M_.shape[1], M_.shape[1]))
            m_ = min(M_.shape[0], M_.shape[1])
            K[:m_, :m_] = (M_ @ M_.T)[:m_, :m_]
            self.cf = sla.cho_factor(np.eye(M_.shape[1]) + K, lower=True)
    monkeypatch.setattr(lrr, "ZSolve", Transposed)
    assert not _pins_hold()
    monkeypatch.setattr(lrr, "ZSolve", orig_zs)
    assert _pins_hold()


# --------------------------------------------- the DFC driver with t > 1 blocks

def _subspace_projectors(d):
    """Per subspace k, the n x n projector P_k onto the row space of that
    subspace's columns (zero outside its own rows and columns).  For
    independent subspaces the shape-interaction matrix V V^T of M is the sum
    of the P_k (Section 2.1: block diagonal after sorting by subspace)."""
    n = d.M.shape[1]
    out = []
    for k in range(d.k):
        idx = np.flatnonzero(d.labels == k)
        _, s, Vt = np.linalg.svd(d.M[:, idx], full_matrices=False)
        rk = int((s > 1e-10 * s[0]).sum())
        P = np.zeros((n, n))
        P[np.ix_(idx, idx)] = Vt[:rk].T @ Vt[:rk]
        out.append(P)
    return out


def _block_lambda(M, perm, offsets):
    """A lam above which every clean block problem of eq. (2) has S = 0 and
    Z_i = M^+ C_i (derived sufficient condition): with Z_i = U_z S_z V_z^T,
    Y = (M^+)^T U_z V_z^T is a dual certificate (M^T Y = U_z V_z^T is a
    subgradient of the nuclear norm at Z_i) whose columns must have norm
    below lam.  Returns 1.5 times the largest such column norm."""
    Mp = np.linalg.pinv(M, rcond=1e-10)
    worst = 0.0
    for i in range(len(offsets) - 1):
        Zi = Mp @ M[:, perm[offsets[i]:offsets[i + 1]]]
        Uz, sz, Vzt = np.linalg.svd(Zi, full_matrices=False)
        kz = int((sz > 1e-10 * sz[0]).sum())
        Y = Mp.T @ (Uz[:, :kz] @ Vzt[:kz])
        worst = max(worst, float(np.linalg.norm(Y, axis=0).max()))
    return 1.5 * worst


def _clean_dfc_case():
    """Clean data from 3 independent 3-dimensional subspaces of R^40, 20
    points each, split at random into t = 3 uneven blocks that each hold at
    least 4 points of every subspace (so every block spans the row space)."""
    d = synth.union_of_subspaces(21, 40, 3, 3, 20, 0.0)
    rng = np.random.default_rng(5)
    for _ in range(1000):
        perm = rng.permutation(60).astype(np.int64)
        offsets = np.array([0, 17, 38, 60], dtype=np.int64)
        ok = all(np.bincount(d.labels[perm[offsets[i]:offsets[i + 1]]], minlength=3).min() >= 4 for i in range(3))
        if ok:
            return d, perm, offsets
    raise RuntimeError("no spanning partition drawn")


def _dfc_pin_holds(d, perm, offsets, lam):
    P = _subspace_projectors(d)
    res = lrr.dfc_lrr(d.M, perm, offsets, lam, eps=1e-10, max_iter=3000)
    return (res.Z.shape == (60, 60) and np.allclose(res.Z, sum(P), atol=1e-7)
            and np.abs(res.S).max() < 1e-7 and res.k1 == 9)


def test_dfc_on_spanning_blocks_returns_the_shape_interaction_matrix():
    """Algorithm 1 with t = 3 on clean independent subspaces where every block
    spans the row space of M: each block solution is M^+ C_i = V V^T[:, cols_i],
    Z_1 spans the column space of [Z_1 .. Z_t] (Cor. 4), so the column
    projection is exact and DFC-LRR returns V V^T = sum_k P_k with S = 0, the
    columns back in their original order."""
    d, perm, offsets = _clean_dfc_case()
    lam = _block_lambda(d.M, perm, offsets)
    assert _dfc_pin_holds(d, perm, offsets, lam)


def test_dfc_projects_onto_block_one_when_it_misses_a_subspace():
    """Block 1 holds points of subspaces 0 and 1 only.  Its solution's column
    space is then range(P_0) + range(P_1), and the C step projects every
    block's columns onto it: the estimate is P_0 + P_1 (the columns of
    subspace 2 project to zero), with k1 = 6."""
    d = synth.union_of_subspaces(21, 40, 3, 3, 20, 0.0)
    rng = np.random.default_rng(6)
    lab = d.labels
    first = np.concatenate([rng.permutation(np.flatnonzero(lab == 0))[:7],
                            rng.permutation(np.flatnonzero(lab == 1))[:8]])
    rest = rng.permutation(np.setdiff1d(np.arange(60), first))
    perm = np.concatenate([rng.permutation(first), rest]).astype(np.int64)
    offsets = np.array([0, 15, 38, 60], dtype=np.int64)
    lam = _block_lambda(d.M, perm, offsets)
    P = _subspace_projectors(d)
    res = lrr.dfc_lrr(d.M, perm, offsets, lam, eps=1e-10, max_iter=3000)
    assert res.k1 == 6
    assert np.allclose(res.Z, P[0] + P[1], atol=1e-7)
    assert np.abs(res.S).max() < 1e-7


def test_planted_dfc_driver_mistakes_are_caught(monkeypatch):
    """Blocks concatenated out of order, or the C-step basis taken from the
    last block instead of block 1, each break one of the two DFC pins."""
    d, perm, offsets = _clean_dfc_case()
    lam = _block_lambda(d.M, perm, offsets)
    assert _dfc_pin_holds(d, perm, offsets, lam)
    orig_proj = lrr.col_proj
    monkeypatch.setattr(lrr, "col_proj", lambda Zb, basis: orig_proj(list(Zb)[::-1], basis))
    assert not _dfc_pin_holds(d, perm, offsets, lam)
    monkeypatch.setattr(lrr, "col_proj", orig_proj)
    assert _dfc_pin_holds(d, perm, offsets, lam)

    # basis from the last block: invisible when every block spans, caught by
    # the pin whose block 1 misses a subspace
    seen = []
    orig_alm, orig_orth = lrr.lrr_alm, lrr.orth_basis

    def recording_alm(*a, **k):
        r = orig_alm(*a, **k)
        seen.append(r)
        return r

    def last_block_basis(U, drop_tol=1e-10):
        return orig_orth(seen[-1].J_U if seen else U, drop_tol)

    monkeypatch.setattr(lrr, "lrr_alm", recording_alm)
    monkeypatch.setattr(lrr, "orth_basis", last_block_basis)
    with pytest.raises(AssertionError):
        test_dfc_projects_onto_block_one_when_it_misses_a_subspace()
    monkeypatch.setattr(lrr, "orth_basis", orig_orth)
    monkeypatch.setattr(lrr, "lrr_alm", orig_alm)
    test_dfc_projects_onto_block_one_when_it_misses_a_subspace()


# ------------------------------------------ footnote variant (dictionary C_i)

def test_lowrank_blockdiag_keeps_the_global_top_k():
    """The truncated SVD of a block-diagonal matrix, from blocks with known
    singular values: the k largest over all blocks survive."""
    rng = np.random.default_rng(12)
    specs = [np.array([5.0, 1.0, 0.2]), np.array([3.0, 2.5]), np.array([4.0, 0.1, 0.05, 0.01])]
    blocks = []
    for sv in specs:
        l = len(sv) + 2
        U = np.linalg.qr(rng.standard_normal((l, len(sv))))[0]
        V = np.linalg.qr(rng.standard_normal((l, len(sv))))[0]
        blocks.append((U * sv) @ V.T)
    out = lrr.lowrank_blockdiag(blocks, 4)        # keeps 5, 4, 3, 2.5
    got = [np.linalg.svd(o, compute_uv=False) for o in out]
    assert np.allclose(got[0][:2], [5.0, 0.0], atol=1e-12)
    assert np.allclose(got[1][:2], [3.0, 2.5], atol=1e-12)
    assert np.allclose(got[2][:2], [4.0, 0.0], atol=1e-12)
    # the kept parts are the blocks' own leading triplets
    U, s, Vt = np.linalg.svd(blocks[0])
    assert np.allclose(out[0], s[0] * np.outer(U[:, 0], Vt[0]), atol=1e-12)


def test_footnote_variant_on_clean_blocks_gives_each_blocks_shape_interaction():
    """Clean independent subspaces, every block holding enough points of each:
    with dictionary C_i the block solution is the shape-interaction matrix of
    C_i itself (Section 2.1), V_i V_i^T of C_i's row space; at full rank
    (k = sum of the block ranks) the block-diagonal approximation is exact, so
    the estimate is diag(V_i V_i^T) in the original order, and S = 0."""
    d, perm, offsets = _clean_dfc_case()
    t = len(offsets) - 1
    lam = 0.0
    ranks = []
    expect = np.zeros((60, 60))
    for i in range(t):
        cols = perm[offsets[i]:offsets[i + 1]]
        C = d.M[:, cols]
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        rk = int((s > 1e-10 * s[0]).sum())
        ranks.append(rk)
        expect[np.ix_(cols, cols)] = Vt[:rk].T @ Vt[:rk]
        Cp = np.linalg.pinv(C, rcond=1e-10)
        Zi = Cp @ C
        Uz, sz, Vzt = np.linalg.svd(Zi)
        kz = int((sz > 1e-10).sum())
        lam = max(lam, 1.5 * np.linalg.norm(Cp.T @ (Uz[:, :kz] @ Vzt[:kz]), axis=0).max())
    res = lrr.dfc_lrr_local(d.M, perm, offsets, lam, eps=1e-10, max_iter=3000, k=sum(ranks))
    assert np.allclose(res.Z, expect, atol=1e-7)
    assert np.abs(res.S).max() < 1e-7
    # the default rank is block 1's SVT rank; the approximation has that rank
    # and singular values 1 (every block's are)
    res1 = lrr.dfc_lrr_local(d.M, perm, offsets, lam, eps=1e-10, max_iter=3000)
    assert res1.k1 == ranks[0]
    sv = np.linalg.svd(res1.Z, compute_uv=False)
    assert np.allclose(sv[:ranks[0]], 1.0, atol=1e-7) and sv[ranks[0]] < 1e-7


def test_footnote_variant_with_one_block_is_lrr_truncated():
    w = synth.workload("tiny_20x30")
    M = w.M
    n = M.shape[1]
    perm = np.arange(n)
    res = lrr.dfc_lrr_local(M, perm, np.array([0, n]), w.lam, eps=1e-8)
    ref = lrr.lrr_alm(M, M, w.lam, eps=1e-8)
    U, s, Vt = np.linalg.svd(ref.Z)
    k = ref.rank
    assert np.allclose(res.Z, (U[:, :k] * s[:k]) @ Vt[:k], atol=1e-10)


def test_segmentation_from_the_c_step_basis_equals_the_dense_route():
    """The C step's output lies in span(Q1), so its left singular vectors are
    Q1 times those of Q1^T Z: the affinity from the basis equals the one from
    the SVD of the dense Z, and the k-eigenpair embedding gives the labels of
    the full eigendecomposition."""
    from oracle import segment as seg
    w = synth.workload("small_dfc_60x240")
    M = w.M.astype(np.float64)
    res = lrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps)
    Q = lrr.orth_basis(res.blocks[0].J_U)
    A_dense = seg.affinity(res.Z)
    A_basis = seg.affinity(res.Z, basis=Q)
    assert np.abs(A_dense - A_basis).max() < 1e-10
    Yf = seg.spectral_embedding(A_dense, w.data.k, subset=False)
    Ys = seg.spectral_embedding(A_dense, w.data.k, subset=True)
    # the embeddings agree up to an orthogonal map of the k coordinates
    assert np.abs(Yf @ Yf.T - Ys @ Ys.T).max() < 1e-8
    assert seg.same_partition(seg.kmeans(Yf, w.data.k, seed=0), seg.kmeans(Ys, w.data.k, seed=0))
