"""Pins for the oracle's reverse-mode derivative of unrolled ALM iterations
(oracle/adjoint.py): every adjoint against central finite differences of the
forward map it differentiates, in float64, plus planted mistakes."""
import numpy as np
import pytest

from oracle import adjoint, lrr
from paper_1304_5583_gb300 import synth


def _fd_dir(f, x, dx, h=1e-6):
    return (f(x + h * dx) - f(x - h * dx)) / (2 * h)


@pytest.mark.parametrize("shape", [(9, 6), (6, 9), (7, 7)])
def test_svt_adjoint_matches_central_differences(shape):
    """<Abar, dA> = <Jbar, dJ(A)[dA]> for random directions, on spectra that
    straddle the threshold (kept, dropped and near-threshold values)."""
    rng = np.random.default_rng(sum(shape))
    k = min(shape)
    U = np.linalg.qr(rng.standard_normal((shape[0], k)))[0]
    V = np.linalg.qr(rng.standard_normal((shape[1], k)))[0]
    s = np.linspace(2.0, 0.05, k)
    A = (U * s) @ V.T
    tau = 0.66           # between singular values (the map has a kink at s = tau)
    assert np.min(np.abs(s - tau)) > 1e-3
    Jb = rng.standard_normal(shape)
    Ab = adjoint.svt_adjoint(A, tau, Jb)
    for _ in range(5):
        dA = rng.standard_normal(shape)
        fd = _fd_dir(lambda X: np.sum(Jb * lrr.svt(X, tau)[0]), A, dA)
        assert np.sum(Ab * dA) == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_shrink_adjoint_matches_central_differences():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((5, 8)) * np.array([0.1, 2, 0.3, 1.5, 0.05, 3, 0.9, 1.1])
    theta = 0.8
    Eb = rng.standard_normal(X.shape)
    Xb, dth = adjoint.shrink_adjoint(X, theta, Eb)
    dX = rng.standard_normal(X.shape)
    fd = _fd_dir(lambda Y: np.sum(Eb * lrr.col_shrink(Y, theta)), X, dX)
    assert np.sum(Xb * dX) == pytest.approx(fd, rel=1e-7)
    fdt = (np.sum(Eb * lrr.col_shrink(X, theta + 1e-6)) - np.sum(Eb * lrr.col_shrink(X, theta - 1e-6))) / 2e-6
    assert dth == pytest.approx(fdt, rel=1e-7)


def _small_case():
    d = synth.union_of_subspaces(4, 10, 2, 2, 8, 0.15)
    W = np.random.default_rng(9).standard_normal((16, 16))
    return d.M, W


# a penalty start at which both nonsmooth steps act within the first iterations
MU0, K, LAM = 1.0, 8, 0.6


def test_small_case_exercises_both_prox_steps():
    M, _ = _small_case()
    r = lrr.lrr_alm(M, M, LAM, mu0=MU0, fixed_iters=K, keep_trace=True)
    ranks = [row[3] for row in r.trace]
    assert 0 < min(ranks[1:]) and max(ranks) < M.shape[1]          # thresholded, not all kept
    nz = np.linalg.norm(r.E, axis=0) > 0
    assert 0 < nz.sum() < M.shape[1]                               # some columns shrunk to zero, some not


def test_forward_equals_the_alm_iterate():
    M, _ = _small_case()
    Z = adjoint.unrolled_forward(M, LAM, K, mu0=MU0)
    ref = lrr.lrr_alm(M, M, LAM, mu0=MU0, fixed_iters=K).Z
    assert np.array_equal(Z, ref)


def _grad_pin_holds(checkpoint=3):
    M, W = _small_case()
    loss = lambda Mx, lx: adjoint.weighted_loss(adjoint.unrolled_forward(Mx, lx, K, mu0=MU0), W)
    Z = adjoint.unrolled_forward(M, LAM, K, mu0=MU0)
    Mb, lb = adjoint.unrolled_grad(M, LAM, K, 2 * W * W * Z, mu0=MU0, checkpoint=checkpoint)
    h = 1e-6
    ok = True
    for i in range(M.shape[0]):
        for j in range(M.shape[1]):
            E = np.zeros_like(M)
            E[i, j] = h
            fd = (loss(M + E, LAM) - loss(M - E, LAM)) / (2 * h)
            ok &= abs(Mb[i, j] - fd) <= 1e-5 * max(1.0, abs(fd))
    fdl = (loss(M, LAM + h) - loss(M, LAM - h)) / (2 * h)
    ok &= abs(lb - fdl) <= 1e-5 * max(1.0, abs(fdl))
    return bool(ok)


def test_unrolled_gradient_matches_central_differences():
    """Every entry of dL/dM and dL/dlam for L = ||Z_K o W||_F^2 against central
    differences of the forward map (h = 1e-6), with checkpoints every 3
    iterations."""
    assert _grad_pin_holds(3)


def test_checkpoint_spacing_does_not_change_the_gradient():
    M, W = _small_case()
    Z = adjoint.unrolled_forward(M, LAM, K, mu0=MU0)
    g1 = adjoint.unrolled_grad(M, LAM, K, 2 * W * W * Z, mu0=MU0, checkpoint=1)
    g5 = adjoint.unrolled_grad(M, LAM, K, 2 * W * W * Z, mu0=MU0, checkpoint=5)
    assert np.allclose(g1[0], g5[0], rtol=1e-12, atol=1e-12) and g1[1] == pytest.approx(g5[1], rel=1e-12)


def test_planted_adjoint_mistakes_are_caught(monkeypatch):
    """Dropping the observation path (C = M), the left-complement term of the
    SVT derivative, or the threshold's dependence on lam each break the pin."""
    orig_svt, orig_shrink = adjoint.svt_adjoint, adjoint.shrink_adjoint

    def no_complement(A, tau, Jb):
        if A.shape[0] < A.shape[1]:
            return no_complement(A.T, tau, Jb.T).T
        U, s, Vt = np.linalg.svd(A, full_matrices=False)
        full = orig_svt(A, tau, Jb)
        fs = np.where(s > 0, np.maximum(s - tau, 0) / np.where(s > 0, s, 1), 0)
        return full - (Jb @ Vt.T - U @ (U.T @ Jb @ Vt.T)) * fs @ Vt
    monkeypatch.setattr(adjoint, "svt_adjoint", no_complement)
    # the square SVT input has no left complement: check the tall case directly
    rng = np.random.default_rng(1)
    A = rng.standard_normal((9, 5))
    Jb = rng.standard_normal((9, 5))
    dA = rng.standard_normal((9, 5))
    fd = _fd_dir(lambda X: np.sum(Jb * lrr.svt(X, 0.3)[0]), A, dA)
    assert abs(np.sum(adjoint.svt_adjoint(A, 0.3, Jb) * dA) - fd) > 1e-4
    monkeypatch.setattr(adjoint, "svt_adjoint", orig_svt)

    monkeypatch.setattr(adjoint, "shrink_adjoint", lambda X, th, Eb: (orig_shrink(X, th, Eb)[0], 0.0))
    assert not _grad_pin_holds(3)
    monkeypatch.setattr(adjoint, "shrink_adjoint", orig_shrink)

    monkeypatch.setattr(adjoint, "svt_adjoint", lambda A, tau, Jb: Jb * (np.linalg.norm(A) > 0))
    assert not _grad_pin_holds(3)
    monkeypatch.setattr(adjoint, "svt_adjoint", orig_svt)
    assert _grad_pin_holds(3)
