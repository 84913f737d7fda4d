"""Singular-value thresholding (lrr_svt, the J-step kernels) against the
oracle's closed-form SVT on controlled spectra."""
import numpy as np
import pytest

from oracle import lrr as olrr

pytestmark = pytest.mark.gpu


def _mk(rng, rows, cols, svals):
    k = len(svals)
    U = np.linalg.qr(rng.standard_normal((rows, k)))[0]
    V = np.linalg.qr(rng.standard_normal((cols, k)))[0]
    return (U * svals) @ V.T


CASES = {
    "graded_tall": (300, 150, lambda r: np.geomspace(1, 1e-4, 150), 1e-2),
    "graded_wide": (150, 400, lambda r: np.geomspace(1, 1e-4, 150), 1e-2),
    "clustered": (1000, 500, lambda r: np.r_[1 + 1e-4 * r.standard_normal(200), 1e-3 * r.random(300)], 5e-4),
    "low_rank_plus_noise": (1000, 500, lambda r: np.r_[np.geomspace(3, 0.1, 400), 1e-6 * np.ones(100)], 1e-4),
    "ragged_small": (37, 21, lambda r: np.geomspace(2, 0.01, 21), 0.05),
    "single_column": (50, 1, lambda r: np.array([0.7]), 0.2),
    "all_below_threshold": (80, 40, lambda r: np.geomspace(0.09, 0.001, 40), 0.1),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_svt_matches_closed_form(lib, name, dtype):
    import torch
    from paper_1304_5583_gb300 import binding
    rows, cols, spec, tau = CASES[name]
    rng = np.random.default_rng(abs(hash(name)) % 2**31)
    A = _mk(rng, rows, cols, spec(rng))
    dt = np.float32 if dtype == "f32" else np.float64
    A = A.astype(dt)
    Jref, U, s, Vt = olrr.svt(A.astype(np.float64), tau)
    J, rank = binding.svt(torch.from_numpy(np.asfortranarray(A)).cuda(), tau)
    J = J.cpu().numpy().astype(np.float64)
    assert rank == U.shape[1]
    nrm = max(np.linalg.norm(Jref), 1e-300)
    tol = 5e-6 if dtype == "f32" else 1e-12
    if U.shape[1] == 0:
        assert np.abs(J).max() == 0.0
    else:
        assert np.linalg.norm(J - Jref) / nrm < tol
