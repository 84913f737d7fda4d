"""Parity of the CUDA path (through the C ABI) with the float64 oracle."""
import numpy as np
import pytest

from oracle import lrr as olrr
from paper_1304_5583_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _to_dev(M, dtype):
    import torch
    return torch.from_numpy(np.asfortranarray(M.astype(dtype))).cuda()


def _run(lib, w, precision="f32", batched=True, entry="dfc", eps=None, **kw):
    from paper_1304_5583_gb300 import binding
    dt = np.float64 if precision == "f64" else np.float32
    Md = _to_dev(w.M, dt)
    o = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=eps or w.eps, max_iter=w.max_iter,
                        precision=precision, batched=batched, **kw)
    if entry == "lrr":
        res = binding.lrr_solve(Md, w.perm, o)
    else:
        res = binding.dfc_lrr_solve(Md, w.perm, w.offsets, o)
    return res, w.M.astype(dt).astype(np.float64)


def test_tiny_lrr_float64_matches_oracle(lib):
    w = synth.workload("tiny_20x30")
    res, M = _run(lib, w, "f64", entry="lrr")
    assert res.status == 0
    ref = olrr.lrr_alm(M[:, w.perm], M, w.lam, eps=w.eps, max_iter=w.max_iter)
    assert res.iters[0] == ref.iters
    Zg = res.Z.cpu().numpy()[:, w.perm]       # back to the observation order of the oracle run
    assert _rel(Zg, ref.Z) < 1e-9
    assert _rel(res.S.cpu().numpy()[:, w.perm], ref.E) < 1e-9


def test_plain_lrr_100x500_float64_matches_oracle(lib):
    w = synth.workload("plain_lrr_100x500")
    res, M = _run(lib, w, "f64", entry="lrr")
    assert res.status == 0
    ref = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, max_iter=w.max_iter)
    assert res.iters[0] == ref.iters[0]
    assert _rel(res.Z.cpu().numpy(), ref.Z) < 1e-8
    assert _rel(res.S.cpu().numpy(), ref.S) < 1e-8
    assert res.resid[0].max() < w.eps


@pytest.mark.parametrize("batched", [True, False])
def test_small_dfc_float32_matches_oracle(lib, batched):
    w = synth.workload("small_dfc_60x240")
    res, M = _run(lib, w, "f32", batched=batched)
    assert res.status == 0
    ref = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, max_iter=w.max_iter, fixed_iters=list(res.iters))
    assert _rel(res.Z.cpu().numpy(), ref.Z) < 1e-5
    assert _rel(res.S.cpu().numpy(), ref.S) < 1e-5
    assert res.k1 == ref.k1
    free = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, max_iter=w.max_iter)
    assert np.all(np.abs(res.iters - free.iters) <= 2)


def test_batched_and_sequential_blocks_agree_bitwise(lib):
    w = synth.workload("small_dfc_60x240")
    a, _ = _run(lib, w, "f32", batched=True)
    b, _ = _run(lib, w, "f32", batched=False)
    assert np.array_equal(a.iters, b.iters)
    assert np.array_equal(a.Z.cpu().numpy(), b.Z.cpu().numpy())
    assert np.array_equal(a.S.cpu().numpy(), b.S.cpu().numpy())


def test_nonfinite_input_is_rejected(lib):
    from paper_1304_5583_gb300 import binding
    w = synth.workload("tiny_20x30")
    M = w.M.copy()
    M[3, 4] = np.nan
    o = binding.options(w.lam)
    res = binding.dfc_lrr_solve(_to_dev(M, np.float32), w.perm, w.offsets, o, raise_on_error=False)
    assert res.status == -2


def test_invalid_partition_is_rejected(lib):
    from paper_1304_5583_gb300 import binding
    w = synth.workload("tiny_20x30")
    o = binding.options(w.lam)
    bad = w.perm.copy()
    bad[0] = bad[1]
    res = binding.dfc_lrr_solve(_to_dev(w.M, np.float32), bad, w.offsets, o, raise_on_error=False)
    assert res.status == -1
