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


def _run(lib, w, precision="f32", batched=True, entry="dfc", eps=None, max_iter=None, **kw):
    from paper_1304_5583_gb300 import binding
    dt = np.float64 if precision == "f64" else np.float32
    Md = _to_dev(w.M, dt)
    o = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=eps or w.eps,
                        max_iter=max_iter or w.max_iter, precision=precision, batched=batched, **kw)
    if entry == "lrr":
        res = binding.lrr_solve(Md, w.perm, o, raise_on_error=False)
    else:
        res = binding.dfc_lrr_solve(Md, w.perm, w.offsets, o, raise_on_error=False)
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
    if batched:
        # the free-running oracle stops within two iterations of the GPU
        # (both schedules take the same iterations; checked once)
        free = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, max_iter=w.max_iter)
        assert np.all(np.abs(res.iters - free.iters) <= 2)


def test_partition_drawn_by_the_library_from_a_seed(lib):
    # D step inside the library (perm and offsets NULL) == the oracle's draw
    # from the same seed passed in explicitly; the result is then checked
    # against the oracle like any other partition
    from oracle import partition as opart
    from paper_1304_5583_gb300 import binding
    w = synth.workload("small_dfc_60x240")
    Md = _to_dev(w.M, np.float32)
    o = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=w.eps, max_iter=w.max_iter,
                        precision="f32")
    a = binding.dfc_lrr_solve(Md, None, None, o, t=3, seed=11)
    perm, off = opart.partition(w.M.shape[1], 3, 11)
    b = binding.dfc_lrr_solve(Md, perm, off, o)
    assert a.status == 0 and b.status == 0
    assert np.all(np.abs(a.iters - b.iters) <= 1)
    assert _rel(a.Z.cpu().numpy(), b.Z.cpu().numpy().astype(np.float64)) < 1e-6
    M = w.M.astype(np.float32).astype(np.float64)
    ref = olrr.dfc_lrr(M, perm, off, w.lam, eps=w.eps, max_iter=w.max_iter, fixed_iters=list(a.iters))
    assert _rel(a.Z.cpu().numpy(), ref.Z) < 1e-5


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


def test_small_dfc_mixed_precision_matches_oracle(lib):
    w = synth.workload("small_dfc_60x240")
    res, M = _run(lib, w, "mixed")
    assert res.status == 0
    ref = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, max_iter=w.max_iter, fixed_iters=list(res.iters))
    assert _rel(res.Z.cpu().numpy(), ref.Z) < 1e-5
    assert _rel(res.S.cpu().numpy(), ref.S) < 1e-5


@pytest.mark.parametrize("precision", ["f32", "mixed", "f64"])
def test_tiny_and_ragged_shapes(lib, precision):
    """m not a multiple of 8, blocks of one and two columns, t close to n."""
    d = synth.union_of_subspaces(21, 13, 2, 2, 9, 0.1)
    M = d.M
    n = M.shape[1]
    perm = np.random.default_rng(3).permutation(n)
    offsets = np.array([0, 1, 3, 8, n], dtype=np.int64)
    w = synth.Workload("ragged", d, perm, offsets, lam=0.3, eps=1e-6 if precision != "f64" else 1e-9)
    res, Mr = _run(lib, w, precision)
    assert res.status == 0
    ref = olrr.dfc_lrr(Mr, perm, offsets, w.lam, eps=w.eps, fixed_iters=list(res.iters))
    tol = 1e-9 if precision == "f64" else 1e-5
    assert _rel(res.Z.cpu().numpy(), ref.Z) < tol
    # S is mostly zero columns, so its relative error is the least forgiving;
    # in the mixed form the bf16 warm-up phase leaves ~1e-5 there
    assert _rel(res.S.cpu().numpy(), ref.S) < (1e-4 if precision == "mixed" else tol)


def test_segmentation_labels_identical_plain_lrr(lib):
    """Segmentation (Section 4.1.2 post-processing) of the GPU and oracle
    estimates gives the same partition on the 100 x 500 problem."""
    from oracle import segment
    w = synth.workload("plain_lrr_100x500")
    res, M = _run(lib, w, "f64", entry="lrr")
    ref = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps)
    a = segment.segment(res.Z.cpu().numpy(), w.data.k, seed=0)
    b = segment.segment(ref.Z, w.data.k, seed=0)
    assert segment.same_partition(a, b)


def test_zero_matrix_reports_rank_error(lib):
    from paper_1304_5583_gb300 import binding
    w = synth.workload("tiny_20x30")
    res = binding.dfc_lrr_solve(_to_dev(np.zeros_like(w.M), np.float32), w.perm, w.offsets, binding.options(0.1),
                                raise_on_error=False)
    assert res.status == -5


def test_max_iter_exhaustion_reports_not_converged_with_valid_outputs(lib):
    """A solve cut off at max_iter returns LRR_NOT_CONVERGED (+1) and still
    writes the combined estimate: it equals the oracle's Algorithm 1 output
    after the same number of iterations per block."""
    w = synth.workload("small_dfc_60x240")
    # 130 of the 166 iterations the blocks need: block 1's SVT already keeps
    # directions (k1 = 10), so the combined estimate is not zero
    res, M = _run(lib, w, "f32", max_iter=130)
    assert res.status == 1
    assert np.all(res.iters == 130)
    ref = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, fixed_iters=130)
    assert res.k1 == ref.k1 > 0
    assert _rel(res.Z.cpu().numpy(), ref.Z) < 1e-5
    assert _rel(res.S.cpu().numpy(), ref.S) < 1e-5
    # the primal residual is reported exactly, ||Z - J||_inf as an upper bound
    assert np.allclose(res.resid[:, 0], ref.resid[:, 0], rtol=1e-4)
    assert np.all(res.resid[:, 1] >= ref.resid[:, 1] * (1 - 1e-4))


def test_mixed_precision_before_refinement(lib):
    """The mixed form's bf16 phase on its own: plain LRR (t = 1, no C step)
    stopped at the last iteration before its SVT input first exceeds half the
    threshold (the iteration after which the float32 refinement takes over)
    matches the float64 oracle at the same iteration count to 1e-3."""
    w = synth.workload("diff_200x1000")
    M = w.M.astype(np.float32).astype(np.float64)
    tr = olrr.lrr_alm(M[:, w.perm], M, w.lam, eps=w.eps, max_iter=w.max_iter, keep_trace=True).trace
    # trace row k-1 is iteration k: (mu, r1, r2, rank, ||Z + Y2/mu||_F)
    s = next(k for k, row in enumerate(tr, start=1) if row[4] > 0.5 / row[0])
    last_bf16 = s - 1
    assert last_bf16 >= 5
    res, _ = _run(lib, w, "mixed", entry="lrr", max_iter=last_bf16)
    assert res.status == 1 and res.iters[0] == last_bf16
    ref = olrr.lrr_alm(M[:, w.perm], M, w.lam, fixed_iters=last_bf16)
    Zg = res.Z.cpu().numpy()[:, w.perm].astype(np.float64)
    err = _rel(Zg, ref.Z)
    print(f"mixed before refinement: iteration {last_bf16}, rel err {err:.3e}")
    assert err < 1e-3


@pytest.mark.parametrize("name,entry", [("small_dfc_60x240", "dfc"), ("tiny_20x30", "lrr")])
def test_factored_output_reproduces_the_dense_estimate(lib, name, entry):
    """Section 2.2's factored form at the boundary: Z = F[:, :k] G[:k] with F
    orthonormal equals the dense combined estimate, and the dense estimate
    still matches the oracle."""
    import torch
    from paper_1304_5583_gb300 import binding
    w = synth.workload(name)
    dt = np.float32
    Md = _to_dev(w.M, dt)
    # float32 stops at eps 1e-6 (the 20 x 30 workload's 1e-8 is a float64 target)
    eps = max(w.eps, 1e-6)
    o = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=eps, max_iter=w.max_iter,
                        precision="f32")
    if entry == "lrr":
        res = binding.lrr_solve(Md, w.perm, o, want_factors=True)
    else:
        res = binding.dfc_lrr_solve(Md, w.perm, w.offsets, o, want_factors=True)
    assert res.status == 0
    k = res.factor_k
    assert 0 < k <= res.F.shape[1]
    assert k == (res.k1 if w.t > 1 else res.rank_M)
    F = res.F[:, :k].double()
    G = res.G[:k].double()
    assert torch.allclose(F.T @ F, torch.eye(k, dtype=torch.float64, device=F.device), atol=1e-5)
    Z = res.Z.double()
    assert float(torch.linalg.norm(F @ G - Z) / torch.linalg.norm(Z)) < 1e-5
    M = w.M.astype(dt).astype(np.float64)
    ref = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, fixed_iters=list(res.iters))
    assert _rel(res.Z.cpu().numpy(), ref.Z) < 1e-5


def test_autotuned_launch_shape_gives_bitwise_identical_results(lib):
    """The autotuner only changes how the pivots of a Jacobi round are spread
    over the CTAs of a block's cluster; every pivot does the same arithmetic,
    so the solve is bitwise unchanged."""
    w = synth.workload("small_dfc_60x240")
    a, _ = _run(lib, w, "f32")
    b, _ = _run(lib, w, "f32", autotune=True)
    c, _ = _run(lib, w, "f32", autotune=True)      # cached choice
    assert a.status == b.status == c.status == 0
    assert np.array_equal(a.iters, b.iters) and np.array_equal(a.Z.cpu().numpy(), b.Z.cpu().numpy())
    assert np.array_equal(b.Z.cpu().numpy(), c.Z.cpu().numpy())


@pytest.mark.parametrize("precision", ["f32", "mixed"])
def test_tensor_core_products_match_oracle(lib, precision):
    """The float32 products on the tensor cores in split TF32 (tc_products)
    instead of the CUDA cores: same parity with the oracle."""
    w = synth.workload("small_dfc_60x240")
    res, M = _run(lib, w, precision, tc_products=True)
    assert res.status == 0
    ref = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, max_iter=w.max_iter, fixed_iters=list(res.iters))
    assert _rel(res.Z.cpu().numpy(), ref.Z) < 1e-5


# ranks at clear gaps of the combined block spectrum (0.941 | 0.858 and
# 0.62 | 2e-6 on this workload).  The truncated subspace moves by about the
# blocks' float32 error over the relative gap at the cut: the default k1 = 12
# falls between 1.00187 and 1.00169, and rank 24 (0.9996 | 0.9931, a 0.6 % gap)
# measured 2.2e-5, so neither is determined to 1e-5 in float32
@pytest.mark.parametrize("rank", [30, 36])
def test_footnote_variant_matches_oracle(lib, rank):
    """Dictionary C_i per block (the footnote to eq. (2)), blocks solved as
    independent problems on concurrent streams, C step = truncated SVD of
    diag(Z_1..Z_t): against the oracle at the GPU's iteration counts."""
    from paper_1304_5583_gb300 import binding
    w = synth.workload("small_dfc_60x240")
    Md = _to_dev(w.M, np.float32)
    o = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=w.eps, max_iter=w.max_iter,
                        precision="f32")
    res = binding.dfc_lrr_solve_local(Md, w.perm, w.offsets, o, rank=rank, streams=3)
    assert res.status == 0
    M = w.M.astype(np.float32).astype(np.float64)
    ref = olrr.dfc_lrr_local(M, w.perm, w.offsets, w.lam, eps=w.eps, fixed_iters=list(res.iters),
                             k=rank if rank > 0 else None)
    assert res.k1 == ref.k1
    assert _rel(res.Z.cpu().numpy(), ref.Z) < 1e-5
    assert _rel(res.S.cpu().numpy(), ref.S) < 1e-5


def test_batch_of_independent_problems_matches_one_by_one(lib):
    """lrr_solve_batch: problems of different sizes on concurrent streams give
    bitwise the results of solving them one at a time."""
    from paper_1304_5583_gb300 import binding
    Ms = []
    for seed, (m, k, n_s) in enumerate([(40, 3, 20), (60, 4, 15), (30, 2, 25), (50, 3, 18)]):
        d = synth.union_of_subspaces(100 + seed, m, k, 3, n_s, 0.1)
        Ms.append(_to_dev(d.M, np.float32))
    o = binding.options(0.2, eps=1e-6, precision="f32")
    outs, st = binding.solve_batch(Ms, o, streams=4)
    assert np.all(st == 0)
    for M, (Z, S, it) in zip(Ms, outs):
        n = M.shape[1]
        one = binding.lrr_solve(M, np.arange(n), o)
        assert np.array_equal(one.iters, it)
        assert np.array_equal(one.Z.cpu().numpy(), Z.cpu().numpy())
