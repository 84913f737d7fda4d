"""Host-side parts of the Python binding (no GPU): layout helpers, option
marshalling and the workspace query with a drawn partition."""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def binding():
    from paper_1304_5583_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def test_column_major_and_leading_dim(binding):
    a = torch.arange(12.0).reshape(3, 4)               # row-major
    c = binding.column_major(a)
    assert c.stride(0) == 1 and torch.equal(c, a)
    assert binding.leading_dim(c) == 3
    b = torch.zeros(4, 5).t()                            # already column-major (5 x 4, ld 5)
    assert binding.column_major(b) is b and binding.leading_dim(b) == 5
    single = torch.zeros(7, 1)
    assert binding.leading_dim(binding.column_major(single)) == 7


def test_options_marshal_every_field(binding):
    o = binding.options(0.25, rho=1.2, mu0=1e-5, mu_max=1e9, eps=1e-7, max_iter=77, precision="mixed",
                        batched=False, jacobi_sweeps=5, rank_tol=1e-8, mixed_switch=0.3, profile=True)
    assert (o.lambda_, o.rho, o.mu0, o.mu_max, o.eps) == (0.25, 1.2, 1e-5, 1e9, 1e-7)
    assert (o.max_iter, o.precision, o.batched, o.jacobi_sweeps) == (77, binding.LRR_PREC_MIXED, 0, 5)
    assert (o.rank_tol, o.mixed_switch, o.profile) == (1e-8, 0.3, 1)
    with pytest.raises(KeyError):
        binding.options(0.1, precision="fp16")


def test_workspace_query_with_a_drawn_partition(binding):
    M = binding.column_major(torch.zeros(20, 60))        # only the shape and layout are read
    o = binding.options(0.1)
    perm, off = binding.partition(60, 3, 5)
    explicit = binding.workspace_bytes(M, perm, off, o)
    drawn = binding.workspace_bytes(M, None, None, o, t=3, seed=5)
    assert explicit > 0 and drawn == explicit
    with pytest.raises(ValueError):
        binding.workspace_bytes(M, None, None, o)         # t is needed without offsets
    assert binding.workspace_bytes(M, perm, np.array([0, 30, 30, 60]), o) == 0


def test_phase_transition_success_criterion_on_oracle_solutions():
    """The oracle constraints (Appendix) within 1e-4, evaluated on the float64
    oracle's LRR solutions of the paper's generator: a low outlier fraction
    recovers the row space and the outliers, a corrupted estimate fails."""
    import numpy as np
    from oracle import lrr as olrr
    from paper_1304_5583_gb300 import phase, synth
    d = synth.union_of_subspaces(1, 60, 3, 3, 30, 0.1, recipe="paper")
    r = olrr.lrr_alm(d.M, d.M, 0.5, eps=1e-8, max_iter=2000)
    V0 = phase.row_space_of_inliers(d)
    assert phase.oracle_constraints_hold(r.Z, r.E, V0, d.outlier)
    Zbad = r.Z.copy()
    Zbad[:, 0] += 1e-3 * np.random.default_rng(0).standard_normal(Zbad.shape[0])
    assert not phase.oracle_constraints_hold(Zbad, r.E, V0, d.outlier)
    Ebad = r.E.copy()
    Ebad[:, np.flatnonzero(~d.outlier)[0]] += 1e-3
    assert not phase.oracle_constraints_hold(r.Z, Ebad, V0, d.outlier)
