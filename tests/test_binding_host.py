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
