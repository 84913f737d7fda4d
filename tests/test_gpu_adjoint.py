"""The differentiable unrolled LRR (lrr_unrolled_forward / _backward and its
torch.autograd.Function) against the float64 oracle (oracle/adjoint.py, itself
pinned to central differences) and against stored float64 central
differences of the 200 x 1000, K = 30 configuration."""
import json
import os

import numpy as np
import pytest

from oracle import adjoint
from paper_1304_5583_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _small():
    d = synth.union_of_subspaces(4, 10, 2, 2, 8, 0.15)
    W = np.random.default_rng(9).standard_normal((16, 16))
    return d.M, W, dict(lam=0.6, K=8, mu0=1.0)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision,tol_z,tol_g", [("f64", 1e-10, 1e-8), ("f32", 1e-5, 1e-3)])
def test_small_unrolled_forward_and_gradient_match_oracle(lib, precision, tol_z, tol_g):
    import torch
    from paper_1304_5583_gb300 import binding
    M, W, c = _small()
    dt = torch.float64 if precision == "f64" else torch.float32
    Md = torch.from_numpy(np.asfortranarray(M)).to(dt).cuda()
    Mh = Md.double().cpu().numpy()
    o = binding.unrolled_options(c["lam"], c["K"], mu0=c["mu0"], checkpoint=3, precision=precision)
    Z = binding.unrolled_forward(Md, o).double().cpu().numpy()
    Zr = adjoint.unrolled_forward(Mh, c["lam"], c["K"], mu0=c["mu0"])
    assert _rel(Z, Zr) < tol_z
    Zbar = 2 * W * W * Zr
    Mb, lb = binding.unrolled_backward(Md, o, torch.from_numpy(Zbar).to(dt).cuda())
    Mr, lr = adjoint.unrolled_grad(Mh, c["lam"], c["K"], Zbar, mu0=c["mu0"], checkpoint=3)
    print(f"{precision}: Z {_rel(Z, Zr):.2e}, dL/dM {_rel(Mb.double().cpu().numpy(), Mr):.2e}, "
          f"dL/dlam {abs(lb - lr) / abs(lr):.2e}")
    assert _rel(Mb.double().cpu().numpy(), Mr) < tol_g
    assert abs(lb - lr) <= tol_g * abs(lr)


def test_autograd_function_gives_the_library_gradient(lib):
    import torch
    from paper_1304_5583_gb300 import binding
    M, W, c = _small()
    Md = torch.from_numpy(np.asfortranarray(M)).double().cuda().requires_grad_(True)
    lam = torch.tensor(c["lam"], dtype=torch.float64, device="cuda", requires_grad=True)
    Wd = torch.from_numpy(W).cuda()
    Z = binding.unrolled_lrr(Md, lam, c["K"], mu0=c["mu0"], checkpoint=3)
    loss = ((Z * Wd) ** 2).sum()
    loss.backward()
    Mr, lr = adjoint.unrolled_grad(M, c["lam"], c["K"], 2 * W * W * Z.detach().cpu().numpy(), mu0=c["mu0"],
                                   checkpoint=3)
    assert _rel(Md.grad.cpu().numpy(), Mr) < 1e-8
    assert float(lam.grad) == pytest.approx(lr, rel=1e-8)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_config_200x1000_gradient_against_central_differences(lib, precision):
    """K = 30 unrolled iterations on the 200 x 1000 workload, checkpoints every
    5: dL/dM at 50 seeded entries and dL/dlam against float64 central
    differences (h = 1e-6) of the oracle's forward map."""
    import torch
    from paper_1304_5583_gb300 import binding
    with open(os.path.join(GOLDEN, "adjoint_fd_diff_200x1000.json")) as f:
        g = json.load(f)
    w = synth.workload(g["workload"])
    dt = torch.float64 if precision == "f64" else torch.float32
    Md = torch.from_numpy(np.asfortranarray(w.M.astype(np.float32))).to(dt).cuda()
    n = w.M.shape[1]
    W = torch.from_numpy(np.random.default_rng(g["w_seed"]).standard_normal((n, n))).to(dt).cuda()
    o = binding.unrolled_options(g["lam"], g["K"], mu0=g["mu0"], rho=g["rho"], mu_max=g["mu_max"],
                                 checkpoint=g["checkpoint"], precision=precision)
    Z = binding.unrolled_forward(Md, o)
    Mb, lb = binding.unrolled_backward(Md, o, 2 * W * W * Z)
    ij = np.array(g["entries_ij"])
    got = Mb.double().cpu().numpy()[ij[:, 0], ij[:, 1]]
    fd = np.array(g["fd_dM"])
    err = float(np.linalg.norm(got - fd) / np.linalg.norm(fd))
    errl = abs(lb - g["fd_dlam"]) / abs(g["fd_dlam"])
    ora = np.array(g["oracle_dM"])
    erro = float(np.linalg.norm(got - ora) / np.linalg.norm(ora))
    print(f"{precision}: 50 entries of dL/dM vs central differences {err:.2e}, vs the oracle's reverse mode "
          f"{erro:.2e}; dL/dlam {errl:.2e}")
    # The central differences carry cancellation error: |L| eps / h ~ 1e-8 per
    # entry against entries of 1e-4 .. 4e-3, so about 2e-5 relative over the 50
    # entries (the oracle's own reverse mode is 2.1e-5 from them).  float64 is
    # therefore held to the differences at 1e-4 and to the oracle's reverse mode
    # (the same 30 iterations in float64) at 1e-8.  float32: the rounding of
    # the forward iterates passes through the SVT derivative's 1/(s_i - s_j)
    # factors 30 times; held at 1e-2.
    if precision == "f64":
        assert err < 1e-4 and errl < 1e-4
        assert erro < 1e-8
        assert abs(lb - g["oracle_dlam"]) <= 1e-8 * abs(g["oracle_dlam"])
    else:
        assert err < 1e-2 and errl < 1e-2
