"""All-block parity of the C step on the 500x5000 workload, sampled: block 2's
columns of the GPU's Z-hat against Q1 Q1^T Z_2 from the oracle (blocks 1 and 2
at the GPU's iteration counts).  The 500x5000 workload has a clean gap at k1
(k1 = 100, the rank of the union of subspaces), so these columns are as well
conditioned as block 1's.  Long (two oracle block solves): run with -m gpu_long."""
import numpy as np
import pytest

from oracle import lrr as olrr
from paper_1304_5583_gb300 import synth

pytestmark = pytest.mark.gpu_long


def test_other_blocks_match_the_oracle(lib):
    import torch
    from paper_1304_5583_gb300 import binding
    w = synth.workload("dfc_500x5000")
    Md = torch.from_numpy(np.asfortranarray(w.M.astype(np.float32))).cuda()
    o = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=w.eps, max_iter=w.max_iter,
                        precision="f32")
    res = binding.dfc_lrr_solve(Md, w.perm, w.offsets, o)
    assert res.status == 0
    M = w.M.astype(np.float32).astype(np.float64)
    fixed = [int(res.iters[0]), int(res.iters[1])] + [0] * (w.t - 2)
    fx = olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, eps=w.eps, blocks_only=[0, 1], fixed_iters=fixed)
    Q = olrr.orth_basis(fx.blocks[0].J_U)
    Zp = Q @ (Q.T @ fx.blocks[1].Z)
    cols = w.perm[w.offsets[1]:w.offsets[2]]
    Zg = res.Z.cpu().numpy()[:, cols].astype(np.float64)
    assert res.k1 == Q.shape[1]
    assert np.linalg.norm(Zg - Zp) / np.linalg.norm(Zp) < 1e-5
