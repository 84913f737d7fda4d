"""Helpers shared by the GPU parity tests: oracle runs (cached per session,
keyed by the inputs they depend on) and the C-ABI calls on a workload."""
from __future__ import annotations

import functools

import numpy as np

from oracle import lrr as olrr
from paper_1304_5583_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(M, dtype):
    import torch
    return torch.from_numpy(np.asfortranarray(M.astype(dtype))).cuda()


def run(w, precision="f32", batched=True, entry="dfc", eps=None, max_iter=None, raise_on_error=True, **kw):
    """Solve workload w through the C ABI; returns (result, the float64 copy
    of the matrix the GPU saw)."""
    from paper_1304_5583_gb300 import binding
    dt = np.float64 if precision == "f64" else np.float32
    Md = to_dev(w.M, dt)
    o = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=eps or w.eps,
                        max_iter=max_iter or w.max_iter, precision=precision, batched=batched, **kw)
    if entry == "lrr":
        res = binding.lrr_solve(Md, w.perm, o, raise_on_error=raise_on_error)
    else:
        res = binding.dfc_lrr_solve(Md, w.perm, w.offsets, o, raise_on_error=raise_on_error)
    return res, w.M.astype(dt).astype(np.float64)


@functools.lru_cache(maxsize=4)
def oracle_blocks(name: str, precision: str, fixed: tuple):
    """The float64 oracle's F step on the listed blocks of workload `name` at
    fixed per-block iteration counts (0 = block not run), on the matrix the
    GPU saw in `precision`."""
    w = synth.workload(name)
    dt = np.float64 if precision == "f64" else np.float32
    M = w.M.astype(dt).astype(np.float64)
    which = [i for i, k in enumerate(fixed) if k > 0]
    return olrr.dfc_lrr(M, w.perm, w.offsets, w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=w.eps,
                        max_iter=w.max_iter, blocks_only=which, fixed_iters=list(fixed))


def block_projected(name, precision, iters, blocks):
    """Columns of the combined estimate for each listed block, computed by the
    oracle from block 1 and that block alone (Algorithm 1's C step restricted
    to those columns: Q1 Q1^T Z_j, Q1 an orthonormal basis of col(Z_1)), at the
    GPU's iteration counts.  Returns ({block: n x l_j array}, k1)."""
    t = len(iters)
    fixed = [0] * t
    for b in set([0] + list(blocks)):
        fixed[b] = int(iters[b])
    fx = oracle_blocks(name, precision, tuple(fixed))
    Q = olrr.orth_basis(fx.blocks[0].J_U)
    return {b: Q @ (Q.T @ fx.blocks[b].Z) for b in blocks}, Q.shape[1]
