"""Writes tests/golden/adjoint_fd_diff_200x1000.json: float64 central
differences (h = 1e-6) of L = ||Z_K o W||_F^2 for the differentiable
configuration (plain LRR, t = 1, on the 200 x 1000 union of 5 rank-8
subspaces with 5 % outlier columns; K = 30 unrolled ALM iterations; lam = 0.1;
mu0 = 0.1, rho = 1.1; W ~ N(0, 1) from seed 5) at 50 seeded entries of M and
in lam, next to the oracle's reverse-mode gradient at the same points.  Calls
only oracle/ and the seeded input generators.

usage: python tests/golden/make_adjoint_fd.py [--workers N]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CFG = dict(workload="diff_200x1000", K=30, lam=0.1, mu0=0.1, rho=1.1, mu_max=1e10, checkpoint=5, w_seed=5,
           entry_seed=2024, entries=50, h=1e-6)


def _loss(args):
    dM, dl = args
    import numpy as np
    from oracle import adjoint
    from paper_1304_5583_gb300 import synth
    w = synth.workload(CFG["workload"])
    M = w.M.astype(np.float32).astype(np.float64)
    if dM is not None:
        i, j, h = dM
        M = M.copy()
        M[i, j] += h
    n = M.shape[1]
    W = np.random.default_rng(CFG["w_seed"]).standard_normal((n, n))
    Z = adjoint.unrolled_forward(M, CFG["lam"] + dl, CFG["K"], mu0=CFG["mu0"], rho=CFG["rho"], mu_max=CFG["mu_max"])
    return adjoint.weighted_loss(Z, W)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=4)
    a = ap.parse_args()
    cores = os.cpu_count() or 1
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = str(max(1, cores // max(1, a.workers)))
    sys.path.insert(0, ROOT)
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import numpy as np
    from oracle import adjoint
    from paper_1304_5583_gb300 import synth
    w = synth.workload(CFG["workload"])
    M = w.M.astype(np.float32).astype(np.float64)
    m, n = M.shape
    rng = np.random.default_rng(CFG["entry_seed"])
    flat = rng.choice(m * n, CFG["entries"], replace=False)
    ent = [(int(f % m), int(f // m)) for f in flat]
    h = CFG["h"]
    jobs = []
    for i, j in ent:
        jobs += [((i, j, h), 0.0), ((i, j, -h), 0.0)]
    jobs += [(None, h), (None, -h)]
    t0 = time.time()
    with ProcessPoolExecutor(max_workers=a.workers, mp_context=mp.get_context("spawn")) as ex:
        vals = list(ex.map(_loss, jobs))
    t1 = time.time()
    fd_M = [(vals[2 * k] - vals[2 * k + 1]) / (2 * h) for k in range(len(ent))]
    fd_l = (vals[-2] - vals[-1]) / (2 * h)
    W = np.random.default_rng(CFG["w_seed"]).standard_normal((n, n))
    Z = adjoint.unrolled_forward(M, CFG["lam"], CFG["K"], mu0=CFG["mu0"], rho=CFG["rho"], mu_max=CFG["mu_max"])
    Mb, lb = adjoint.unrolled_grad(M, CFG["lam"], CFG["K"], 2 * W * W * Z, mu0=CFG["mu0"], rho=CFG["rho"],
                                   mu_max=CFG["mu_max"], checkpoint=CFG["checkpoint"])
    t2 = time.time()
    out = dict(CFG, M_dtype="float32-rounded", loss=adjoint.weighted_loss(Z, W), entries_ij=ent, fd_dM=fd_M,
               fd_dlam=fd_l, oracle_dM=[float(Mb[i, j]) for i, j in ent], oracle_dlam=float(lb))
    path = os.path.join(HERE, "adjoint_fd_diff_200x1000.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    err = max(abs(a_ - b_) / max(1.0, abs(b_)) for a_, b_ in zip(out["oracle_dM"], fd_M))
    print(f"finite differences {t1 - t0:.0f} s, reverse mode {t2 - t1:.0f} s; max |oracle - fd| / max(1, |fd|) "
          f"over M entries {err:.2e}, lam: {lb:.6e} vs {fd_l:.6e} -> {path}", flush=True)


if __name__ == "__main__":
    main()
