"""Writes the float64 oracle's segmentation labels of the full-size DFC-LRR
workloads to tests/golden/labels_<workload>.json.  Calls only oracle/ and the
seeded input generators: the oracle runs Algorithm 1 to convergence on the
float32-rounded input (the matrix the CUDA path sees), then the Section 4.1.2
post-processing (oracle/segment.py) labels the combined estimate.

usage: python tests/golden/make_oracle_labels.py [workload ...] [--workers N]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=["dfc_500x5000", "dfc_faces_2016x2432"])
    ap.add_argument("--workers", type=int, default=4)
    args = ap.parse_args()
    cores = os.cpu_count() or 1
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = str(max(1, cores // max(1, args.workers)))
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import lrr, segment
    from paper_1304_5583_gb300 import synth
    for name in args.workloads:
        w = synth.workload(name)
        M = w.M.astype(np.float32).astype(np.float64)
        t0 = time.time()
        res = lrr.dfc_lrr(M, w.perm, w.offsets, w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=w.eps,
                          max_iter=w.max_iter, workers=args.workers)
        t1 = time.time()
        # the C step's output lies in span(Q1): its singular vectors come from
        # the k1 x n matrix Q1^T Z (an SVD of the dense 20000 x 20000 Z
        # crashed inside LAPACK)
        basis = lrr.orth_basis(res.blocks[0].J_U) if w.t > 1 else None
        lab = segment.segment(res.Z, w.data.k, seed=0, basis=basis)
        t2 = time.time()
        out = {"workload": name, "recipe": "synth.workload(%r, seed=0), float32-rounded M" % name,
               "oracle": "oracle.lrr.dfc_lrr to convergence, then oracle.segment.segment(Z, k, seed=0)",
               "k": int(w.data.k), "k1": int(res.k1), "iters": [int(x) for x in res.iters],
               "matched_accuracy_vs_truth": segment.matched_accuracy(lab, w.data.labels),
               "labels": [int(x) for x in lab]}
        path = os.path.join(HERE, f"labels_{name}.json")
        with open(path, "w") as f:
            json.dump(out, f)
        print(f"{name}: solve {t1 - t0:.0f} s, segment {t2 - t1:.0f} s, k1 {res.k1}, "
              f"accuracy {out['matched_accuracy_vs_truth']:.4f} -> {path}", flush=True)


if __name__ == "__main__":
    main()
