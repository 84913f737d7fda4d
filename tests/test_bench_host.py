"""Host-side arithmetic of bench.py: the algorithmic work counts behind the
roofline figures, the CPU-baseline extrapolation and the config object both
arms print (no GPU)."""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1304_5583_gb300 import synth  # noqa: E402


def _args(**kw):
    a = dict(workload="small_dfc_60x240", precision="mixed", sequential=False, no_autotune=False)
    a.update(kw)
    return argparse.Namespace(**a)


def test_jacobi_work_counts_per_block_sweep():
    """4 p^3 per block-sweep (method) and 8 L p^2 + 4 p^3 (as executed), with
    p = min(r, l) and L the other side, summed over the blocks' sweeps."""
    w = synth.workload("small_dfc_60x240")
    r = 24
    l = np.diff(w.offsets)
    sweeps = np.arange(1, w.t + 1)
    method, impl = bench.jacobi_work(w, r, sweeps)
    p = np.minimum(l, r)
    L = np.maximum(l, r)
    assert method == float(np.sum(sweeps * 4 * p ** 3))
    assert impl == float(np.sum(sweeps * (8 * L * p * p + 4 * p ** 3)))


def test_algorithmic_work_of_the_products_and_updates():
    w = synth.workload("small_dfc_60x240")
    m = w.M.shape[0]
    r, it = 24, np.full(w.t, 10)
    l = np.diff(w.offsets)
    work = bench.algorithmic_work(w, r, it)
    assert work["zgemm"]["flops"] == float(np.sum(it * 2 * r * m * l))
    assert work["eupdate"]["bytes"] == float(np.sum(it * 4 * m * l * 8))
    assert work["zupdate"]["bytes"] == float(np.sum(it * 4 * r * l * 7))


def test_extrapolation_scales_with_block_width():
    w = synth.workload("small_dfc_60x240")
    l = np.diff(w.offsets).astype(float)
    iters = np.array([100, 200, 300])
    v = bench.extrapolate(w, 2.0, 5.0, iters)
    assert abs(v - (5.0 + float(np.sum(iters * 2.0 * l / l[0])))) < 1e-9


def test_both_arms_print_the_same_config():
    w = synth.workload("small_dfc_60x240")
    a = bench.workload_config(_args(), w, 1)
    b = bench.workload_config(_args(), w, 1)
    assert a == b
    assert {"workload", "m", "n", "t", "lambda", "eps", "precision"} <= set(a)
    assert a["m"] == 60 and a["n"] == 240 and a["t"] == 3
    assert bench.workload_config(_args(), w, 2)["parallelism"] == "replicas"
