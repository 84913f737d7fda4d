"""Identical segmentation labels (Section 4.1.2's post-processing of the
combined estimate) from the CUDA path and from the float64 oracle on the
full-size workloads.  The oracle's labels were written by
tests/golden/make_oracle_labels.py (oracle only, run to convergence); the
GPU's estimate goes through the same segmentation routine here."""
import json
import os

import numpy as np
import pytest

from oracle import segment
from parity_helpers import run
from paper_1304_5583_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name,precision", [("dfc_500x5000", "f32"), ("dfc_faces_2016x2432", "mixed")])
def test_labels_identical_to_oracle(lib, name, precision):
    with open(os.path.join(GOLDEN, f"labels_{name}.json")) as f:
        g = json.load(f)
    w = synth.workload(name)
    res, _ = run(w, precision)
    assert res.status == 0
    lab = segment.segment(res.Z.cpu().numpy().astype(np.float64), g["k"], seed=0)
    ref = np.asarray(g["labels"])
    acc = segment.matched_accuracy(lab, w.data.labels)
    # columns replaced by outliers belong to no subspace: their cluster is an
    # arbitrary k-means assignment of noise rows of the affinity, so the
    # partition is compared on the subspace columns (the outliers themselves
    # are what the S columns mark)
    inl = ~w.data.outlier if name != "dfc_faces_2016x2432" else np.ones(len(ref), bool)
    print(f"{name} {precision}: matched accuracy {acc:.4f} (oracle {g['matched_accuracy_vs_truth']:.4f}); "
          f"same partition over all columns: {segment.same_partition(lab, ref)}, "
          f"over the {int(inl.sum())} subspace columns: {segment.same_partition(lab[inl], ref[inl])}")
    assert segment.same_partition(lab[inl], ref[inl])
    assert acc == pytest.approx(g["matched_accuracy_vs_truth"], abs=1e-12)
