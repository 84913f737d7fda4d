"""GB300-native DFC-LRR (divide-and-conquer low-rank representation).

The solver is the C-ABI library libdfc_lrr.so built from csrc/ (see build.py);
``binding`` marshals torch tensors into its calls.  Nothing here computes on
the host: without the built library the solver entry points raise.
"""
__all__ = ["binding", "synth", "build"]
