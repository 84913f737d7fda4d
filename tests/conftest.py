import os
import sys

import pytest


def _one_blas_thread():
    # the oracle's matrices in the CPU tests are small: one BLAS thread is
    # fastest.  GPU runs keep every core: their oracle runs are full-size.
    for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    markexpr = getattr(config.option, "markexpr", "") or ""
    if "gpu" not in markexpr or "not gpu" in markexpr:
        _one_blas_thread()
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def lib():
    """The CUDA library through its C-ABI binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_5583_gb300 import binding
    return binding.load()
