"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares; host-side argument checks run without a device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names.update(re.findall(r"LRR_API\s+[\w\s\*]+?\b(\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1304_5583_gb300 import binding, build
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1304_5583_gb300 import binding
    names = _declared()
    assert names == set(binding.EXPORTS), names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_defaults(lib):
    from paper_1304_5583_gb300 import binding
    assert binding.status_string(0) == "ok"
    assert "NaN" in binding.status_string(-2)
    o = binding.LrrOptions()
    lib.lrr_default_options(ctypes.byref(o))
    assert o.rho == 1.1 and o.mu0 == 1e-6 and o.mu_max == 1e10 and o.max_iter == 1000


def _problem(n=30, m=20, t=3, perm=None, offsets=None):
    from paper_1304_5583_gb300 import binding
    p = binding.LrrProblem()
    p.M = ctypes.c_void_p(0x1000)   # never dereferenced by the host-side checks
    p.m, p.n, p.ldm, p.t = m, n, m, t
    perm = np.arange(n, dtype=np.int64) if perm is None else perm
    offsets = np.linspace(0, n, t + 1).astype(np.int64) if offsets is None else offsets
    p.perm = perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    p.offsets = offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    return p, (perm, offsets)


def test_workspace_size_and_argument_validation(lib):
    from paper_1304_5583_gb300 import binding
    o = binding.options(0.1)
    p, keep = _problem()
    assert lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(o)) > 0
    bad_perm = np.arange(30, dtype=np.int64); bad_perm[0] = 1
    p2, keep2 = _problem(perm=bad_perm)
    assert lib.lrr_workspace_bytes(ctypes.byref(p2), ctypes.byref(o)) == 0
    p3, keep3 = _problem(offsets=np.array([0, 10, 10, 30], np.int64))
    assert lib.lrr_workspace_bytes(ctypes.byref(p3), ctypes.byref(o)) == 0
    o.rho = 1.0
    assert lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(o)) == 0
    # lrr_solve insists on one block; rejected before any device work
    o = binding.options(0.1)
    r = binding.LrrResult()
    assert lib.lrr_solve(ctypes.byref(p), ctypes.byref(o), None, 0, ctypes.byref(r), None) == -1


def test_tensor_core_product_rejects_bad_shapes_without_a_device(lib):
    # argument checks come before any device work, so fake pointers are safe here
    fake = ctypes.c_void_p(0x1000)
    f = lib.lrr_gemm_bf16
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    assert f(fake, 64, fake, 64, fake, 128, 128, 65535 * 128 + 1, 64, None) == -1   # too many column tiles
    assert f(fake, 32, fake, 64, fake, 128, 128, 128, 64, None) == -1               # lda < K
    assert f(None, 64, fake, 64, fake, 128, 128, 128, 64, None) == -1



@pytest.mark.parametrize("field,value", [("lambda_", 0.0), ("lambda_", -1.0), ("rho", 0.9), ("mu0", 0.0),
                                         ("mu_max", 1e-7), ("eps", 0.0), ("max_iter", 0), ("precision", 3),
                                         ("precision", -1)])
def test_every_invalid_option_is_rejected_on_the_host(lib, field, value):
    from paper_1304_5583_gb300 import binding
    p, keep = _problem()
    o = binding.options(0.1)
    assert lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(o)) > 0
    setattr(o, field, value)
    assert lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(o)) == 0
    r = binding.LrrResult()
    assert lib.dfc_lrr_solve(ctypes.byref(p), ctypes.byref(o), None, 0, ctypes.byref(r), None) == -1


@pytest.mark.parametrize("case", ["offsets_start", "offsets_end", "perm_range", "t_zero", "t_above_n", "ldm", "null_M"])
def test_every_invalid_problem_is_rejected_on_the_host(lib, case):
    from paper_1304_5583_gb300 import binding
    n, t = 30, 3
    perm = np.arange(n, dtype=np.int64)
    offsets = np.array([0, 10, 20, 30], np.int64)
    if case == "offsets_start":
        offsets = np.array([1, 10, 20, 30], np.int64)
    if case == "offsets_end":
        offsets = np.array([0, 10, 20, 29], np.int64)
    if case == "perm_range":
        perm = perm.copy(); perm[5] = n
    p, keep = _problem(n=n, t=t, perm=perm, offsets=offsets)
    if case == "t_zero":
        p.t = 0
    if case == "t_above_n":
        p.t = n + 1
    if case == "ldm":
        p.ldm = p.m - 1
    if case == "null_M":
        p.M = None
    o = binding.options(0.1)
    assert lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(o)) == 0
    r = binding.LrrResult()
    assert lib.dfc_lrr_solve(ctypes.byref(p), ctypes.byref(o), None, 0, ctypes.byref(r), None) == -1


def test_workspace_grows_with_the_problem(lib):
    from paper_1304_5583_gb300 import binding
    o = binding.options(0.1)
    sizes = []
    for n in (30, 60, 120):
        p, keep = _problem(n=n, t=3)
        sizes.append(lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(o)))
    assert sizes[0] < sizes[1] < sizes[2]
    # the mixed form adds its bf16 operands
    p, keep = _problem(n=60, t=3)
    om = binding.options(0.1, precision="mixed")
    assert lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(om)) > sizes[1]


def test_factor_max_rank_bounds_the_factored_output():
    """min(m, l_1) for t > 1, min(m, n) for t = 1, 0 for an invalid problem."""
    import ctypes
    from paper_1304_5583_gb300 import binding
    lib = binding.load()
    off = np.array([0, 7, 19, 30], dtype=np.int64)
    p = binding.LrrProblem()
    p.m, p.n, p.ldm, p.t = 12, 30, 12, 3
    p.offsets = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    assert lib.lrr_factor_max_rank(ctypes.byref(p)) == 7
    p.m = 5
    assert lib.lrr_factor_max_rank(ctypes.byref(p)) == 5
    p.t, p.m = 1, 40
    assert lib.lrr_factor_max_rank(ctypes.byref(p)) == 30
    p.t = 0
    assert lib.lrr_factor_max_rank(ctypes.byref(p)) == 0
