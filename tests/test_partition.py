"""D step (Algorithm 1, Section 2.2): the seeded random partition.  The oracle's
generator is pinned to published reference outputs and to uniformity; the
library's host-side dfc_partition must reproduce it bit for bit (no GPU)."""
import ctypes
import itertools
import math

import numpy as np
import pytest

from oracle import partition as opart


def test_splitmix64_reference_outputs():
    # published first outputs of SplitMix64 seeded with 1234567
    g = opart.SplitMix64(1234567)
    assert [g.next() for _ in range(5)] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                            4593380528125082431, 16408922859458223821]


def _chi2_over_orders(shuffle, n, draws):
    orders = {p: i for i, p in enumerate(itertools.permutations(range(n)))}
    counts = np.zeros(len(orders))
    for s in range(draws):
        counts[orders[tuple(shuffle(n, s))]] += 1
    expect = draws / len(orders)
    return float(np.sum((counts - expect) ** 2 / expect)), len(orders) - 1


def _chi2_threshold(df):
    from scipy.stats import chi2
    return chi2.ppf(1 - 1e-6, df)


def test_shuffle_is_uniform_over_all_orders():
    stat, df = _chi2_over_orders(lambda n, s: opart.permutation(n, s), 4, 24000)
    assert stat < _chi2_threshold(df), stat


def test_planted_naive_shuffle_fails_the_uniformity_pin():
    # swapping with a position uniform in [0, n) instead of [0, i] is the
    # classic biased shuffle; the pin above must reject it
    def naive(n, seed):
        g = opart.SplitMix64(seed)
        a = list(range(n))
        for i in range(n - 1, 0, -1):
            j = g.below(n)
            a[i], a[j] = a[j], a[i]
        return a
    stat, df = _chi2_over_orders(naive, 4, 24000)
    assert stat > _chi2_threshold(df), stat


def test_even_split_and_permutation():
    for n, t in [(1, 1), (7, 7), (10, 3), (240, 3), (20000, 40), (2432, 8)]:
        perm, off = opart.partition(n, t, 5)
        assert sorted(perm.tolist()) == list(range(n))
        sizes = np.diff(off)
        assert off[0] == 0 and off[-1] == n and len(sizes) == t
        assert sizes.min() >= n // t and sizes.max() <= math.ceil(n / t)
    with pytest.raises(ValueError):
        opart.partition(3, 4, 0)


@pytest.fixture(scope="module")
def lib():
    from paper_1304_5583_gb300 import binding, build
    build.build()
    return binding.load()


@pytest.mark.parametrize("n,t,seed", [(1, 1, 0), (2, 2, 1), (30, 3, 7), (240, 3, 11), (5000, 10, 2 ** 64 - 1),
                                      (100003, 40, 12345678901234567)])
def test_library_partition_matches_oracle_bit_for_bit(lib, n, t, seed):
    from paper_1304_5583_gb300 import binding
    perm, off = binding.partition(n, t, seed)
    operm, ooff = opart.partition(n, t, seed)
    assert np.array_equal(perm, operm)
    assert np.array_equal(off, ooff)


def test_library_partition_rejects_bad_arguments(lib):
    buf = np.zeros(8, np.int64)
    ptr = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    assert lib.dfc_partition(0, 1, 0, ptr, ptr) == -1
    assert lib.dfc_partition(3, 0, 0, ptr, ptr) == -1
    assert lib.dfc_partition(3, 4, 0, ptr, ptr) == -1
    assert lib.dfc_partition(3, 2, 0, None, None) == -1
    assert lib.dfc_partition(3, 2, 0, None, ptr) == 0


def test_solve_arguments_accept_a_drawn_partition(lib):
    # host-side validation with perm and offsets left to the library
    from paper_1304_5583_gb300 import binding
    p = binding.LrrProblem()
    p.M = ctypes.c_void_p(0x1000)   # never dereferenced by the host-side checks
    p.m, p.n, p.ldm, p.t, p.seed = 20, 30, 20, 3, 99
    o = binding.options(0.1)
    assert lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(o)) > 0
    p.t = 31
    assert lib.lrr_workspace_bytes(ctypes.byref(p), ctypes.byref(o)) == 0
