"""CPU oracle of the D step (Algorithm 1, Section 2.2).  TEST INFRASTRUCTURE ONLY.

Only the test suite uses this module; it shares no code with the library.

The D step splits the n columns of M at random into t blocks.  When the caller
gives no permutation, the library draws it from a seed, so both sides restate
the same published generators:

* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; 64-bit constants of Vigna's
  public-domain reference): the state advances by 0x9e3779b97f4a7c15 and each
  output is the state passed through two xor-shift-multiply rounds and a final
  xor-shift.
* A uniform integer in [0, k): draw until the value is at most
  2^64 - 1 - (2^64 mod k), then reduce mod k (every residue equally likely).
* Durstenfeld's Fisher-Yates shuffle of 0..n-1: for i = n-1 down to 1, swap
  entry i with entry j, j uniform in [0, i].
* Even split (the paper's l = n/t): offsets[i] = floor(i n / t).

Parity pins: the SplitMix64 reference outputs for seed 1234567, and the
uniformity of the shuffle over all n! orders for small n.
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK

    def next(self) -> int:
        self.state = (self.state + GAMMA) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def below(self, k: int) -> int:
        """Uniform integer in [0, k) by rejection."""
        limit = MASK - ((1 << 64) % k) % k
        x = self.next()
        while x > limit:
            x = self.next()
        return x % k


def permutation(n: int, seed: int) -> np.ndarray:
    """Fisher-Yates (Durstenfeld) shuffle of the identity."""
    rng = SplitMix64(seed)
    a = list(range(n))
    for i in range(n - 1, 0, -1):
        j = rng.below(i + 1)
        a[i], a[j] = a[j], a[i]
    return np.array(a, dtype=np.int64)


def even_offsets(n: int, t: int) -> np.ndarray:
    """Block boundaries of t blocks of sizes floor(n/t) or ceil(n/t)."""
    return np.array([(i * n) // t for i in range(t + 1)], dtype=np.int64)


def partition(n: int, t: int, seed: int):
    """The D step drawn from a seed: (perm, offsets)."""
    if not (1 <= t <= n):
        raise ValueError("need 1 <= t <= n")
    return permutation(n, seed), even_offsets(n, t)
