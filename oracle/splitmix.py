"""SplitMix64 (Steele, Lea, Flood 2014; reference code by S. Vigna), oracle copy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Counter form: the k-th output (k = 0, 1, ...) of the stream seeded with s is
mix(s + (k + 1) * 0x9E3779B97F4A7C15) where
mix(z) = z3 ^ (z3 >> 31), z2 = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9,
z3 = (z2 ^ (z2 >> 27)) * 0x94D049BB133111EB (all mod 2^64).  A double in
[0, 1) is (out >> 11) * 2^-53.
"""
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1


def splitmix64(seed, k):
    """k-th output of the stream seeded with ``seed`` (Python ints)."""
    z = (seed + (k + 1) * GAMMA) & MASK
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def uniform01(seed, k):
    return (splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0)


def complex_start_vector(seed, n):
    """Entry i = (2 u_{2i} - 1) + 1j (2 u_{2i+1} - 1)."""
    out = np.empty(n, dtype=np.complex128)
    for i in range(n):
        out[i] = complex(2.0 * uniform01(seed, 2 * i) - 1.0, 2.0 * uniform01(seed, 2 * i + 1) - 1.0)
    return out
