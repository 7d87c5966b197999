"""SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Used as a counter-based generator: the i-th value of stream ``seed`` is the SplitMix64 output for the
state seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64).  A uniform double on [-1, 1) is formed from the
top 53 bits: u = (z >> 11) * 2^-53, value = 2 u - 1.  This draws the start vector of the eigenvalue
estimate; the CUDA library implements the same published generator independently.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n):
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.arange(1, n + 1, dtype=np.uint64) * GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed, n):
    z = splitmix64(seed, n)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0
