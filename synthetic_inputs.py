"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the benchmark.

Holds no arithmetic of the method: only random right-hand sides drawn with NumPy's default
generator, ``numpy.random.default_rng(seed).standard_normal(ndof)``, and the Poisson request stream of
the serving workload.  The DoF count is computed by each caller on its own side.
"""
import numpy as np


def rhs_normal(ndof, seed):
    """One N(0, 1) right-hand side of length ndof (FP64)."""
    return np.random.default_rng(seed).standard_normal(ndof)


def rhs_batch(ndof, seeds):
    """Column-major (ndof x nrhs) block of N(0, 1) right-hand sides, one seed per column."""
    return np.stack([rhs_normal(ndof, s) for s in seeds], axis=1)


def poisson_arrivals(n, rate, seed):
    """Arrival times (seconds) of n requests of a Poisson process with the given rate (1/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def request_mix(n, seed, sizes=(16, 32, 64, 128, 256), orders=(2, 3, 4)):
    """(N, k, rhs_seed) per request: N and k uniform over the given sets."""
    rng = np.random.default_rng(seed)
    Ns = rng.choice(np.array(sizes), size=n)
    ks = rng.choice(np.array(orders), size=n)
    return [(int(a), int(b), int(seed * 100003 + i)) for i, (a, b) in enumerate(zip(Ns, ks))]
