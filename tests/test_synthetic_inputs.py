"""CPU tests of the seeded input generators shared by the oracle tests, the GPU tests and the bench:
reproducible, of the stated distributions, and the same on every call."""
import numpy as np

import synthetic_inputs as si


def test_rhs_is_reproducible_and_standard_normal():
    a, b = si.rhs_normal(200000, 7), si.rhs_normal(200000, 7)
    assert np.array_equal(a, b) and not np.array_equal(a, si.rhs_normal(200000, 8))
    assert abs(a.mean()) < 0.01 and abs(a.std() - 1.0) < 0.01
    B = si.rhs_batch(1000, [3, 4, 5])
    assert B.shape == (1000, 3) and np.array_equal(B[:, 1], si.rhs_normal(1000, 4))


def test_poisson_arrivals_have_the_requested_rate():
    t = si.poisson_arrivals(20000, 50.0, seed=1)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.05 / 50.0          # exponential gaps of mean 1 / rate
    assert abs(gaps.std() - 1 / 50.0) < 0.05 / 50.0
    assert np.array_equal(t, si.poisson_arrivals(20000, 50.0, seed=1))


def test_request_mix_is_uniform_over_sizes_and_orders():
    mix = si.request_mix(30000, seed=42)
    Ns = np.array([m[0] for m in mix])
    ks = np.array([m[1] for m in mix])
    for N in (16, 32, 64, 128, 256):
        assert abs((Ns == N).mean() - 0.2) < 0.02
    for k in (2, 3, 4):
        assert abs((ks == k).mean() - 1 / 3) < 0.02
    assert len({m[2] for m in mix}) == len(mix)               # distinct right-hand-side seeds
    assert mix == si.request_mix(30000, seed=42)
