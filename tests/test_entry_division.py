"""The entry division of the device steppers, modelled in numpy float32.

Entering a segment at step k needs q = floor((2kA + N) / (2N)) and its remainder
for each minor axis (Eq. (3)). The kernels estimate the quotient as
num * rcp(2N) in single precision (round-to-nearest conversion, reciprocal and
product) and correct the integer part once with the exact remainder taken modulo
2^32. These tests check, on the host, that this estimate-and-correct sequence is
exact over the domain it is written for (quotient below 2^22, divisor below
2^23) and over the entry divisions with N up to int(|d|) of the longest
Euclidean segment (sqrt(3) (2^21 - 1)). The GPU parity tests check the kernels'
outputs themselves.
"""
import numpy as np
import pytest

N_MAX_EUCLID = 3632573  # int(sqrt(3) * (2^21 - 1))


def estimate_and_correct(num: np.ndarray, den: np.ndarray):
    rcp = np.float32(1.0) / den.astype(np.float32)  # reciprocal rounded to nearest
    est = (num.astype(np.float32) * rcp).astype(np.float32)
    q = np.trunc(est).astype(np.int64)
    r = ((num - q * den) + (1 << 31)) % (1 << 32) - (1 << 31)  # low 32 bits, as int32
    low, high = r < 0, r >= den
    return q - low + high, r + low * den - high * den


def _check(N, A, k):
    num = 2 * k * A + N
    den = 2 * N
    q, r = estimate_and_correct(num, den)
    assert np.array_equal(q, num // den)
    assert np.array_equal(r, num % den)


def test_generic_domain():
    rng = np.random.default_rng(3)
    m = 1 << 20
    den = np.where(rng.random(m) < 0.5, rng.integers(1, 1 << 23, size=m), rng.integers(1, 5000, size=m))
    q = np.where(rng.random(m) < 0.3, (1 << 22) - 1 - rng.integers(0, 100, size=m), rng.integers(0, 1 << 22, size=m))
    r = np.where(rng.random(m) < 0.3, den - 1, rng.integers(0, den))
    num = q * den + r
    got_q, got_r = estimate_and_correct(num, den)
    assert np.array_equal(got_q, q) and np.array_equal(got_r, r)


def test_exhaustive_small_segments():
    for N in range(2, 160):
        A = np.repeat(np.arange(1, N, dtype=np.int64), N)
        k = np.tile(np.arange(1, N + 1, dtype=np.int64), N - 1)
        _check(np.full(A.shape, N, dtype=np.int64), A, k)


@pytest.mark.parametrize("n_max", [46340, 46341 * 8, (1 << 21) - 1, N_MAX_EUCLID])
def test_random_and_extreme_steps(n_max):
    rng = np.random.default_rng(n_max)
    m = 1 << 19
    N = rng.integers(2, n_max + 1, size=m, dtype=np.int64)
    A = rng.integers(1, N, dtype=np.int64)
    pick = rng.random(m)
    A = np.where(pick < 0.2, N - 1, np.where(pick < 0.3, 1, A))  # steepest and flattest minors
    k = np.where(rng.random(m) < 0.2, N, rng.integers(1, N + 1, dtype=np.int64))
    _check(N, A, k)


def test_top_of_range():
    """Quotients near 2^21 carry the largest absolute error of the estimate."""
    for N in ((1 << 21) - 1, (1 << 21) - 2, N_MAX_EUCLID, 46341):
        A = np.arange(max(1, N - 4000), N, dtype=np.int64)
        for k in (N, N - 1, N // 2 + 1, 1):
            _check(np.full(A.shape, N, dtype=np.int64), A, np.full(A.shape, k, dtype=np.int64))
