"""The mixture kernels divide by a per-frame or per-stream divisor d = 2 m
(m = min(t, N) or N, 1 <= m <= 65535) with one multiply: floor(n R / 2^40),
R = ceil(2^40 / d), for numerators n < 2^22.  Check the sufficient condition
of the multiply-by-reciprocal theorem (2^40 <= R d <= 2^40 + 2^18) for every
such divisor, and the identity itself against exact integer division on
every multiple boundary of a spread of divisors."""
import numpy as np

TWO40 = 1 << 40
NMAX = 1 << 22


def _recip(d: int) -> int:
    return (TWO40 + d - 1) // d


def test_reciprocal_condition_for_every_divisor():
    for m in range(1, 65536):
        d = 2 * m
        r = _recip(d)
        assert TWO40 <= r * d <= TWO40 + (1 << 18), d


def test_multiply_matches_division_on_multiple_boundaries():
    rng = np.random.default_rng(40)
    ms = sorted(set([1, 2, 3, 7, 64, 255, 256, 257, 1000, 4095, 4096, 32767, 65534, 65535] +
                    rng.integers(1, 65536, size=60).tolist()))
    for m in ms:
        d = 2 * m
        r = _recip(d)
        k = np.arange(0, NMAX // d + 2, dtype=object)
        n = np.concatenate([k * d, k * d - 1, k * d + 1])
        n = np.array([x for x in n if 0 <= x < NMAX], dtype=object)
        got = (n * r) >> 40
        want = n // d
        assert (got == want).all(), m
