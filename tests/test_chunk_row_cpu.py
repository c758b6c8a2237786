"""The per-chunk kernels find a chunk's row as the high word of u * m with
m = ceil(2^32 / cpr) instead of dividing.  Check the identity
floor(u * m / 2^32) == u // cpr on every row boundary (u = y*cpr - 1, y*cpr,
y*cpr + cpr - 1) for every even chunks-per-row up to 512 and every row up to
8192, which covers every frame the library accepts."""
import numpy as np


def test_multiply_high_row_matches_division():
    rows = np.arange(0, 8193, dtype=np.uint64)
    for cpr in range(2, 513, 2):
        m = np.uint64(((1 << 32) + cpr - 1) // cpr)
        starts = rows * np.uint64(cpr)
        u = np.concatenate([starts, starts + np.uint64(cpr - 1), starts[1:] - np.uint64(1)])
        u = u[u < np.uint64(8192 * cpr)]
        got = (u * m) >> np.uint64(32)
        assert np.array_equal(got, u // np.uint64(cpr)), cpr
