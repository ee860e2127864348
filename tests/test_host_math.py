"""Host-side integer arithmetic the kernels rely on (CPU only).

Work-item indices are split by multiply-high division: for 0 <= n < 2^32 and a divisor d >= 2,
m = ceil(2^64 / d) (computed as floor((2^64 - 1) / d) + 1) gives floor(n m / 2^64) = floor(n / d)
(division by invariant integers using multiplication, Granlund and Montgomery 1994); d = 1 uses
m = 0 and the quotient n.  Checked here exhaustively at the edges and on random operands, in exact
integer arithmetic, with the same expressions the library uses."""
import numpy as np


def _magic(d):
    return 0 if d <= 1 else (2**64 - 1) // d + 1


def _udiv(n, m):
    return (n * m) >> 64 if m else n


def test_multiply_high_division_edges():
    ds = [1, 2, 3, 5, 7, 64, 152, 1000, 65535, 65536, 2**31 - 1, 2**31, 2**32 - 2, 2**32 - 1]
    ns = [0, 1, 2, 63, 64, 65, 2**16, 2**31 - 1, 2**31, 2**32 - 2, 2**32 - 1]
    for d in ds:
        m = _magic(d)
        assert m < 2**64
        for n in ns + [d - 1, d, d + 1, 2 * d - 1, 2 * d, (2**32 - 1) // d * d, (2**32 - 1) // d * d - 1]:
            if 0 <= n < 2**32:
                assert _udiv(n, m) == n // d, (n, d)


def test_multiply_high_division_random():
    rng = np.random.default_rng(5)
    for d in rng.integers(2, 2**32, size=300, dtype=np.uint64):
        d = int(d)
        m = _magic(d)
        for n in rng.integers(0, 2**32, size=200, dtype=np.uint64):
            n = int(n)
            assert _udiv(n, m) == n // d
