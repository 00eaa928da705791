"""The kernels divide indices by runtime constants with the Granlund-Montgomery
round-up multiplier (q = (mulhi(n, m) + n) >> s, s = ceil(log2 d),
m = floor(2^32 (2^s - d) / d) + 1), valid for n < 2^31. This checks the same
integer recipe exhaustively for small operands and on random and extreme
operands for divisors up to the largest lattice extents."""
import numpy as np


def make_fastdiv(d):
    s = 0
    while (1 << s) < d:
        s += 1
    m = ((1 << 32) * ((1 << s) - d)) // d + 1
    assert 0 <= m < (1 << 32)
    return m, s


def fdiv(n, m, s):
    hi = (n * m) >> 32
    total = hi + n
    assert total < (1 << 32)
    return total >> s


def test_exhaustive_small():
    for d in range(1, 300):
        m, s = make_fastdiv(d)
        for n in range(0, 5000):
            assert fdiv(n, m, s) == n // d


def test_random_and_extreme_operands():
    rng = np.random.default_rng(0)
    divisors = list(range(1, 2049)) + [3 * 5 * 7 * 11, 12 * 24 * 24, 24 * 24 * 24 * 24, (1 << 30) - 1, (1 << 30) + 3]
    edge = [0, 1, (1 << 31) - 1, (1 << 31) - 2, (1 << 30), (1 << 30) - 1]
    for d in divisors:
        m, s = make_fastdiv(d)
        ns = list(rng.integers(0, 1 << 31, size=200)) + edge + [d - 1, d, d + 1, 2 * d - 1, 2 * d]
        for n in ns:
            n = int(n)
            if n >= (1 << 31):
                continue
            assert fdiv(n, m, s) == n // d, (n, d)
