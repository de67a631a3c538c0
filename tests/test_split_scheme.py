"""The integer slicing of the tensor-core residual, restated in Python integers.

The CUDA kernel `k_oz_split` writes every binary64 value x of a row (or column) whose
largest magnitude lies below 2^e as seven signed base-256 digits: V = round(x 2^(56-e))
from the bits of x, then q_1 = round(V / 2^48), V -= q_1 2^48, ..., q_7 = V.  This test
checks the arithmetic itself on random rows (zeros, signs, exponent spread, subnormals):
the digits fit the ranges the exactness argument of the accumulation needs
(|q_1| <= 256, |q_s| <= 128) and reproduce x within 2^(e-57), the half-unit of the
56-bit grid.  The GPU parity tests check the kernel's residual against the oracle.
"""
import struct
from fractions import Fraction

import numpy as np


def fixed56(x: float, e: int) -> int:
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    E = (b >> 52) & 0x7FF
    M = b & ((1 << 52) - 1)
    if E != 0:
        M |= 1 << 52
    sh = (E if E != 0 else 1) - 1019 - e
    if sh >= 0:
        v = M << sh
    elif sh > -60:
        v = (M + (1 << (-sh - 1))) >> (-sh)
    else:
        v = 0
    return -v if b >> 63 else v


def digits(V: int) -> list[int]:
    q = []
    for s in range(7):
        sh = 8 * (6 - s)
        if sh > 0:
            d = (V + (1 << (sh - 1))) >> sh
            V -= d << sh
        else:
            d = V
        q.append(d)
    return q


def row_exponent(row) -> int:
    """Smallest e with max |x| < 2^e (0 for a zero row), as `k_oz_rowexp` computes it."""
    mx = float(np.max(np.abs(row)))
    return int(np.frexp(mx)[1]) if mx > 0 else 0


def check_row(row):
    e = row_exponent(row)
    for x in row:
        q = digits(fixed56(float(x), e))
        assert abs(q[0]) <= 256 and all(abs(d) <= 128 for d in q[1:])
        val = Fraction(2) ** (e - 8) * sum(Fraction(d) * Fraction(2) ** (-8 * s) for s, d in enumerate(q))
        assert abs(val - Fraction(float(x))) <= Fraction(2) ** (e - 57)


def test_random_rows():
    rng = np.random.default_rng(1)
    for trial in range(1500):
        row = rng.standard_normal(8) * np.exp2(rng.integers(-40, 40, 8))
        if trial % 5 == 0:
            row[rng.integers(0, 8)] = 0.0
        check_row(row)


def test_extremes():
    tiny = np.nextafter(0.0, 1.0)
    check_row(np.array([tiny, -3 * tiny, 0.0]))                 # subnormal row
    check_row(np.array([1e-310, 2.5e-308, -1e-300]))            # subnormal and normal mixed
    check_row(np.array([1.7e308, -1e300, 1.0, -1e-300]))        # near the overflow threshold
    check_row(np.array([0.5, -0.5, 0.25]))                      # powers of two: ties of the digit rounding
    check_row(np.array([255.0 / 256, -1.0 + 2.0 ** -53, 2.0 ** -60]))


def test_exact_values_are_exact():
    """Values with at most 56 significant bits below the row's exponent are reproduced
    exactly (no rounding of V)."""
    rng = np.random.default_rng(2)
    for _ in range(300):
        k = rng.integers(-2 ** 52, 2 ** 52, 4).astype(np.float64)
        row = np.ldexp(k, -20)
        e = row_exponent(row)
        for x in row:
            q = digits(fixed56(float(x), e))
            val = Fraction(2) ** (e - 8) * sum(Fraction(d) * Fraction(2) ** (-8 * s) for s, d in enumerate(q))
            assert val == Fraction(float(x))
