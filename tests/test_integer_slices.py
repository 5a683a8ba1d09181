"""The arithmetic behind the tensor-core FP64 contractions, restated on the CPU
in Python integers (no GPU, no library code): the claims of the
error-free integer-slice product that the kernels rely on.

Each FP64 value x of a row (or column) is written in fixed point against the
largest binary exponent E of that row, x = sign M 2^(E - 1075) with M the
53-bit significand shifted right by E - e(x), and the top 49 bits of M are cut
into seven 7-bit slices, M ~ sum_s a_s 2^(46 - 7 s).  For a dot product of
length K <= 64 the diagonals D_d = sum_{s+t=d} sum_k a_sk b_tk (d = 0..6)
are accumulated, then acc = sum_d D_d 2^(7 (6 - d)) and one rounding.

Checked here:
* |D_d| < 2^23 even for all-maximal slices, so an FP32 accumulator holds
  every partial sum exactly; |acc| < 2^63 (int64);
* the dropped diagonals and truncated bits keep every entry within
  2^-39.8 max|x| max|y| (K = 64) - the bound the GPU tests use with a factor
  4 of margin - on rows spanning many orders of magnitude;
* integers whose products and sums are exact in FP64 come out exactly.
"""
import math
import struct

import numpy as np

S, BITS, K = 7, 7, 64


def _bexp(x):
    return (struct.unpack("<q", struct.pack("<d", float(x)))[0] >> 52) & 0x7FF


def _slices(x, E):
    b = struct.unpack("<q", struct.pack("<d", float(x)))[0]
    ex = (b >> 52) & 0x7FF
    if ex == 0 or E - ex >= 53:
        return [0] * S
    M = ((b & ((1 << 52) - 1)) | (1 << 52)) >> (E - ex)
    a = [(M >> (46 - BITS * s)) & ((1 << BITS) - 1) for s in range(S)]
    return [-v for v in a] if b < 0 else a


def _dot(xs, ys):
    """sum_k x_k y_k by the slice scheme; returns (value, diagonals, acc)."""
    E = max(_bexp(x) for x in xs)
    F = max(_bexp(y) for y in ys)
    A = [_slices(x, E) for x in xs]
    B = [_slices(y, F) for y in ys]
    D = [sum(A[k][s] * B[k][d - s] for k in range(len(xs)) for s in range(d + 1)) for d in range(S)]
    acc = sum(D[d] << (BITS * (S - 1 - d)) for d in range(S))
    val = math.ldexp(float(acc), E + F - 2100) if E and F else 0.0
    return val, D, acc


def test_diagonals_fit_fp32_and_recombination_fits_int64():
    top = (1 << BITS) - 1
    worst = [(d + 1) * K * top * top for d in range(S)]      # all slices maximal, same sign
    assert max(worst) < 2 ** 23                              # exact in FP32 (integers below 2^24)
    acc = sum(w << (BITS * (S - 1 - d)) for d, w in enumerate(worst))
    assert acc < 2 ** 63
    # the same numbers from the scheme itself: x = y = the largest values below 2^E
    x = [math.nextafter(2.0, 0.0)] * K
    _, D, a = _dot(x, x)
    assert all(abs(v) <= w for v, w in zip(D, worst)) and abs(a) < 2 ** 63


def test_error_within_the_stated_bound_on_wide_ranges():
    rng = np.random.default_rng(5)
    worst = 0.0
    for trial in range(60):
        n = int(rng.integers(1, K + 1))
        x = rng.standard_normal(n) * 10.0 ** rng.uniform(-12, 3, n)       # entries over 15 decades
        y = rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 6) * 10.0 ** rng.uniform(-3, 0, n)
        if trial % 7 == 0:
            x[::3] = 0.0
        val, _, _ = _dot(x, y)
        exact = math.fsum(float(a) * float(b) for a, b in zip(x, y))
        scale = np.max(np.abs(x)) * np.max(np.abs(y))
        worst = max(worst, abs(val - exact) / scale)
    assert worst < 2.0 ** -39.8
    assert worst > 0.0          # the scheme does drop bits: the bound is not vacuous


def test_exact_on_integer_inputs():
    rng = np.random.default_rng(6)
    for _ in range(20):
        x = rng.integers(-1000, 1001, size=K).astype(float)
        y = rng.integers(-1000, 1001, size=K).astype(float)
        val, _, _ = _dot(x, y)
        assert val == float(int(np.dot(x.astype(np.int64), y.astype(np.int64))))
