"""The split sum behind the FP32 mass partials and reductions, emulated in NumPy FP32.

The kernels (split_add2i in ace_kernels.cuh) add each FP32 value v as t = v + 192. For
|v| < 64, t lies in [128, 256), where FP32 values are 2^-16 apart, so h = t - 192 is v
rounded to a multiple of 2^-16, the bit pattern difference bits(t) - bits(192) equals
h * 2^16 exactly, and the remainder v - h is exact. The kernels sum the raw bit patterns
of t in a 32-bit integer modulo 2^32 and the remainders in FP32. These tests check that
arithmetic on the host, bit for bit in FP32, against exact rational sums. The kernels'
results are checked against FP64 sums on the GPU (tests/test_gpu_mass_paths.py).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

C192 = np.float32(192.0)
BITS192 = int(np.array([192.0], dtype=np.float32).view(np.uint32)[0])


def split_sum(v):
    """Emulate split_add2i over the values in order; returns (integer part in units of
    2^-16, FP32 remainder sum, the rounded parts h, the largest |partial remainder sum|)."""
    v = np.asarray(v, dtype=np.float32)
    t = (v + C192).astype(np.float32)
    h = (t - C192).astype(np.float32)
    ai = int(t.view(np.uint32).astype(np.uint64).sum()) % (1 << 32)
    m = (ai - len(v) * BITS192) % (1 << 32)
    if m >= 1 << 31:
        m -= 1 << 32
    lo = np.float32(0.0)
    lo_max = 0.0
    for r in (v - h).astype(np.float32):
        lo = np.float32(lo + r)
        lo_max = max(lo_max, abs(float(lo)))
    return m, lo, h, lo_max


def test_bits_of_t_give_the_rounded_part_exactly():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.uniform(-63.9, 63.9, 20000), rng.uniform(-2, 2, 20000), rng.normal(0, 1e-6, 2000),
                        [0.0, -0.0, 2.0 ** -17, -(2.0 ** -17), 63.99, -63.99, 1.5, 2.0 ** -16]]).astype(np.float32)
    t = (v + C192).astype(np.float32)
    h = (t - C192).astype(np.float32)
    diff = t.view(np.uint32).astype(np.int64) - BITS192
    # the bit-pattern difference is the rounded part in units of 2^-16
    assert np.array_equal(diff.astype(np.float64) * 2.0 ** -16, h.astype(np.float64))
    # h is v rounded to the nearest multiple of 2^-16, and the remainder is exact
    assert np.all(np.abs(v.astype(np.float64) - h.astype(np.float64)) <= 2.0 ** -17)
    r = (v - h).astype(np.float32)
    assert np.array_equal(r.astype(np.float64), v.astype(np.float64) - h.astype(np.float64))


@pytest.mark.parametrize("n,scale", [(16, 1.0), (4 * 4095, 1.99), (8192, 1.99), (1000, 1e-3)])
def test_integer_part_is_the_exact_sum_of_the_rounded_parts(n, scale):
    rng = np.random.default_rng(n)
    v = (rng.uniform(-1.0, 1.0, n) * scale).astype(np.float32)
    m, lo, h, lo_max = split_sum(v)
    exact_h = sum(Fraction(float(x)) for x in h)
    assert Fraction(m, 1 << 16) == exact_h
    # the total is the exact sum up to the FP32 rounding of the remainder sum: each of
    # the n additions rounds by at most half a unit in the last place of the largest
    # partial remainder sum
    exact = math.fsum(float(x) for x in v)
    total = m * 2.0 ** -16 + float(lo)
    assert abs(total - exact) <= n * float(np.spacing(np.float32(lo_max))) / 2


def test_bound_of_the_integer_sum():
    """8192 values just below 2, all of one sign, keep the true sum of the rounded parts
    below 2^15, so the 32-bit wrap-around total is still exact (the reductions give a
    thread at most 8192 values; the quad step kernels' bands 4 x 4095)."""
    v = np.full(8192, np.float32(1.9999), dtype=np.float32)
    m, lo, h, _ = split_sum(v)
    assert Fraction(m, 1 << 16) == sum(Fraction(float(x)) for x in h)
    assert abs(m) < 1 << 31
    v = -v
    m, lo, h, _ = split_sum(v)
    assert Fraction(m, 1 << 16) == sum(Fraction(float(x)) for x in h)


def test_values_of_two_or_more_are_why_the_kernels_check_the_maximum():
    """Beyond the bound the integer total wraps: 2^15 values of 40 overflow it. The
    kernels track the largest magnitude a thread saw and sum its values again in FP64
    when it reaches 2, so this case never reaches their split path."""
    v = np.full(1 << 15, np.float32(40.0), dtype=np.float32)
    m, lo, h, _ = split_sum(v)
    assert Fraction(m, 1 << 16) != sum(Fraction(float(x)) for x in h)
