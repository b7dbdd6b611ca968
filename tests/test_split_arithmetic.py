"""CPU model of the split-precision congruence arithmetic (QCS_TF32X3), behind the
error bound that the GPU split tests state.

Each FP64 operand x is rounded to FP32 and then to a TF32 high part h (10
explicit mantissa bits, rounded to nearest with ties away from zero, as the
conversion the kernel uses); the remainder x - h, taken in FP64, gives the TF32
low part l the same way.  The tensor cores form h_a h_b + h_a l_b + l_a h_b
(TF32 x TF32 products are exact in FP32) and accumulate in FP32.  The dropped l_a l_b term and the split itself cost about
2^-21 of each product, the FP32 accumulation of 3 x 2n terms at most
3 * 2n * 2^-24 of the sum of magnitudes.
"""
from __future__ import annotations

import numpy as np
import pytest


def to_tf32(x32: np.ndarray) -> np.ndarray:
    """Round FP32 values to TF32: nearest, ties away from zero (13 low mantissa bits cleared)."""
    bits = x32.astype(np.float32).view(np.uint32)
    bits = (bits + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return bits.view(np.float32)


def split(x: np.ndarray):
    """hi = tf32(fp32(x)), lo = tf32(fp32(x - hi)) with the remainder taken in FP64."""
    hi = to_tf32(x.astype(np.float32))
    lo = to_tf32((x - hi.astype(np.float64)).astype(np.float32))
    return hi, lo


def split_dot(a: np.ndarray, b: np.ndarray) -> np.float32:
    """sum_k a_k b_k as the three-pass split with FP32 accumulation, pass by pass."""
    ah, al = split(a)
    bh, bl = split(b)
    acc = np.float32(0.0)
    for x, y in ((ah, bh), (ah, bl), (al, bh)):
        for k in range(a.shape[0]):
            acc = np.float32(acc + np.float32(x[k] * y[k]))
    return acc


def test_tf32_rounding_model():
    x = np.array([1.0, 1.0 + 2.0**-11, 1.0 + 2.0**-10, 1.0 + 3 * 2.0**-11, -1.0 - 2.0**-11], np.float32)
    r = to_tf32(x)
    # 1 + 2^-11 is the midpoint of 1 and 1 + 2^-10: ties go away from zero
    assert list(r) == [1.0, 1.0 + 2.0**-10, 1.0 + 2.0**-10, 1.0 + 2.0**-9, -1.0 - 2.0**-10]


@pytest.mark.parametrize("n2", [16, 32])
def test_split_products_meet_the_stated_error(n2):
    """Over random rows of the magnitudes T meets (unit-norm walker rows, orthogonal
    snapshot rows), the split dot product stays within 2^-21 + 3 n2 2^-24 of the sum of
    the products' magnitudes, and a single TF32 pass (no low parts) does not."""
    rng = np.random.default_rng(n2)
    worst, worst_single = 0.0, 0.0
    for _ in range(400):
        a = rng.standard_normal(n2) / np.sqrt(n2)
        b = rng.standard_normal(n2) / np.sqrt(n2)
        exact = float(np.dot(a, b))
        scale = float(np.dot(np.abs(a), np.abs(b)))
        worst = max(worst, abs(float(split_dot(a, b)) - exact) / scale)
        ah, _ = split(a)
        bh, _ = split(b)
        single = float(np.dot(ah.astype(np.float64), bh.astype(np.float64)))
        worst_single = max(worst_single, abs(single - exact) / scale)
    bound = 2.0**-21 + 3 * n2 * 2.0**-24
    assert worst <= bound, (worst, bound)
    assert worst_single > 10 * bound  # the low parts matter
