"""CPU model of the three-way BF16 split behind the FP32 tensor-core products (csrc/tc_gemm.cu),
checked exactly.  No GPU.

x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2), with bf16() round-to-nearest-even to an
8-bit significand.  Each difference is exact in FP32, and x1 + x2 + x3 = x exactly for every FP32 x
whose leading bit is at least 2^-110 (BF16 keeps FP32's exponent range; below that x3 would need
BF16 subnormals).  The BF16x6 product keeps the pairs with p + q <= 4; the dropped ones (a2 b3,
a3 b2, a3 b3) stay below 2^-23 |a b|."""
import numpy as np


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split3(x):
    x = np.asarray(x, dtype=np.float32)
    x1 = bf16(x)
    r1 = (x - x1).astype(np.float32)
    x2 = bf16(r1)
    r2 = (r1 - x2).astype(np.float32)
    x3 = bf16(r2)
    return x1, x2, x3, r1, r2


def random_fp32(n, seed, lo=-100, hi=100):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) * 2.0 ** rng.integers(lo, hi, n)
    # add values just above and below powers of two, where the rounding carries into a new binade
    p = 2.0 ** rng.integers(lo, hi, 64)
    x = np.concatenate([x, p * (1 + 2.0 ** -23), p * (1 - 2.0 ** -24), -p * (1 + 2.0 ** -8 + 2.0 ** -16)])
    return x.astype(np.float32)


def test_split_is_exact():
    x = random_fp32(20000, 1)
    x1, x2, x3, r1, r2 = split3(x)
    xd = x.astype(np.float64)
    # the residuals were formed exactly in FP32
    assert np.array_equal(r1.astype(np.float64), xd - x1.astype(np.float64))
    assert np.array_equal(r2.astype(np.float64), r1.astype(np.float64) - x2.astype(np.float64))
    # x3 needed no rounding, so the three pieces carry x exactly
    assert np.array_equal(x3, r2)
    assert np.array_equal(x1.astype(np.float64) + x2.astype(np.float64) + x3.astype(np.float64), xd)
    for piece in (x1, x2, x3):
        assert np.array_equal(bf16(piece), piece)


def test_piece_magnitudes_and_dropped_pairs():
    a = random_fp32(20000, 2, -60, 60)
    b = random_fp32(20000, 3, -60, 60)
    a1, a2, a3, _, _ = (p.astype(np.float64) for p in split3(a))
    b1, b2, b3, _, _ = (p.astype(np.float64) for p in split3(b))
    ad, bd = a.astype(np.float64), b.astype(np.float64)
    assert np.all(np.abs(a2) <= 2.0 ** -8 * np.abs(ad))
    assert np.all(np.abs(a3) <= 2.0 ** -16 * np.abs(ad))
    kept6 = a1 * b1 + a1 * b2 + a2 * b1 + a1 * b3 + a2 * b2 + a3 * b1
    dropped = ad * bd - kept6
    assert np.all(np.abs(dropped) <= 2.0 ** -23 * np.abs(ad * bd))
    kept3 = a1 * b1 + a1 * b2 + a2 * b1
    assert np.all(np.abs(ad * bd - kept3) <= 2.0 ** -15 * np.abs(ad * bd))
