"""CPU model of the arithmetic of the FP64 product emulated on the BF16 tensor cores (csrc/ozaki.cu),
checked against exact rational arithmetic.  No GPU.

The scheme is an error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump (2012), restated
here from its description, not from the kernel's code:

* row i of op(A) is scaled by 2^-(E_i+1) and column j of op(B) by 2^-(F_j+1), where 2^E_i (2^F_j)
  is the smallest power of two above every magnitude of the row (column);
* each scaled entry is truncated to a 56-bit fixed-point integer X = trunc(x 2^(55-E)) and written
  in balanced radix 2^7, X = sum_{p=1..8} a_p 2^(56-7p) with |a_p| <= 64, most significant digit
  first, each digit the nearest integer to the remainder;
* the digit products a_p b_q 2^-7(p+q) with p + q <= 9 are summed: the diagonals d = p + q <= 7
  exactly per 512-deep chunk of K (FP32 accumulators that never exceed 2^24 units), added into a
  64-bit integer in units of 2^-49; the diagonals d = 8, 9 into one FP32 accumulator over all of K;
* C_ij = 2^(E_i+F_j+2) (acc 2^-49 + shared).

The model shows which error bound the scheme has: it is relative to the row and column scales,
|err_ij| <= K 2^(E_i+F_j) (2^-52.6 + 2^-53 + K 2^-62.2) (truncation and dropped pairs, the final
rounding to FP64, the FP32 accumulator of d = 8, 9), not to (|A| |B|)_ij as a native FP64 product's
bound is.  With rows or columns whose entries span many binades the two differ, and the last test
shows it.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

CHUNK = 512      # K of one exact chunk
SLICE = 16       # K of one MMA
KMAX = 32768     # K of one launch
NDIG = 8
DROP = 10        # pairs with p + q >= DROP are not formed
PAIRS = [(p, q) for p in range(1, NDIG + 1) for q in range(1, NDIG + 1) if p + q < DROP]


def scale_exp(v):
    """Smallest E with |x| < 2^E for every x of v (None for an all-zero vector)."""
    m = max(abs(float(x)) for x in v)
    return None if m == 0.0 else math.frexp(m)[1]


def fixed(x, E):
    return int(Fraction(float(x)) * Fraction(2) ** (55 - E))  # int() truncates toward zero


def balanced_digits(X):
    out = []
    for p in range(1, NDIG + 1):
        sh = 56 - 7 * p
        a = (X + (1 << (sh - 1))) >> sh if sh > 0 else X  # nearest integer, ties up
        X -= a << sh
        out.append(a)
    assert X == 0
    return out


def split(Mat, exps, axis):
    """Digits D[r, k, p] of the rows (axis 0) or columns (axis 1) of Mat."""
    R = Mat.shape[axis]
    K = Mat.shape[1 - axis]
    D = np.zeros((R, K, NDIG), dtype=np.int64)
    for r in range(R):
        if exps[r] is None:
            continue
        for k in range(K):
            x = Mat[r, k] if axis == 0 else Mat[k, r]
            D[r, k] = balanced_digits(fixed(x, exps[r]))
    return D


def model_gemm(A, B):
    """The emulated product of A (M x K) and B (K x N), as the scheme forms it."""
    M, K = A.shape
    N = B.shape[1]
    E = [scale_exp(A[i]) for i in range(M)]
    F = [scale_exp(B[:, j]) for j in range(N)]
    DA = split(A, E, 0)             # M x K x 8
    DB = split(B, F, 1)             # N x K x 8
    acc = np.zeros((M, N), dtype=object)
    for c0 in range(0, K, CHUNK):
        ck = slice(c0, min(K, c0 + CHUNK))
        for d in range(2, 8):
            S = sum(DA[:, ck, p - 1] @ DB[:, ck, q - 1].T for p, q in PAIRS if p + q == d)
            # the FP32 tensor-memory slot of diagonal d holds S units of 2^-7d exactly
            assert np.max(np.abs(S)) < 2 ** 24
            acc = acc + S.astype(object) * (1 << (49 - 7 * d))
    shared = np.zeros((M, N), dtype=np.float32)
    for s0 in range(0, K, SLICE):
        sk = slice(s0, min(K, s0 + SLICE))
        for p, q in PAIRS:
            if p + q < 8:
                continue
            T = DA[:, sk, p - 1] @ DB[:, sk, q - 1].T  # one MMA: an exact integer below 2^17
            shared = (shared.astype(np.float64) + T * 2.0 ** (-7 * (p + q))).astype(np.float32)
    C = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            if E[i] is None or F[j] is None:
                continue
            s = float(int(acc[i, j])) * 2.0 ** -49 + float(shared[i, j])
            C[i, j] = math.ldexp(s, E[i] + F[j] + 2)
    return C, E, F


def exact_gemm(A, B):
    M, K = A.shape
    N = B.shape[1]
    Af = [[Fraction(float(x)) for x in row] for row in A]
    Bf = [[Fraction(float(B[k, j])) for k in range(K)] for j in range(N)]
    return [[sum(a * b for a, b in zip(Af[i], Bf[j])) for j in range(N)] for i in range(M)]


def scheme_bound(K, Ei, Fj):
    return K * 2.0 ** (Ei + Fj) * (2.0 ** -52.6 + 2.0 ** -53 + K * 2.0 ** -62.2)


def errors(A, B):
    C, E, F = model_gemm(A, B)
    X = exact_gemm(A, B)
    M, N = C.shape
    err = np.array([[abs(Fraction(C[i, j]) - X[i][j]) for j in range(N)] for i in range(M)], dtype=float)
    bound = np.array([[scheme_bound(A.shape[1], E[i], F[j]) for j in range(N)] for i in range(M)])
    absprod = np.abs(A) @ np.abs(B)
    return err, bound, absprod


def test_digits_are_balanced_and_exact_in_bf16():
    rng = np.random.default_rng(1)
    xs = list(rng.standard_normal(300) * 2.0 ** rng.integers(-30, 30, 300))
    xs += [1.0 - 2 ** -53, -(1.0 - 2 ** -53), 0.5, -0.5, 2 ** -1074, 1.5 * 2 ** -1000, 0.0]
    for x in xs:
        E = math.frexp(abs(x))[1] if x != 0 else 0
        X = fixed(x, E)
        assert abs(X) < 2 ** 55
        a = balanced_digits(X)
        assert all(abs(v) <= 64 for v in a)  # 7 bits: exact in BF16's 8-bit significand
        assert sum(v << (56 - 7 * p) for p, v in enumerate(a, 1)) == X
        # the truncation drops less than 2^-55 of the scale 2^E
        assert abs(Fraction(x) - Fraction(X) * Fraction(2) ** (E - 55)) < Fraction(2) ** (E - 55)


def test_accumulator_ranges():
    """Worst case |a_p| = |b_q| = 64: a diagonal d <= 7 of one 512-deep chunk stays below 2^24 (exact
    in FP32), and the 64-bit sum in units of 2^-49 over one launch's K stays below 2^63."""
    per_diag = {d: sum(1 for p, q in PAIRS if p + q == d) for d in range(2, 10)}
    assert len(PAIRS) == 36 and per_diag[8] == 7 and per_diag[9] == 8
    assert max(per_diag[d] for d in range(2, 8)) * CHUNK * 64 * 64 < 2 ** 24
    worst = sum(per_diag[d] * KMAX * 64 * 64 * 2 ** (49 - 7 * d) for d in range(2, 8))
    assert worst < 2 ** 63


@pytest.mark.parametrize("K", [1, 37, 1100])
def test_error_within_the_scheme_bound(K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((4, K))
    B = rng.standard_normal((K, 3))
    err, bound, _ = errors(A, B)
    assert np.all(err <= bound)


def test_small_integers_are_exact():
    rng = np.random.default_rng(3)
    A = rng.integers(-1000, 1000, (3, 200)).astype(float)
    B = rng.integers(-1000, 1000, (200, 4)).astype(float)
    err, _, _ = errors(A, B)
    assert np.all(err == 0)


def test_bound_is_relative_to_the_scales_not_to_the_entries():
    """Rows of A and columns of B whose entries span 2^-40 .. 1: the scheme's bound holds, while the
    error relative to (|A| |B|)_ij exceeds 2^-50 where the small entries meet the large ones."""
    rng = np.random.default_rng(7)
    K = 64
    A = rng.standard_normal((3, K)) * 2.0 ** -40
    B = rng.standard_normal((K, 3)) * 2.0 ** -40
    A[:, 0] = 1.0  # one large entry per row of A, in the column whose row of B is small ...
    B[1, :] = 1.0  # ... and one large entry per column of B, where A is small
    err, bound, absprod = errors(A, B)
    assert np.all(err <= bound)
    assert np.max(err / absprod) > 2.0 ** -50
