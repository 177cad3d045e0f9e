"""The exact-splitting product (Ozaki, Ogita, Oishi and Rump, Numer.
Algorithms 59, 2012) that the complex128 tensor-core update implements,
restated here in numpy integer arithmetic so that its error bound is pinned
on the CPU, independently of the kernel (the GPU tests compare the kernel
with numpy's own product).

Each real row of the 2 x 2 embedding of C and each complex column of R is
scaled by the power of two just above its largest |component| and cut into
eight 7-bit fixed-point slices; the products of slice orders 0..7 are
accumulated exactly (each order's sum stays below 2^23, the FP32
accumulator's exact range) and combined in 64-bit integers before one
rounding.  Pins: exact on integer operands; within 2 K 2^-53 of the row and
column scales on random operands over 24 decades (K = 2 kc real terms); the
order sums never reach 2^23; dropping an order or misplacing the scale breaks
the bound.
"""
from fractions import Fraction

import numpy as np
import pytest

S, BITS = 8, 7


def _row_exp(a):
    """e with |x| < 2^e over the last axis (frexp exponent), -2000 for zeros."""
    m = np.max(np.abs(a), axis=-1)
    e = np.frexp(m)[1]
    return np.where(m > 0, e, -2000)


def _slices(x, e):
    """x (float64, any shape) scaled by 2^-e (e broadcast) into S signed
    7-bit integer slices, most significant first: x = 2^e sum_i s_i 2^-7(i+1)
    up to the truncation below 2^-56."""
    m, E = np.frexp(np.abs(x))
    M = np.round(m * 2.0 ** 53).astype(np.int64)                    # exact: 53-bit mantissa
    sh = (e - E - 3).astype(np.int64)                                # Y = M 2^-sh
    Y = np.where(sh >= 0, M >> np.clip(sh, 0, 63), M << np.clip(-sh, 0, 3))
    Y = np.where((x == 0) | (sh >= 64), 0, Y)
    assert np.all(Y < 2 ** 56)
    sgn = np.where(x < 0, -1, 1).astype(np.int64)
    return [sgn * ((Y >> (49 - BITS * i)) & 127) for i in range(S)]


def split_product(C, R, orders=range(S), scale_shift=55):
    """C (m x kc) times R (kc x n), complex128, by exact splitting."""
    kc = C.shape[1]
    A = np.zeros((2 * C.shape[0], 2 * kc))              # real rows 2r = [Cr, -Ci], 2r+1 = [Ci, Cr]
    A[0::2, 0::2], A[0::2, 1::2] = C.real, -C.imag
    A[1::2, 0::2], A[1::2, 1::2] = C.imag, C.real
    B = np.zeros((R.shape[1], 2 * kc))                  # complex column c: [Rr, Ri] per pivot
    B[:, 0::2], B[:, 1::2] = R.T.real, R.T.imag
    eA = np.repeat(_row_exp(np.concatenate([C.real, C.imag], axis=1)), 2)
    eB = _row_exp(np.concatenate([R.T.real, R.T.imag], axis=1))
    As = _slices(A, eA[:, None])
    Bs = _slices(B, eB[:, None])
    G = [sum(As[i] @ Bs[g - i].T for i in range(g + 1)) for g in range(S)]   # exact int64 order sums
    for g in range(S):
        assert np.abs(G[g]).max(initial=0) < 2 ** 23      # exact in an FP32 accumulator
    G = [G[g] if g in orders else np.zeros_like(G[g]) for g in range(S)]
    hi = sum(G[g] * (1 << (BITS * (3 - g))) for g in range(4))
    lo = sum(G[g] * (1 << (BITS * (7 - g))) for g in range(4, 8))
    V = hi * (1 << 20) + (lo >> 8)
    assert np.abs(V).max(initial=0) < 2 ** 62
    D = V.astype(np.float64) * np.ldexp(1.0, (eA[:, None] + eB[None, :] - scale_shift))
    return D[0::2] + 1j * D[1::2], eA[0::2], eB


def _exact(C, R, i, j):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(
        np.concatenate([C[i].real, -C[i].imag]), np.concatenate([R[:, j].real, R[:, j].imag]))), \
        sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(
            np.concatenate([C[i].real, C[i].imag]), np.concatenate([R[:, j].imag, R[:, j].real])))


def test_integer_operands_are_exact():
    rng = np.random.default_rng(1)
    C = rng.integers(-1000, 1000, (64, 32)) + 1j * rng.integers(-1000, 1000, (64, 32))
    R = rng.integers(-1000, 1000, (32, 64)) + 1j * rng.integers(-1000, 1000, (32, 64))
    D, _, _ = split_product(C, R)
    assert np.array_equal(D, C @ R)
    C2 = np.full((64, 32), 127.0 * (1 + 1j))            # every slice at 127 in the first order
    D2, _, _ = split_product(C2, C2.T.copy())
    assert np.array_equal(D2, C2 @ C2.T)


@pytest.mark.parametrize("kc,spread", [(32, 0), (7, 6), (1, 3), (32, 12)])
def test_error_bound_against_exact_products(kc, spread):
    rng = np.random.default_rng(kc + spread)
    C = (rng.standard_normal((16, kc)) + 1j * rng.standard_normal((16, kc))) * 10.0 ** rng.uniform(-spread, spread, (16, 1))
    R = (rng.standard_normal((kc, 16)) + 1j * rng.standard_normal((kc, 16))) * 10.0 ** rng.uniform(-spread, spread, (1, 16))
    D, eA, eB = split_product(C, R)
    for i in range(0, 16, 3):
        for j in range(0, 16, 5):
            re, im = _exact(C, R, i, j)
            bound = Fraction(2 * 2 * kc) * Fraction(2) ** -53 * Fraction(2) ** int(eA[i] + eB[j])
            assert abs(Fraction(float(D[i, j].real)) - re) <= bound
            assert abs(Fraction(float(D[i, j].imag)) - im) <= bound


def test_planted_mistakes_break_the_bound():
    """Dropping order 4, or taking the scale one binade off, is caught."""
    rng = np.random.default_rng(9)
    C = rng.standard_normal((8, 32)) + 1j * rng.standard_normal((8, 32))
    R = rng.standard_normal((32, 8)) + 1j * rng.standard_normal((32, 8))
    ref = C @ R
    good, eA, eB = split_product(C, R)
    scale = np.ldexp(1.0, eA[:, None] + eB[None, :])
    tol = 4 * 64 * 2.0 ** -53 * scale
    assert np.all(np.abs(good - ref) <= tol)
    dropped, _, _ = split_product(C, R, orders=[0, 1, 2, 3, 5, 6, 7])
    assert np.any(np.abs(dropped - ref) > tol)
    shifted, _, _ = split_product(C, R, scale_shift=54)
    assert np.any(np.abs(shifted - ref) > tol)
