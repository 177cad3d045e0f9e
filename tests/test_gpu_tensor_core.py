"""Tensor-core (tcgen05) front updates of the mixed-precision path.

One tile (64 x kc by kc x 128 complex, BF16 or FP16 inputs, FP32
accumulation) is compared with products computed in the test with numpy:
the product of the scaled and rounded operands, and the unrounded product.  The
solves check that with these updates the FP64 Krylov iteration still reaches
its residual and the field matches the oracle's direct solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle.fdfd import Problem  # noqa: E402

DEV = "cuda:0"


def _rounded(a, e, fmt):
    """a * 2^e rounded to FP16 (fmt 0) / BF16 (fmt 1) by torch, as float64."""
    t = torch.from_numpy(np.ldexp(a.astype(np.float32), e).astype(np.float32))
    return t.to(torch.float16 if fmt == 0 else torch.bfloat16).to(torch.float64).numpy()


def _scale_exp(a):
    """e with the largest |component| of a, times 2^e, in [1, 2)."""
    m = float(np.max(np.abs(np.concatenate([a.real.ravel(), a.imag.ravel()]).astype(np.float32))))
    return 0 if m == 0 else 1 - int(np.frexp(m)[1])


@pytest.mark.parametrize("fmt,bound", [(1, 3e-2), (0, 5e-3)])
@pytest.mark.parametrize("kc,cs,rs", [(32, 1.0, 1.0), (7, 1e-3, 1e6), (1, 3.0, 1e-5)])
def test_tile_product_matches_numpy(fmt, bound, kc, cs, rs):
    """One tensor-core tile D = C R (64 x kc by kc x 128 complex) against
    products computed here: (i) the float64 product of the operands after the
    documented power-of-two scaling and FP16 / BF16 rounding (torch's
    conversions), which the FP32 accumulation of 2 kc real products may miss
    only by its own rounding; (ii) the unrounded float64 product, within the
    input rounding (2^-8 BF16, 2^-11 FP16, relative to the largest entry,
    times the growth of the sum).  Ranges far from 1 (1e-3 x 1e6) exercise the
    scaling, without which FP16 would overflow."""
    from paper_2509_20801_gb300 import stdd_tc_tile_product
    rng = np.random.default_rng(40 + kc)
    C = (rng.standard_normal((64, kc)) + 1j * rng.standard_normal((64, kc))) * cs
    R = (rng.standard_normal((kc, 128)) + 1j * rng.standard_normal((kc, 128))) * rs
    D = stdd_tc_tile_product(C, R, fmt=fmt)
    C32 = C.astype(np.complex64).astype(np.complex128)
    R32 = R.astype(np.complex64).astype(np.complex128)
    ea, eb = _scale_exp(C32), _scale_exp(R32)
    Cr, Ci = _rounded(C32.real, ea, fmt), _rounded(C32.imag, ea, fmt)
    Rr, Ri = _rounded(R32.real, eb, fmt), _rounded(R32.imag, eb, fmt)
    exact_r = (Cr @ Rr - Ci @ Ri) * 2.0 ** -(ea + eb)
    exact_i = (Cr @ Ri + Ci @ Rr) * 2.0 ** -(ea + eb)
    # sums of the magnitudes of the terms of each component
    mag_r = (np.abs(Cr) @ np.abs(Rr) + np.abs(Ci) @ np.abs(Ri)) * 2.0 ** -(ea + eb)
    mag_i = (np.abs(Cr) @ np.abs(Ri) + np.abs(Ci) @ np.abs(Rr)) * 2.0 ** -(ea + eb)
    # FP32 accumulation inside the tensor core: the products of FP16 / BF16
    # operands are exact, their sum may be aligned and truncated rather than
    # rounded, a few units of 2^-23 per term and per instruction; far below
    # the operand rounding (2^-9 / 2^-12), so a wrong scaling, embedding or
    # rounding of the operands still fails
    gam = 2 * (2 * kc + 8) * 2.0 ** -24
    ratio = max(float(np.max(np.abs(D.real - exact_r) / mag_r)), float(np.max(np.abs(D.imag - exact_i) / mag_i)))
    assert ratio <= gam, f"accumulation error {ratio:.3e} of the term magnitudes > {gam:.3e}"
    ref = C32 @ R32
    err = np.abs(D - ref).max() / np.abs(ref).max()
    assert 0.0 < err < bound


@pytest.mark.parametrize("mode", ["bf16", "fp16"])
def test_solve_with_tensor_core_updates(mode):
    from paper_2509_20801_gb300 import STDD_PREC_C64_BF16, STDD_PREC_C64_FP16, Solver
    prec = STDD_PREC_C64_BF16 if mode == "bf16" else STDD_PREC_C64_FP16
    w = W.cylinder()
    P = Problem.from_workload(w)
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV), precision=prec)
    s.factor()
    s.set_sources(torch.from_numpy(w.b).to(DEV))
    x = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, restart=30, rtol=1e-10, maxit=300)
    got = x[0].cpu().numpy().ravel()
    b = w.b[0].ravel()
    assert np.linalg.norm(b - P.A @ got) / np.linalg.norm(b) <= 1.5e-10
    ref = P.solve(b)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-7
    s.close()


# ---------------------------------------------------------------- complex128
# The exact-splitting path of the complex128 update (STDD_OPT_FP64_TC):
# eight 7-bit BF16 slices per value, scaled per real row of the embedded C
# and per complex column of R; the expected values are computed here.

def _row_col_scales(C, R):
    """2^e per complex row of C and per complex column of R, |x| < 2^e over
    both components (frexp exponents)."""
    def e(v):
        m = np.max(np.abs(np.concatenate([v.real, v.imag], axis=-1)), axis=-1)
        return np.where(m > 0, np.frexp(m)[1], -1074).astype(np.float64)
    return np.ldexp(1.0, e(C).astype(int)), np.ldexp(1.0, e(R.T).astype(int))


def test_f64_tile_product_exact_on_integers():
    """Integer entries (products and sums exact in binary64): the split
    product loses nothing, so D equals the exact product bitwise."""
    from paper_2509_20801_gb300 import stdd_tc_f64_tile_product
    rng = np.random.default_rng(5)
    C = rng.integers(-1000, 1000, (64, 32)) + 1j * rng.integers(-1000, 1000, (64, 32))
    R = rng.integers(-1000, 1000, (32, 64)) + 1j * rng.integers(-1000, 1000, (32, 64))
    D = stdd_tc_f64_tile_product(C, R)
    assert np.array_equal(D, C @ R)
    # the largest slice values in every position: all group sums at their bound
    C2 = np.full((64, 32), 127.0 * (1 + 1j))
    D2 = stdd_tc_f64_tile_product(C2, C2.T.copy())
    assert np.array_equal(D2, C2 @ C2.T)


@pytest.mark.parametrize("kc,spread", [(32, 0), (7, 6), (1, 3), (32, 12)])
def test_f64_tile_product_error_bound(kc, spread):
    """Random operands whose rows and columns span 10^+-spread: every entry of
    D within 4 (2 kc) 2^-53 sC_i sR_j of the float64 product (sC, sR the row
    and column power-of-two scales; the split product's bound and float64's
    own rounding each contribute at most half of it), and the relative
    Frobenius error at the level of float64, far below BF16 (2^-8)."""
    from paper_2509_20801_gb300 import stdd_tc_f64_tile_product
    rng = np.random.default_rng(6 + kc + spread)
    C = (rng.standard_normal((64, kc)) + 1j * rng.standard_normal((64, kc))) * 10.0 ** rng.uniform(-spread, spread, (64, 1))
    R = (rng.standard_normal((kc, 64)) + 1j * rng.standard_normal((kc, 64))) * 10.0 ** rng.uniform(-spread, spread, (1, 64))
    D = stdd_tc_f64_tile_product(C, R)
    ref = C @ R
    sC, sR = _row_col_scales(C, R)
    bound = 4 * (2 * kc) * 2.0 ** -53 * np.outer(sC, sR)
    assert np.all(np.abs(D - ref) <= bound)
    if spread == 0:
        assert np.linalg.norm(D - ref) <= 1e-14 * np.linalg.norm(ref)


def test_f64_tile_product_refuses_nonfinite_input():
    from paper_2509_20801_gb300 import StddError, stdd_tc_f64_tile_product
    C = np.ones((64, 4), complex)
    C[3, 2] = np.inf
    with pytest.raises(StddError) as e:
        stdd_tc_f64_tile_product(C, np.ones((4, 64), complex))
    assert e.value.status == 1
