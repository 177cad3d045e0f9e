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
