"""Tensor-core (tcgen05) front updates of the mixed-precision path.

The tile self-test multiplies one 64 x 32 by 32 x 128 complex tile with BF16
or FP16 inputs and FP32 accumulation and compares with a double-precision
host product; the bound is the input rounding (2^-8 for BF16, 2^-11 for FP16,
relative to the largest entry, times the growth of a 64-term real sum).  The
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


@pytest.mark.parametrize("fmt,bound", [(1, 3e-2), (0, 5e-3)])
def test_tile_product_matches_host(fmt, bound):
    from paper_2509_20801_gb300 import stdd_tc_selftest
    err = stdd_tc_selftest(0, fmt)
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
