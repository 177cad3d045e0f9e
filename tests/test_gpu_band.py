"""Band-space FGMRES (STDD_OPT_BAND) on the GPU: the same solutions as the
standard FP64 iteration and the oracle's direct solve, the same iteration
counts (+-2: the band form fixes the coefficient of r0), user starts, several
right-hand sides, one strip, and the argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle.fdfd import Problem  # noqa: E402

DEV = "cuda:0"


def _solve(w, band, precision=0, order=0, x0=None, rtol=1e-12):
    from paper_2509_20801_gb300 import STDD_OPT_BAND, STDD_OPT_ORDER, Solver, stdd_set_option
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV), precision=precision)
    stdd_set_option(s.ctx, STDD_OPT_BAND, 1 if band else 0)
    stdd_set_option(s.ctx, STDD_OPT_ORDER, order)
    s.factor()
    b = torch.from_numpy(w.b).to(DEV)
    s.set_sources(b)
    x = torch.empty_like(b)
    try:
        s.solve(x, restart=40, rtol=rtol, maxit=400, x0=x0)
        hist = [s.history(q) for q in range(w.nrhs)]
    finally:
        s.close()
    return x.cpu().numpy(), hist


CASES = {
    "cylinder": lambda: W.cylinder(),
    "ragged4": lambda: W.random_medium(203, 77, ppw=16, seed=21, npml=8, nsub=4, overlap=5, interface_pml=9, nsrc=2),
    "strips6": lambda: W.cylinder(nx=240, ny=60, ppw=20, npml=10, nsub=6, overlap=4, interface_pml=10, radius=0.4),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_band_fgmres_matches_direct_and_standard(case):
    w = CASES[case]()
    P = Problem.from_workload(w)
    xb, hb = _solve(w, True)
    xs, hs = _solve(w, False)
    for q in range(w.nrhs):
        ref = P.solve(w.b[q].ravel())
        assert np.linalg.norm(xb[q].ravel() - ref) <= 1e-9 * np.linalg.norm(ref)
        assert abs(len(hb[q]) - len(hs[q])) <= 2, (len(hb[q]), len(hs[q]))
        assert hb[q][0] == pytest.approx(1.0) and hb[q][-1] <= 1e-12


def test_band_fgmres_with_user_start():
    w = CASES["ragged4"]()
    P = Problem.from_workload(w)
    rng = np.random.default_rng(3)
    x0 = torch.from_numpy((rng.standard_normal(w.b.shape) + 1j * rng.standard_normal(w.b.shape)) * 1e-2).to(DEV)
    xb, hb = _solve(w, True, x0=x0)
    for q in range(w.nrhs):
        ref = P.solve(w.b[q].ravel())
        assert np.linalg.norm(xb[q].ravel() - ref) <= 1e-9 * np.linalg.norm(ref)
        assert hb[q][0] > 1.0      # the start's own residual comes first


def test_band_mode_one_strip_is_the_direct_solve():
    w = W.random_medium(48, 40, ppw=20, seed=7, npml=6, nsub=1)
    P = Problem.from_workload(w)
    xb, hb = _solve(w, True)
    ref = P.solve(w.b[0].ravel())
    assert np.linalg.norm(xb[0].ravel() - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision,order", [(1, 0), (0, 1), (0, 2)])
def test_band_mode_needs_fp64_additive(precision, order):
    from paper_2509_20801_gb300 import StddError
    from paper_2509_20801_gb300 import binding as B
    with pytest.raises(StddError) as e:
        _solve(CASES["cylinder"](), True, precision=precision, order=order)
    assert e.value.status == B.STDD_EINVAL


def test_band_history_ends_with_the_true_residual():
    from paper_2509_20801_gb300 import STDD_OPT_BAND, Solver, stdd_residual, stdd_set_option
    w = CASES["ragged4"]()
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV))
    stdd_set_option(s.ctx, STDD_OPT_BAND, 1)
    s.factor()
    b = torch.from_numpy(w.b).to(DEV)
    s.set_sources(b)
    x = torch.empty_like(b)
    s.solve(x, restart=40, rtol=1e-10, maxit=400)
    for q in range(w.nrhs):
        r = torch.empty(w.n, dtype=torch.complex128, device=DEV)
        rel = stdd_residual(s.ctx, x[q].reshape(-1).contiguous(), b[q].reshape(-1).contiguous(), r)
        assert rel <= 1e-10
        assert s.history(q)[-1] == pytest.approx(rel, rel=1e-6)
    s.close()
