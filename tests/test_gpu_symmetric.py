"""The symmetric form (STDD_OPT_SYMMETRIC): fronts of D A_k, D the local
stretch products, lower-triangle front updates mirrored with the working
matrix's sign pattern.  Against the oracle: every strip's and box's local
solve and M^-1 (1e-10, FP64 factors), the FGMRES solution (1e-9); complex64
factors reach the FP64 residual; 64 x 64 and 32 x 32 tiles give bitwise equal
factors; the executed update work is about half of the full form's; with
pivoting on the option has no effect (row interchanges break the symmetry).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle.checkerboard import CheckerboardDDM  # noqa: E402
from oracle.fdfd import Problem  # noqa: E402
from oracle.stddm import DDM  # noqa: E402

DEV = "cuda:0"


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _solver(w, sym, precision=0, leaf=None, tile=None, pivoting=0, fp64_tc=0):
    from paper_2509_20801_gb300 import (STDD_OPT_FP64_TC, STDD_OPT_LEAF, STDD_OPT_PIVOTING, STDD_OPT_SYMMETRIC,
                                        STDD_OPT_UPDATE_TILE, Solver, stdd_set_option)
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV), precision=precision)
    stdd_set_option(s.ctx, STDD_OPT_SYMMETRIC, sym)
    stdd_set_option(s.ctx, STDD_OPT_FP64_TC, fp64_tc)
    if leaf is not None:
        stdd_set_option(s.ctx, STDD_OPT_LEAF, leaf)
    if tile is not None:
        stdd_set_option(s.ctx, STDD_OPT_UPDATE_TILE, tile)
    if pivoting:
        stdd_set_option(s.ctx, STDD_OPT_PIVOTING, 1)
    return s


@pytest.fixture(scope="module")
def rnd():
    w = W.random_medium(203, 77, ppw=16, seed=21, npml=8, nsub=4, overlap=5, interface_pml=9, nsrc=2)
    P = Problem.from_workload(w)
    return w, P, DDM.from_workload(w, P)


@pytest.fixture(scope="module")
def cyl():
    w = W.cylinder()
    P = Problem.from_workload(w)
    return w, P, DDM.from_workload(w, P)


@pytest.mark.parametrize("fp64_tc", [0, 1])
@pytest.mark.parametrize("which,leaf", [("rnd", None), ("cyl", None), ("cyl", 64)])
def test_symmetric_local_solves_and_preconditioner_match_oracle(which, leaf, fp64_tc, rnd, cyl):
    """fp64_tc = 1: the large-front updates on the tensor cores by exact
    splitting, to the same FP64 bars."""
    from paper_2509_20801_gb300 import stdd_apply_preconditioner, stdd_local_solve
    w, P, D = {"rnd": rnd, "cyl": cyl}[which]
    s = _solver(w, 1, leaf=leaf, fp64_tc=fp64_tc)
    s.factor()
    for k, st in enumerate(D.strips):
        t = W.random_vector(st.width * P.ny, seed=50 + k)[0]
        z = torch.empty(st.width * P.ny, dtype=torch.complex128, device=DEV)
        stdd_local_solve(s.ctx, k, torch.from_numpy(t).to(DEV), z)
        assert _rel(z.cpu().numpy(), D.local_solve(k, t)) < 1e-10, k
    v_h = W.random_vector(P.n, seed=51)[0]
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    stdd_apply_preconditioner(s.ctx, torch.from_numpy(v_h).to(DEV), z)
    assert _rel(z.cpu().numpy(), D.apply_Minv(v_h)) < 1e-10
    # the whole solve reaches the direct solution
    b = w.b[:1].copy()
    s.set_sources(torch.from_numpy(b).to(DEV))
    x = torch.empty(b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, restart=40, rtol=1e-12, maxit=400)
    assert _rel(x[0].cpu().numpy().ravel(), P.solve(b[0].ravel())) <= 1e-9
    s.close()


def test_symmetric_boxes_match_oracle():
    """Checkerboard boxes: each box's own y stretches enter D."""
    from paper_2509_20801_gb300 import (STDD_OPT_SYMMETRIC, Solver, stdd_apply_preconditioner,
                                        stdd_set_decomposition_2d, stdd_set_option)
    w = W.random_medium(97, 83, ppw=16, seed=31, npml=8, nsub=3, overlap=4, interface_pml=8, nsrc=1)
    P = Problem(w.nx, w.ny, w.dx, w.dy, w.wavelength, w.eps_node, npml=(8, 7, 9, 6))
    s = Solver(w.nx, w.ny, w.dx, w.dy, w.wavelength, torch.from_numpy(P.eps).to(DEV), npml=P.npml,
               pml_order=P.m, pml_R=P.R, nsub=1, overlap=4, interface_pml=5)
    stdd_set_decomposition_2d(s.ctx, 3, 2, 4, 5)
    stdd_set_option(s.ctx, STDD_OPT_SYMMETRIC, 1)
    s.factor()
    C = CheckerboardDDM(P, 3, 2, 4, 5)
    v_h = W.random_vector(P.n, seed=52)[0]
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    stdd_apply_preconditioner(s.ctx, torch.from_numpy(v_h).to(DEV), z)
    assert _rel(z.cpu().numpy(), C.apply_Minv(v_h)) < 1e-10
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_symmetric_tile_shapes_bitwise_and_half_the_update_work(cyl, precision):
    from paper_2509_20801_gb300 import stdd_apply_preconditioner, stdd_get_profile, stdd_set_profiling
    w, P, D = cyl
    v = torch.from_numpy(W.random_vector(P.n, seed=53)[0]).to(DEV)
    outs, work = [], {}
    on = 1 if precision == 0 else 2     # complex64 factors take the form only when asked (value 2)
    for sym, tile in ((on, 64), (on, 32), (on, 0), (0, 64)):
        s = _solver(w, sym, precision=precision, leaf=64, tile=tile)
        stdd_set_profiling(s.ctx, 2)
        s.factor()
        prof = stdd_get_profile(s.ctx, 1)
        work[(1 if sym else 0, tile)] = prof["update_flops_executed"]
        z = torch.empty_like(v)
        stdd_apply_preconditioner(s.ctx, v, z)
        outs.append(z.cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    # one triangle with its diagonal: just over half of the full update
    ratio = work[(1, 64)] / work[(0, 64)]
    assert 0.5 < ratio < 0.56, ratio
    if precision == 0:
        ref = D.apply_Minv(v.cpu().numpy())
        assert _rel(outs[0], ref) < 1e-10 and _rel(outs[3], ref) < 1e-10
        assert not np.array_equal(outs[0], outs[3])          # different factors, same operator


def test_symmetric_complex64_reaches_fp64_residual(cyl):
    """Complex64 factors in the symmetric form (value 2; value 1 keeps it to
    complex128 factors) still carry the FP64 iteration to its residual."""
    w, P, _ = cyl
    s = _solver(w, 2, precision=1)
    s.factor()
    b = w.b[:1].copy()
    s.set_sources(torch.from_numpy(b).to(DEV))
    x = torch.empty(b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, restart=40, rtol=1e-10, maxit=400)
    got = x[0].cpu().numpy().ravel()
    assert np.linalg.norm(b[0].ravel() - P.A @ got) / np.linalg.norm(b[0]) <= 1.5e-10
    s.close()


def test_symmetric_option_inactive_with_pivoting(rnd):
    from paper_2509_20801_gb300 import stdd_apply_preconditioner
    w, P, D = rnd
    v = torch.from_numpy(W.random_vector(P.n, seed=54)[0]).to(DEV)
    outs = []
    for sym in (0, 1):
        s = _solver(w, sym, pivoting=1)
        s.factor()
        z = torch.empty_like(v)
        stdd_apply_preconditioner(s.ctx, v, z)
        outs.append(z.cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    assert _rel(outs[0], D.apply_Minv(v.cpu().numpy())) < 1e-10


def test_symmetric_toggle_refactors_through_the_graph(rnd):
    """The factorization graph is keyed by the launch arguments: switching
    the option between factorizations gives each form's own factors."""
    from paper_2509_20801_gb300 import STDD_OPT_SYMMETRIC, StddError, stdd_apply_preconditioner, stdd_set_option
    w, P, D = rnd
    v = torch.from_numpy(W.random_vector(P.n, seed=55)[0]).to(DEV)
    s = _solver(w, 1)
    ref = {}
    for sym in (1, 0, 1, 0):
        stdd_set_option(s.ctx, STDD_OPT_SYMMETRIC, sym)
        s.factor()
        z = torch.empty_like(v)
        stdd_apply_preconditioner(s.ctx, v, z)
        if sym in ref:
            assert np.array_equal(ref[sym], z.cpu().numpy())
        ref[sym] = z.cpu().numpy()
        assert _rel(ref[sym], D.apply_Minv(v.cpu().numpy())) < 1e-10
    with pytest.raises(StddError) as e:
        stdd_set_option(s.ctx, STDD_OPT_SYMMETRIC, 3)
    assert e.value.status == 1
    s.close()


def test_fp64_tensor_core_update_runs_and_is_deterministic(cyl):
    """With STDD_OPT_FP64_TC the profile's executed update work is the BF16
    tensor-core count (36 slice products per tile, far above the FP64
    count); repeated factorizations are bitwise equal; M^-1 matches the
    FP64-pipe factors to the FP64 bar."""
    from paper_2509_20801_gb300 import stdd_apply_preconditioner, stdd_get_profile, stdd_set_profiling
    w, P, D = cyl
    v = torch.from_numpy(W.random_vector(P.n, seed=56)[0]).to(DEV)
    outs, work = {}, {}
    for tc in (1, 1, 0):
        s = _solver(w, 1, leaf=64, fp64_tc=tc)
        stdd_set_profiling(s.ctx, 2)
        s.factor()
        prof = stdd_get_profile(s.ctx, 1)
        work[tc] = (prof["update_flops"], prof["update_flops_executed"])
        z = torch.empty_like(v)
        stdd_apply_preconditioner(s.ctx, v, z)
        if tc in outs:
            assert np.array_equal(outs[tc], z.cpu().numpy())
        outs[tc] = z.cpu().numpy()
        s.close()
    assert work[1][0] == work[0][0]                      # same LDL^T units
    assert work[1][1] > 10 * work[0][1]                  # tensor-core slice products executed
    assert _rel(outs[1], outs[0]) < 1e-11
    assert _rel(outs[1], D.apply_Minv(v.cpu().numpy())) < 1e-10
