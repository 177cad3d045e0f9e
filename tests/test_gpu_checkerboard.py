"""Two-dimensional (checkerboard) partitions on the GPU against the oracle's
box construction (oracle/checkerboard.py): box extents, every box's local
solve (SuperLU of the oracle's local operator, 1e-10), M^-1 summed over boxes
(1e-10), FGMRES to the direct solution (1e-9; complex64 factors 1e-7), one box
row reproducing the strip path bitwise, and the refusals of what needs strips.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle.checkerboard import CheckerboardDDM  # noqa: E402
from oracle.fdfd import Problem  # noqa: E402

DEV = "cuda:0"


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def cyl240():
    w = W.cylinder(nx=240, ny=240, overlap=8, interface_pml=20)
    return w, Problem.from_workload(w)


@pytest.fixture(scope="module")
def ragged():
    # ragged in both axes, different PML widths on the four sides
    w = W.random_medium(97, 83, ppw=16, seed=31, npml=8, nsub=3, overlap=4, interface_pml=8, nsrc=1)
    P = Problem(w.nx, w.ny, w.dx, w.dy, w.wavelength, w.eps_node, npml=(8, 7, 9, 6))
    return w, P


def _boxes_solver(w, P, px, py, overlap, ipml, precision=0, x_cuts=None, y_cuts=None):
    from paper_2509_20801_gb300 import Solver, stdd_set_decomposition_2d
    s = Solver(w.nx, w.ny, w.dx, w.dy, w.wavelength, torch.from_numpy(P.eps).to(DEV), npml=P.npml,
               pml_order=P.m, pml_R=P.R, nsub=1, overlap=overlap, interface_pml=ipml,
               precision=precision)
    stdd_set_decomposition_2d(s.ctx, px, py, overlap, ipml, x_cuts, y_cuts)
    return s


@pytest.mark.parametrize("case,px,py,ov,ip", [("cyl", 2, 2, 8, 20), ("cyl", 3, 3, 8, 20), ("rag", 3, 2, 4, 5)])
def test_boxes_match_oracle(case, px, py, ov, ip, cyl240, ragged):
    from paper_2509_20801_gb300 import stdd_apply_preconditioner, stdd_box_info, stdd_local_solve
    w, P = {"cyl": cyl240, "rag": ragged}[case]
    D = CheckerboardDDM(P, px, py, ov, ip)
    s = _boxes_solver(w, P, px, py, ov, ip)
    s.factor()
    for k, b in enumerate(D.boxes):
        info = stdd_box_info(s.ctx, k)
        assert (info["c0"], info["c1"], info["r0"], info["r1"]) == (b.c0, b.c1, b.r0, b.r1)
        assert (info["x0"], info["x1"], info["y0"], info["y1"]) == (b.x0, b.x1, b.y0, b.y1)
        t = W.random_vector(b.width * b.height, seed=40 + k)[0]
        z = torch.empty(b.width * b.height, dtype=torch.complex128, device=DEV)
        stdd_local_solve(s.ctx, k, torch.from_numpy(t).to(DEV), z)
        assert _rel(z.cpu().numpy(), D.local_solve(k, t)) < 1e-10, k
    v = W.random_vector(P.n, seed=11)[0]
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    stdd_apply_preconditioner(s.ctx, torch.from_numpy(v).to(DEV), z)
    assert _rel(z.cpu().numpy(), D.apply_Minv(v)) < 1e-10
    # FGMRES with the box preconditioner reaches the direct solution
    b = w.b[:1].copy()
    s.set_sources(torch.from_numpy(b).to(DEV))
    x = torch.empty(b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, restart=40, rtol=1e-12, maxit=400)
    assert _rel(x[0].cpu().numpy().ravel(), P.solve(b[0].ravel())) <= 1e-9
    s.close()


def test_boxes_with_explicit_cuts_and_complex64(ragged):
    from paper_2509_20801_gb300 import STDD_PREC_C64, stdd_apply_preconditioner
    w, P = ragged
    xc, yc = [0, 30, 70, 97], [0, 45, 83]
    D = CheckerboardDDM(P, 3, 2, 4, 5)
    # the oracle with the same cuts: rebuild its boxes from explicit parts
    from oracle.checkerboard import Box
    from oracle.stddm import Strip

    def parts(cuts, n, lo, hi, ext=9, ipml=5):
        out = []
        for k in range(len(cuts) - 1):
            c0, c1 = cuts[k], cuts[k + 1]
            x0 = c0 - ext if k > 0 else 0
            x1 = c1 + ext if k < len(cuts) - 2 else n
            out.append(Strip(k, c0, c1, x0, x1, ipml if k > 0 else lo, ipml if k < len(cuts) - 2 else hi))
        return out
    D.boxes = [Box(sx, sy) for sx in parts(xc, P.nx, 8, 7) for sy in parts(yc, P.ny, 9, 6)]
    s = _boxes_solver(w, P, 3, 2, 4, 5, x_cuts=xc, y_cuts=yc)
    s.factor()
    v = W.random_vector(P.n, seed=12)[0]
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    stdd_apply_preconditioner(s.ctx, torch.from_numpy(v).to(DEV), z)
    assert _rel(z.cpu().numpy(), D.apply_Minv(v)) < 1e-10
    s.close()
    s = _boxes_solver(w, P, 3, 2, 4, 5, precision=STDD_PREC_C64, x_cuts=xc, y_cuts=yc)
    s.factor()
    b = w.b[:1].copy()
    s.set_sources(torch.from_numpy(b).to(DEV))
    x = torch.empty(b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, restart=40, rtol=1e-10, maxit=400)
    got = x[0].cpu().numpy().ravel()
    assert np.linalg.norm(b[0].ravel() - P.A @ got) / np.linalg.norm(b[0]) <= 1.5e-10
    assert _rel(got, P.solve(b[0].ravel())) <= 1e-7
    s.close()


def test_one_box_row_is_the_strip_path(cyl240):
    """py = 1 through the 2-D entry point gives the strips' results bitwise."""
    from paper_2509_20801_gb300 import Solver, stdd_apply_preconditioner
    w, P = cyl240
    v = torch.from_numpy(W.random_vector(P.n, seed=13)[0]).to(DEV)
    outs = []
    for two_d in (False, True):
        if two_d:
            s = _boxes_solver(w, P, 3, 1, 8, 20)
        else:
            s = Solver(w.nx, w.ny, w.dx, w.dy, w.wavelength, torch.from_numpy(P.eps).to(DEV), npml=P.npml,
                       pml_order=P.m, pml_R=P.R, nsub=3, overlap=8, interface_pml=20)
        s.factor()
        z = torch.empty_like(v)
        stdd_apply_preconditioner(s.ctx, v, z)
        outs.append(z.cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_boxes_refuse_strip_only_features(cyl240):
    from paper_2509_20801_gb300 import (STDD_OPT_BAND, STDD_OPT_ORDER, StddError, stdd_apply_preconditioner,
                                        stdd_set_decomposition_2d, stdd_set_option)
    w, P = cyl240
    s = _boxes_solver(w, P, 2, 2, 8, 20)
    s.factor()
    v = torch.from_numpy(W.random_vector(P.n, seed=14)[0]).to(DEV)
    z = torch.empty_like(v)
    stdd_set_option(s.ctx, STDD_OPT_ORDER, 1)
    with pytest.raises(StddError) as e:
        stdd_apply_preconditioner(s.ctx, v, z)
    assert e.value.status == 1 and "strip" in str(e.value)
    stdd_set_option(s.ctx, STDD_OPT_ORDER, 0)
    # the refusal came while the application's graph was being captured: the
    # stream must be usable again, and the next application correct
    stdd_apply_preconditioner(s.ctx, v, z)
    D = CheckerboardDDM(P, 2, 2, 8, 20)
    assert _rel(z.cpu().numpy(), D.apply_Minv(v.cpu().numpy())) < 1e-10
    stdd_set_option(s.ctx, STDD_OPT_BAND, 1)
    s.set_sources(torch.from_numpy(w.b[:1].copy()).to(DEV))
    x = torch.empty(w.b[:1].shape, dtype=torch.complex128, device=DEV)
    with pytest.raises(StddError) as e:
        s.solve(x, restart=20, rtol=1e-8, maxit=50)
    assert e.value.status == 1
    with pytest.raises(StddError) as e:      # boxes narrower than overlap + interface PML
        stdd_set_decomposition_2d(s.ctx, 2, 12, 8, 20)
    assert e.value.status == 1
    s.close()
