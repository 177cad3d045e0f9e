"""Pins of the checkerboard (2-D) partition oracle: owned blocks tile the
grid, one box row is the strip method, one box is the direct solve, local
rows equal global rows on owned nodes, the construction is symmetric under
transposing the problem, and FGMRES preconditioned by it reaches the direct
solution."""
import numpy as np
import pytest

import workloads as W
from oracle.checkerboard import CheckerboardDDM
from oracle.fdfd import Problem
from oracle.krylov import gmres
from oracle.stddm import DDM


@pytest.fixture(scope="module")
def prob():
    # ragged in both axes, different PML widths on each side
    w = W.random_medium(97, 83, ppw=16, seed=31, npml=8, nsub=3, overlap=4, interface_pml=8, nsrc=1)
    return w, Problem(w.nx, w.ny, w.dx, w.dy, w.wavelength, w.eps_node, npml=(8, 7, 9, 6))


def test_owned_blocks_tile_the_grid(prob):
    _, P = prob
    D = CheckerboardDDM(P, 3, 2, 4, 5)
    seen = np.zeros((P.nx, P.ny), int)
    for b in D.boxes:
        seen[b.c0:b.c1, b.r0:b.r1] += 1
        # interior sides: 4 overlap + 5 local PML nodes; domain sides: the
        # global PML widths (8, 7) in x and (9, 6) in y
        assert b.x0 == (b.c0 - 9 if b.kx > 0 else 0) and b.x1 == (b.c1 + 9 if b.kx < 2 else P.nx)
        assert b.y0 == (b.r0 - 9 if b.ky > 0 else 0) and b.y1 == (b.r1 + 9 if b.ky < 1 else P.ny)
        assert (b.Lx_lo, b.Lx_hi) == (5 if b.kx > 0 else 8, 5 if b.kx < 2 else 7)
        assert (b.Ly_lo, b.Ly_hi) == (5 if b.ky > 0 else 9, 5 if b.ky < 1 else 6)
    assert np.all(seen == 1)


def test_one_box_row_is_the_strip_method(prob):
    _, P = prob
    v = W.random_vector(P.n, seed=4)[0]
    got = CheckerboardDDM(P, 3, 1, 4, 8).apply_Minv(v)
    ref = DDM(P, 3, 4, 8).apply_Minv(v)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_one_box_is_the_direct_solve(prob):
    _, P = prob
    v = W.random_vector(P.n, seed=5)[0]
    got = CheckerboardDDM(P, 1, 1, 4, 8).apply_Minv(v)
    ref = P.solve(v)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


def test_local_rows_match_global_on_owned_nodes(prob):
    _, P = prob
    D = CheckerboardDDM(P, 2, 3, 4, 8)
    A = P.A.tocsr()
    for k, b in enumerate(D.boxes):
        Al = D.local_A(k).tocsr()
        H = b.height
        for i in (b.c0, (b.c0 + b.c1) // 2, b.c1 - 1):
            for j in (b.r0, (b.r0 + b.r1) // 2, b.r1 - 1):
                rg = A.getrow(i * P.ny + j)
                rl = Al.getrow((i - b.x0) * H + (j - b.y0))
                got = {(c // H + b.x0) * P.ny + (c % H + b.y0): v for c, v in zip(rl.indices, rl.data)}
                want = dict(zip(rg.indices, rg.data))
                # the global row's neighbours inside the local box, same values
                assert set(got) <= set(want)
                for c, val in got.items():
                    assert val == pytest.approx(want[c], rel=1e-14, abs=0)
                assert len(got) == len(want)      # owned nodes are never on the local box's edge


def test_transposed_problem_gives_the_transposed_preconditioner(prob):
    """Swap x and y everywhere (grid, permittivity, PML widths, boxes): the
    preconditioner is the transposed one, exactly up to rounding."""
    w, P = prob
    PT = Problem(w.ny, w.nx, w.dy, w.dx, w.wavelength, w.eps_node.T.copy(), npml=(9, 6, 8, 7))
    v = W.random_vector(P.n, seed=6)[0]
    vT = v.reshape(P.nx, P.ny).T.ravel()
    z = CheckerboardDDM(P, 3, 2, 4, 8).apply_Minv(v)
    zT = CheckerboardDDM(PT, 2, 3, 4, 8).apply_Minv(vT)
    assert np.linalg.norm(zT.reshape(P.ny, P.nx).T.ravel() - z) <= 1e-12 * np.linalg.norm(z)


@pytest.mark.parametrize("px,py", [(2, 2), (3, 2)])
def test_fgmres_with_boxes_reaches_the_direct_solution(prob, px, py):
    w, P = prob
    b = w.b[0].ravel()
    D = CheckerboardDDM(P, px, py, 4, 8)
    x, hist, its = gmres(P.matvec, D.apply_Minv, b, restart=40, rtol=1e-11, maxit=400)
    ref = P.solve(b)
    assert hist[-1] <= 1e-11
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    # more boxes, more iterations than the direct solve's one
    assert its > 1
