"""Pins of the oracle's DDM and Krylov layers.

* Transfer identity: A M^-1 v - v vanishes off the interface bands and equals
  the explicit transfer sum sum_{p != i} T_pi(z_i) on them (rows of A and
  A_p coincide on strip p's owned nodes).
* Algorithm 1 with explicit transfer operators equals Richardson iteration on
  M^-1 sweep by sweep, and converges to the global direct solution (the
  full-domain FDFD of the paper's comparison).
* One strip: M^-1 = A^-1, GMRES converges in one iteration, Algorithm 1 stops
  after the initial solve.
* GMRES: monotone residual, never above the Richardson residual after the
  same number of sweeps, finite termination on a small system, and the
  flexible variant's residual estimate equal to the true residual.
"""
import numpy as np
import pytest

import workloads as W
from oracle.fdfd import Problem
from oracle.krylov import gmres
from oracle.stddm import DDM, partition


@pytest.fixture(scope="module")
def cyl():
    w = W.cylinder()
    P = Problem.from_workload(w)
    D = DDM.from_workload(w, P)
    x = P.solve(w.b[0].ravel())
    return w, P, D, x


@pytest.fixture(scope="module")
def rnd4():
    w = W.random_medium(120, 48, ppw=16, seed=11, npml=8, nsub=4, overlap=3,
                        interface_pml=8, nsrc=2)
    P = Problem.from_workload(w)
    return w, P, DDM.from_workload(w, P)


def test_partition_covers_and_extends():
    st = partition(103, 4, 5, 10, 12, 9)
    assert [s.c1 - s.c0 for s in st] == [26, 26, 26, 25]
    assert st[0].c0 == 0 and st[-1].c1 == 103
    for a, b in zip(st, st[1:]):
        assert a.c1 == b.c0
    assert (st[0].x0, st[0].L_lo, st[0].L_hi) == (0, 12, 10)
    assert (st[1].x0, st[1].x1) == (26 - 15, 52 + 15)
    assert (st[-1].x1, st[-1].L_hi) == (103, 9)
    with pytest.raises(ValueError):
        partition(40, 4, 5, 10, 4, 4)       # extension wider than a strip


def test_local_rows_match_global_on_owned_nodes(rnd4):
    w, P, D = rnd4
    A = P.A.tocsr()
    for s in D.strips:
        Al = D.local_A(s.k).tocsr()
        for col in range(s.c0, s.c1):
            for j in (0, 7, 23, P.ny - 1):
                g = col * P.ny + j
                gl = (col - s.x0) * P.ny + j
                rg = A.getrow(g)
                rl = Al.getrow(gl)
                got = {c + s.x0 * P.ny: v for c, v in zip(rl.indices, rl.data)}
                want = dict(zip(rg.indices, rg.data))
                assert got.keys() == want.keys()
                for c in want:
                    assert got[c] == want[c]


def test_local_solve_residual(rnd4):
    w, P, D = rnd4
    rng = np.random.default_rng(3)
    for k in range(D.nsub):
        Al = D.local_A(k)
        t = rng.standard_normal(Al.shape[0]) + 1j * rng.standard_normal(Al.shape[0])
        z = D.local_solve(k, t)
        assert np.linalg.norm(Al @ z - t) / np.linalg.norm(t) <= 1e-13


def test_transfer_identity(rnd4):
    w, P, D = rnd4
    v = W.random_vector(P.n, seed=5)[0]
    z = D.local_solutions(v)
    d = P.A @ D.apply_Minv(v) - v
    ny = P.ny
    ext = D.overlap + D.interface_pml
    band = np.zeros(P.nx, bool)
    for s in D.strips[1:]:
        band[s.c0 - ext - 1:s.c0 + ext + 1] = True
    off = np.repeat(~band, ny)
    assert np.linalg.norm(d[off]) <= 1e-12 * np.linalg.norm(v)
    assert np.linalg.norm(d[~off]) > 1e-3 * np.linalg.norm(v)   # the bands carry the transfer
    tsum = np.zeros(P.n, complex)
    for p in range(D.nsub):
        tp = np.zeros(D.strips[p].width * ny, complex)
        for i in range(D.nsub):
            if i != p:
                tp += D.transfer(p, i, z[i])
        tsum += D.extend(p, tp)
    assert np.linalg.norm(d - tsum) <= 1e-12 * np.linalg.norm(v)


def test_algorithm1_equals_richardson_and_converges(cyl):
    w, P, D, x = cyl
    b = w.b[0].ravel()
    eg, hist = D.algorithm1(b, tol=1e-12, maxit=30)
    xs = D.richardson(b, len(hist))
    for n, (_, partial) in enumerate(hist):
        assert np.linalg.norm(xs[n] - partial) <= 1e-12 * np.linalg.norm(partial)
    assert hist[-1][0] < 1e-12
    fn = [h[0] for h in hist]
    assert all(b_ < a_ for a_, b_ in zip(fn, fn[1:]))       # overlap field decays
    assert np.linalg.norm(eg - x) / np.linalg.norm(x) <= 1e-10


def test_single_strip_is_the_direct_solve(cyl):
    w, P, _, x = cyl
    D1 = DDM(P, 1, 0, 0)
    b = w.b[0].ravel()
    assert np.linalg.norm(D1.apply_Minv(b) - x) <= 1e-13 * np.linalg.norm(x)
    xg, hist, its = gmres(P.matvec, D1.apply_Minv, b, restart=10, rtol=1e-12)
    assert its == 1
    assert np.linalg.norm(xg - x) / np.linalg.norm(x) <= 1e-12
    eg, h = D1.algorithm1(b, tol=1e-12, maxit=5)
    assert len(h) == 1 and h[0][0] == 0.0


def test_gmres_bounded_by_richardson_and_monotone(rnd4):
    w, P, D = rnd4
    b = w.b[0].ravel()
    nb = np.linalg.norm(b)
    xs = D.richardson(b, 6)
    rich = [np.linalg.norm(b - P.A @ xk) / nb for xk in xs]
    _, hist, its = gmres(P.matvec, D.apply_Minv, b, restart=50, rtol=1e-14, maxit=6)
    assert its == 6
    for k in range(6):
        assert hist[k + 1] <= rich[k] * (1 + 1e-9)
    assert all(b_ <= a_ * (1 + 1e-12) for a_, b_ in zip(hist, hist[1:]))


def test_gmres_converges_to_direct_solution(rnd4):
    w, P, D = rnd4
    for r in range(w.nrhs):
        b = w.b[r].ravel()
        x = P.solve(b)
        for flexible in (True, False):
            xg, hist, its = gmres(P.matvec, D.apply_Minv, b, restart=5, rtol=1e-11,
                                  flexible=flexible)
            assert np.linalg.norm(b - P.A @ xg) / np.linalg.norm(b) <= 1.5e-11
            assert np.linalg.norm(xg - x) / np.linalg.norm(x) <= 1e-8


def test_full_gmres_finite_termination():
    w = W.random_medium(6, 5, ppw=8, seed=4, npml=1)
    P = Problem.from_workload(w)
    b = w.b[0].ravel()
    xg, hist, its = gmres(P.matvec, lambda v: v, b, restart=P.n, rtol=1e-12)
    assert its <= P.n
    assert np.linalg.norm(xg - np.linalg.solve(P.A.toarray(), b)) <= 1e-9 * np.linalg.norm(xg)


def test_fgmres_estimate_is_true_residual_with_varying_preconditioner(rnd4):
    w, P, D = rnd4
    b = w.b[0].ravel()
    calls = []

    def varying(v):                 # alternate between M^-1 and 0.5 M^-1
        calls.append(1)
        return D.apply_Minv(v) * (1.0 if len(calls) % 2 else 0.5)

    xg, hist, its = gmres(P.matvec, varying, b, restart=40, rtol=1e-6, maxit=40)
    true = np.linalg.norm(b - P.A @ xg) / np.linalg.norm(b)
    assert true == pytest.approx(hist[-1], rel=1e-6, abs=1e-12)


def test_printed_sign_of_the_update_does_not_solve(cyl, monkeypatch):
    # with the "+" of Eqs. 18-19 taken literally the synthesis of Eq. 21
    # does not approach A^-1 b; the reading t_p = -sum T_pi does (above)
    w, P, D, x = cyl
    orig = DDM.transfer
    monkeypatch.setattr(DDM, "transfer", lambda self, p, i, e: -orig(self, p, i, e))
    eg, hist = D.algorithm1(w.b[0].ravel(), tol=1e-12, maxit=6)
    assert np.linalg.norm(eg - x) / np.linalg.norm(x) > 1e-2


def test_misplaced_interface_pml_breaks_row_agreement(rnd4, monkeypatch):
    # with no overlap band the interface half node is the one next to the
    # owned block; a PML profile one cell too deep stretches it, and the
    # owned rows of A_p then differ from A's (the transfer identity fails)
    w, P, _ = rnd4
    from oracle import stddm
    orig = stddm.stretch_profile
    monkeypatch.setattr(stddm, "stretch_profile",
                        lambda n, lo, hi, *a: orig(n, lo + 1 if lo else 0, hi, *a))
    D2 = DDM(P, 4, 0, 8)
    s = D2.strips[1]
    Al = D2.local_A(1).tocsr()
    A = P.A.tocsr()
    g = s.c0 * P.ny + 9
    gl = (s.c0 - s.x0) * P.ny + 9
    rl = Al.getrow(gl)
    got = {c + s.x0 * P.ny: v for c, v in zip(rl.indices, rl.data)}
    want = dict(zip(A.getrow(g).indices, A.getrow(g).data))
    assert any(abs(got.get(c, 0) - want[c]) > 1e-9 * abs(want[c]) for c in want)


def test_multiplicative_order_is_the_product_of_strip_projections():
    """I - M^-1 A of the symmetric multiplicative order equals the product
    (I - P_0)(I - P_1)..(I - P_{n-1})..(I - P_1)(I - P_0), applied right to
    left, with P_k = E_k A_k^-1 R_k^I A formed column by column."""
    w = W.random_medium(30, 14, ppw=20, seed=21, npml=4, nsub=3, overlap=2, interface_pml=4)
    prob = Problem.from_workload(w)
    ddm = DDM.from_workload(w, prob)
    n = prob.n
    A = prob.A.toarray()
    I = np.eye(n)
    P = []
    for k in range(ddm.nsub):
        Pk = np.zeros((n, n), complex)
        for c in range(n):
            Pk[:, c] = ddm.extend(k, ddm.local_solve(k, ddm.restrict_owned(k, A[:, c])))
        P.append(Pk)
    E = I.copy()
    for k in list(range(ddm.nsub)) + list(range(ddm.nsub - 2, -1, -1)):
        E = (I - P[k]) @ E
    MA = np.column_stack([ddm.apply_Minv_multiplicative(A[:, c]) for c in range(n)])
    assert np.abs((I - MA) - E).max() < 1e-9 * np.abs(E).max()


def test_multiplicative_one_strip_is_the_direct_solve():
    w = W.random_medium(24, 16, ppw=20, seed=22, npml=4, nsub=1, overlap=2, interface_pml=4)
    prob = Problem.from_workload(w)
    ddm = DDM.from_workload(w, prob)
    b = w.b[0].ravel()
    assert np.linalg.norm(ddm.apply_Minv_multiplicative(b) - prob.solve(b)) < 1e-10 * np.linalg.norm(prob.solve(b))


def test_multiplicative_order_converges_in_fewer_iterations():
    """FGMRES with the multiplicative order reaches the direct solution in
    fewer iterations than with the additive one on a 6-strip problem."""
    w = W.cylinder(nx=240, ny=60, ppw=20, npml=10, nsub=6, overlap=4, interface_pml=10, radius=0.4)
    prob = Problem.from_workload(w)
    ddm = DDM.from_workload(w, prob)
    b = w.b[0].ravel()
    ref = prob.solve(b)
    xa, ha, _ = gmres(lambda x: prob.A @ x, ddm.apply_Minv, b, restart=40, rtol=1e-10, maxit=200, flexible=True)
    xm, hm, _ = gmres(lambda x: prob.A @ x, ddm.apply_Minv_multiplicative, b, restart=40, rtol=1e-10, maxit=200,
                      flexible=True)
    assert np.linalg.norm(xm - ref) < 1e-7 * np.linalg.norm(ref)
    assert len(hm) < len(ha)


def test_red_black_groups_can_be_solved_together():
    """Same-colour strips do not interact: solving all even strips from one
    residual, then all odd ones, equals the sequential red-black order."""
    w = W.random_medium(90, 20, ppw=20, seed=23, npml=4, nsub=6, overlap=3, interface_pml=4)
    prob = Problem.from_workload(w)
    ddm = DDM.from_workload(w, prob)
    v = W.random_vector(prob.n, seed=24)[0]
    z = np.zeros(prob.n, complex)
    for colour in (0, 1):
        r = v - prob.A @ z
        z = z + sum(ddm.extend(k, ddm.local_solve(k, ddm.restrict_owned(k, r))) for k in range(colour, 6, 2))
    ref = ddm.apply_Minv_multiplicative(v, order="red-black")
    assert np.linalg.norm(z - ref) < 1e-12 * np.linalg.norm(ref)


def _band_columns(ddm, nx):
    """Interface bands: [c - e_l - 1, c + e_r + 1) around each interface c,
    e_r / e_l the columns the neighbouring local boxes reach past it."""
    cols = set()
    for k in range(ddm.nsub - 1):
        a, b = ddm.strips[k], ddm.strips[k + 1]
        c = a.c1
        cols.update(range(max(0, c - (c - b.x0) - 1), min(nx, c + (a.x1 - c) + 1)))
    return sorted(cols)


def test_band_space_system_gives_the_solution():
    """T = A M^-1 - I maps into the interface bands, and with r0 = b - A x0
    the band system (I + T_B) s = -(T r0)|_B gives x = x0 + M^-1 (r0 + s)
    with A x = b (dense, on a small 4-strip problem)."""
    w = W.random_medium(44, 10, ppw=20, seed=25, npml=3, nsub=4, overlap=2, interface_pml=3)
    prob = Problem.from_workload(w)
    ddm = DDM.from_workload(w, prob)
    n, ny = prob.n, prob.ny
    A = prob.A.toarray()
    cols = _band_columns(ddm, prob.nx)
    B = np.array([c * ny + j for c in cols for j in range(ny)])
    off = np.setdiff1d(np.arange(n), B)
    rng = np.random.default_rng(26)
    for _ in range(3):
        v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        Tv = A @ ddm.apply_Minv(v) - v
        assert np.abs(Tv[off]).max() < 1e-11 * np.abs(Tv).max()
    # the band system
    b = w.b[0].ravel()
    x0 = 1e-3 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    r0 = b - A @ x0
    TB = np.zeros((len(B), len(B)), complex)
    for i, bi in enumerate(B):
        e = np.zeros(n, complex)
        e[bi] = 1.0
        TB[:, i] = (A @ ddm.apply_Minv(e) - e)[B]
    f = -(A @ ddm.apply_Minv(r0) - r0)[B]
    sB = np.linalg.solve(np.eye(len(B)) + TB, f)
    s = np.zeros(n, complex)
    s[B] = sB
    x = x0 + ddm.apply_Minv(r0 + s)
    assert np.linalg.norm(A @ x - b) < 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - prob.solve(b)) < 1e-9 * np.linalg.norm(x)


def _sym_defect(A, d):
    """max |B - B^T| / max |B| for B = diag(d) A."""
    import scipy.sparse as sp
    B = (sp.diags(d) @ A).tocsr()
    return abs(B - B.T).max() / abs(B).max()


def test_local_operators_are_symmetric_after_stretch_scaling(rnd4):
    """Row u of every local operator times s_x s_y at u -- the box's own
    stretches, local interface PML included (Eqs. 10-13) -- is complex
    symmetric; the factorization may therefore work on D A_k with one
    triangle of each update.  The unscaled operator and the operator scaled
    by the half-node stretches are not symmetric, so the pin tells the node
    products from plausible other diagonals."""
    from oracle.checkerboard import CheckerboardDDM
    from oracle.fdfd import stretch_profile
    w, P, D = rnd4
    for k, s in enumerate(D.strips):
        A = D.local_A(k)
        sx, sxh = D.local_stretch_x(s)
        d = np.outer(sx, P.sy).ravel()
        assert _sym_defect(A, d) <= 1e-15
        assert _sym_defect(A, np.ones_like(d)) > 1e-3
        assert _sym_defect(A, np.outer(sxh[1:], P.syh[1:]).ravel()) > 1e-3
    C = CheckerboardDDM(P, 3, 2, 3, 8)
    for k, b in enumerate(C.boxes):
        sx, _ = stretch_profile(b.width, b.Lx_lo, b.Lx_hi, P.dx, P.k0, P.m, P.R)
        sy, _ = stretch_profile(b.height, b.Ly_lo, b.Ly_hi, P.dy, P.k0, P.m, P.R)
        assert _sym_defect(C.local_A(k), np.outer(sx, sy).ravel()) <= 1e-15
