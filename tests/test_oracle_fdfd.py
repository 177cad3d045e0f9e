"""Pins of the oracle's FDFD layer against closed forms and invariants.

Each check is something the mathematics fixes independently of the oracle's
code: the exact discrete 1-D solution, the 2-D Hankel Green's function
(second-order convergence), the Mie series of a dielectric cylinder,
reciprocity of the PML-stretched operator, and a dense solve on small grids.
The mutation tests plant plausible mistakes in the oracle (on the CPU) and
check that a pin catches each of them.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fdfd
from oracle.fdfd import Problem, sigma_hat_max, stretch_profile
from tests.analytic import discrete_line_source_1d, hankel_green, mie_plane_wave, mie_point_source

K0 = 2 * math.pi


def line_1d_error(L=20, n=400, ppw=20, axis="y", problem_cls=Problem):
    """Max error of a 1-D line-source solve against the exact discrete
    solution of the infinite line, on the non-PML part of the line.  The
    transverse step is made huge so the 2-D stencil reduces to 1-D."""
    h = 1.0 / ppw
    js = n // 2
    if axis == "y":
        P = problem_cls(1, n, 1e8, h, 1.0, np.ones((1, n)), npml=(0, 0, L, L))
    else:
        P = problem_cls(n, 1, h, 1e8, 1.0, np.ones((n, 1)), npml=(L, L, 0, 0))
    b = np.zeros(n, complex)
    b[js] = -1.0 / h
    u = P.solve(b)
    ex = discrete_line_source_1d(n, h, K0, js)
    inner = slice(L + 5, n - L - 5)
    return np.max(np.abs(u[inner] - ex[inner])) / np.max(np.abs(ex))


def test_sigma_max_sign_and_value():
    # Eq. 13 with the sign read so that sigma_max > 0; 20-cell PML at
    # lambda/20, m = 3, R = 1e-8: (m+1)(-ln R)/(2 k0 d) with d = 1 lambda.
    v = sigma_hat_max(20, 0.05, K0, 3, 1e-8)
    assert v > 0
    assert v == pytest.approx(4 * math.log(1e8) / (4 * math.pi), rel=1e-14)
    assert v == pytest.approx(5.86348, abs=1e-5)


def test_pml_profile_structure():
    s, sh = stretch_profile(60, 20, 10, 0.05, K0, 3, 1e-8)
    # interior nodes and the two interface half nodes are unstretched
    assert np.all(s[20:50] == 1.0)
    assert sh[20] == 1.0 and sh[50] == 1.0
    # sigma_max exactly at the outermost half nodes (Eq. 12 with u = L)
    assert sh[0].imag == pytest.approx(sigma_hat_max(20, 0.05, K0, 3, 1e-8), rel=1e-14)
    assert sh[60].imag == pytest.approx(sigma_hat_max(10, 0.05, K0, 3, 1e-8), rel=1e-14)
    # real part 1 everywhere, imaginary part monotone into the PML
    assert np.all(s.real == 1.0) and np.all(sh.real == 1.0)
    assert np.all(np.diff(sh.imag[:21]) < 0) and np.all(np.diff(sh.imag[50:]) > 0)
    assert np.all(np.diff(s.imag[:21]) < 0)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_exact_discrete_1d_line_source(axis):
    # the stencil, the source normalisation and PML absorption together
    err = line_1d_error(axis=axis)
    assert err < 2e-5          # measured 4.0e-6: residual PML reflection


def test_pml_reflection_falls_with_thickness():
    e10, e20, e30 = (line_1d_error(L=L) for L in (10, 20, 30))
    assert e10 > e20 > e30
    assert e30 < 2e-6


def _hankel_error(ppw, size=6.0, L=20):
    h = 1.0 / ppw
    n = int(round(size * ppw)) + 1 + 2 * L
    P = Problem(n, n, h, h, 1.0, np.ones((n, n)), npml=(L,) * 4)
    c = n // 2
    b = np.zeros((n, n), complex)
    b[c, c] = -1.0 / h ** 2
    u = P.solve(b.ravel()).reshape(n, n)
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r = np.hypot(I - c, J - c) * h
    m = (r >= 1.0) & (r <= 2.0)
    ex = hankel_green(K0, r[m])
    return np.linalg.norm(u[m] - ex) / np.linalg.norm(ex)


def test_free_space_green_second_order():
    e10, e20, e40 = _hankel_error(10), _hankel_error(20), _hankel_error(40)
    assert 3.5 < e10 / e20 < 4.6
    assert 3.5 < e20 / e40 < 4.6
    assert e40 < 0.012


def _mie_error(ppw, problem_cls=Problem):
    n = 10 * ppw
    w = W.cylinder(nx=n, ny=n, ppw=ppw, npml=20)
    P = problem_cls.from_workload(w)
    u = P.solve(w.b[0].ravel()).reshape(n, n)
    h = w.dx
    cx, cy = w.meta["center"]
    a = w.meta["radius"]
    si, sj = w.meta["src"]
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    X, Y = I * h, J * h
    r = np.hypot(X - cx, Y - cy)
    m = (r >= a + 0.25) & (r <= a + 2.5) & (np.hypot(X - si * h, Y - sj * h) >= 0.25)
    ex = mie_point_source(X[m], Y[m], cx, cy, a, 4.0, si * h, sj * h, K0)
    return np.linalg.norm(u[m] - ex) / np.linalg.norm(ex)


def test_mie_series_dielectric_cylinder():
    # the 200 x 200, lambda/20 cylinder case and its 2x refinement
    e20, e40 = _mie_error(20), _mie_error(40)
    assert e20 < 0.12          # measured 0.096
    assert e40 < 0.03          # measured 0.023
    assert e20 / e40 > 3.5     # second order: subcell averaging works


def _scattering_error(ppw, radius=0.5):
    n = 6 * ppw
    w = W.cylinder_scattering(n=n, ppw=ppw, radius=radius, npml=20, nsub=2)
    P = Problem.from_workload(w)
    u = P.solve(w.b[0].ravel()).reshape(n, n)
    h = w.dx
    cx, cy = w.meta["center"]
    a = w.meta["radius"]
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    X, Y = I * h, J * h
    r = np.hypot(X - cx, Y - cy)
    m = (r >= a + 0.25) & (r <= a + 1.5)
    ex = mie_plane_wave(X[m], Y[m], cx, cy, a, 4.0, K0)
    return np.linalg.norm(u[m] - ex) / np.linalg.norm(ex)


def test_plane_wave_scattering_matches_mie():
    # the paper's first example (Eq. 7 scattered-field source, eps 4 cylinder)
    # at r = lambda / 2 on a 6 x 6 lambda grid, and its 2x refinement
    e20, e40 = _scattering_error(20), _scattering_error(40)
    assert e20 < 0.2 and e40 < 0.05, (e20, e40)     # measured 0.168, 0.040
    assert e20 / e40 > 3.5, (e20, e40)              # second order


def test_plane_wave_source_is_zero_in_air():
    w = W.cylinder_scattering(n=120, ppw=20, radius=1.0, npml=20, nsub=2)
    air = np.isclose(w.eps_node, 1.0)
    assert air.any() and not np.abs(w.b[0][air]).any()
    assert np.abs(w.b[0][~air]).min() > 0


def _reciprocity_pair(problem_cls=Problem):
    w = W.random_medium(48, 40, ppw=20, seed=7, npml=10)
    P = problem_cls.from_workload(w)
    a = (14, 12)
    b = (31, 27)
    c = (3, 20)                 # inside the x0 PML
    n = P.n

    def src(node):
        v = np.zeros(n, complex)
        v[node[0] * P.ny + node[1]] = 1.0
        return v

    ua, ub, uc = P.solve(src(a)), P.solve(src(b)), P.solve(src(c))
    g = lambda u, node: u[node[0] * P.ny + node[1]]
    S = lambda node: P.sx[node[0]] * P.sy[node[1]]
    return (abs(g(ua, b) - g(ub, a)) / abs(g(ua, b)),
            abs(g(ua, c) / S(a) - g(uc, a) / S(c)) / abs(g(ua, c) / S(a)))


def test_reciprocity():
    # B = diag(sx sy) A is complex symmetric and A^-1 = B^-1 S, so the field
    # at c of a source at a obeys u_a(c)/S_a = u_c(a)/S_c; away
    # from the PML S = 1 and plain reciprocity G(a,b) = G(b,a) holds
    r_int, r_pml = _reciprocity_pair()
    assert r_int <= 1e-10
    assert r_pml <= 1e-10


def test_dense_solve_small_grids():
    for nx, ny, seed in ((10, 10, 1), (16, 12, 2), (32, 32, 3)):
        w = W.random_medium(nx, ny, ppw=8, seed=seed, npml=3)
        P = Problem.from_workload(w)
        b = w.b[0].ravel()
        x_dense = np.linalg.solve(P.A.toarray(), b)
        x = P.solve(b)
        assert np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense) <= 1e-12


def test_uniform_medium_generator():
    cells = W.cell_permittivity(10, 8, 0.1, 0.1, 3.0, [])
    assert np.all(W.node_permittivity(cells) == 3.0)
    # a half plane x <= 0.5 covers exactly half of the subcell centres of
    # the cells straddling x = 0.5 +- half a cell
    half = W.cell_permittivity(10, 8, 0.1, 0.1, 1.0, [(W._rect(-1, 0.45, -1, 2), 5.0)])
    assert half[5, 3] == pytest.approx(3.0, abs=1e-12)   # cell [0.4, 0.5]


# ---------------------------------------------------------------------------
# mutation tests: a plausible mistake planted in the oracle must fail a pin
# ---------------------------------------------------------------------------

def _mutant_problem(monkeypatch, assemble=None, stretch=None):
    if assemble is not None:
        monkeypatch.setattr(fdfd, "assemble", assemble)
    if stretch is not None:
        monkeypatch.setattr(fdfd, "stretch_profile", stretch)
    return Problem


def test_mutation_pml_sign_caught(monkeypatch):
    orig = fdfd.stretch_profile

    def wrong_sign(*a, **k):
        s, sh = orig(*a, **k)
        return np.conj(s), np.conj(sh)

    P = _mutant_problem(monkeypatch, stretch=wrong_sign)
    assert line_1d_error(problem_cls=P) > 1e-2


def test_mutation_half_node_shift_caught(monkeypatch):
    orig = fdfd.stretch_profile

    def shifted(n, *a, **k):
        s, sh = orig(n, *a, **k)
        return s, np.concatenate([sh[1:], sh[-1:]])

    P = _mutant_problem(monkeypatch, stretch=shifted)
    r_int, r_pml = _reciprocity_pair(P)
    assert max(r_int, r_pml) > 1e-6 or line_1d_error(problem_cls=P) > 2e-5


def test_mutation_dropped_eps_caught(monkeypatch):
    orig = fdfd.assemble

    def no_eps(nx, ny, dx, dy, k0, eps, *a):
        return orig(nx, ny, dx, dy, k0, np.ones_like(eps), *a)

    P = _mutant_problem(monkeypatch, assemble=no_eps)
    assert _mie_error(20, P) > 0.12


def test_mutation_transposed_coupling_caught(monkeypatch):
    orig = fdfd.assemble

    def swapped(nx, ny, dx, dy, k0, eps, sx, sxh, sy, syh):
        # couple (i-1) with sx_{i+1/2} and (i+1) with sx_{i-1/2}
        A = orig(nx, ny, dx, dy, k0, eps, sx, sxh, sy, syh)
        I = np.repeat(np.arange(nx), ny)
        J = np.tile(np.arange(ny), nx)
        A = A.tolil()
        for g, (i, j) in enumerate(zip(I, J)):
            if 0 < i < nx - 1:
                A[g, g - ny], A[g, g + ny] = A[g, g + ny], A[g, g - ny]
        return A.tocsr()

    P = _mutant_problem(monkeypatch, assemble=swapped)
    r_int, r_pml = _reciprocity_pair(P)
    assert max(r_int, r_pml) > 1e-6
