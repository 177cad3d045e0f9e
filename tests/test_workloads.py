"""The waveguide-network input generator: its mode solver against the
symmetric-slab dispersion relation (a closed form, and the second-order
convergence of the discrete eigenvalue), its geometry (branch counts and core
widths where the layout fixes them), and the mode it launches, propagated by
the oracle's own 2-D solve with the phase velocity the 1-D eigenvalue
predicts."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import workloads as W
from oracle.fdfd import Problem

N_CORE, N_CLAD = math.sqrt(12.1), math.sqrt(2.085)


def slab_beta(width, wavelength=1.0):
    """Fundamental (even) mode of a symmetric slab with E parallel to the
    faces: kappa tan(kappa w / 2) = gamma, kappa^2 = k0^2 n1^2 - beta^2,
    gamma^2 = beta^2 - k0^2 n2^2 (E and dE/dy continuous at the faces)."""
    k0 = 2 * math.pi / wavelength

    def f(beta):
        kap = math.sqrt(k0 ** 2 * N_CORE ** 2 - beta ** 2)
        gam = math.sqrt(beta ** 2 - k0 ** 2 * N_CLAD ** 2)
        return kap * math.tan(kap * width / 2) - gam

    # the fundamental branch has kappa w / 2 in (0, pi / 2)
    lo = math.sqrt(max(k0 ** 2 * N_CORE ** 2 - (math.pi / width) ** 2, k0 ** 2 * N_CLAD ** 2)) + 1e-9
    return brentq(f, lo, k0 * N_CORE - 1e-9)


def cross_section(ppw, width=0.45, span=6.0, shift=0.37):
    """Node permittivity across a core of the given width, centred `shift`
    cells off a node, from the generator's own subcell averaging."""
    d = 1.0 / ppw
    ny = int(round(span / d)) + 1
    yc = 0.5 * span + shift * d
    cells = W.cell_permittivity(3, ny, d, d, N_CLAD ** 2,
                                [(W._rect(-1.0, 1.0, yc - width / 2, yc + width / 2), N_CORE ** 2)])
    return W.node_permittivity(cells)[1], d, yc


def test_slab_mode_converges_to_the_dispersion_relation():
    # faces on cell edges at every step (width 0.5 = 24, 48, 96 cells), so
    # the averaged permittivity is the face's arithmetic mean on the face
    # node and the discrete eigenvalue converges at second order
    exact = slab_beta(0.5)
    errs = []
    for ppw in (48, 96, 192):
        eps, d, _ = cross_section(ppw, width=0.5, shift=0.0)
        beta, phi = W.slab_mode(eps, d, 1.0)
        errs.append(beta - exact)
    # second order: the error falls about fourfold per halving of the step
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, (errs, r1, r2)
    assert abs(errs[2]) < 2e-4 * exact
    # Richardson extrapolation of the two finest steps lands on the root
    assert abs((4 * errs[2] - errs[1]) / 3) < 2e-5 * exact
    # faces off the grid (the generator's case): first-order smearing, still
    # within 2e-3 at lambda/48 and 2e-4 at lambda/96 of the root for w = 0.45
    exact = slab_beta(0.45)
    for ppw, tol in ((48, 2e-3), (96, 2e-4)):
        eps, d, _ = cross_section(ppw)
        assert abs(W.slab_mode(eps, d, 1.0)[0] - exact) < tol * exact


def test_slab_mode_is_the_fundamental_one():
    eps, d, yc = cross_section(24)
    beta, phi = W.slab_mode(eps, d, 1.0)
    y = np.arange(eps.size) * d
    assert phi.max() == pytest.approx(1.0) and phi.min() > -1e-12      # no node: the fundamental mode
    assert abs(y[np.argmax(phi)] - yc) <= d                             # peak on the core
    far = np.abs(y - yc) > 2.0
    assert np.abs(phi[far]).max() < 1e-6                                # guided: decayed in the cladding
    assert N_CLAD < beta / (2 * math.pi) < N_CORE


def test_waveguide_network_layout():
    w = W.waveguide_network(1024, 512, nsub=4)
    w2 = W.waveguide_network(1024, 512, nsub=4)
    assert np.array_equal(w.eps_node, w2.eps_node) and np.array_equal(w.b, w2.b)
    mid = 0.5 * (12.1 + 2.085)
    d = w.dx
    xs = w.meta["x_stages"]

    def runs(i):
        m = w.eps_node[i] > mid
        starts = np.flatnonzero(m[1:] & ~m[:-1]) + 1
        ends = np.flatnonzero(m[:-1] & ~m[1:]) + 1
        return len(starts), ends - starts

    # columns where every branch runs straight: before splitter 1, after the
    # splitter-2 bends, after the last splitter's bends, before the right PML
    cols = {1: int(0.5 * xs[0] / d), 4: int((xs[2] - 2 * d) / d), 5: w.nx - w.npml[1] - 2}
    for count, i in cols.items():
        n, widths = runs(i)
        assert n == count, (count, i, n)
        # a 0.45 lambda core covers 10 or 11 nodes above the midpoint at lambda/24
        assert np.all((widths >= 10) & (widths <= 11)), widths
    assert w.meta["splitters"] == 4 and w.meta["sbends"] == 8 and w.meta["branches"] == 5
    assert w.eps_node.min() == pytest.approx(2.085) and w.eps_node.max() == pytest.approx(12.1)
    # the source is the fundamental mode of its own column
    i = w.meta["i_src"]
    _, phi = W.slab_mode(w.eps_node[i], d, 1.0)
    assert np.abs(w.b[0, i] + phi / d).max() == 0.0
    assert np.count_nonzero(w.b[0]) == np.count_nonzero(phi)


def test_mode_propagates_with_the_predicted_phase_velocity():
    """A straight guide lit by the generator's mode source, solved by the
    oracle: beyond the source the field along the core keeps its amplitude
    (a guided, lossless mode) and advances in phase by beta_2d per unit
    length, where beta_2d is the propagation constant the 2-D stencil gives
    the 1-D eigenvalue: (2 - 2 cos(beta_2d dx)) / dx^2 = beta^2."""
    ppw, nx, ny, npml = 24, 360, 120, 24
    d = 1.0 / ppw
    yc = 0.5 * (ny - 1) * d
    cells = W.cell_permittivity(nx, ny, d, d, 2.085, [(W._rect(-1.0, nx * d + 1.0, yc - 0.225, yc + 0.225), 12.1)])
    eps = W.node_permittivity(cells)
    i_src = npml + 12
    beta, phi = W.slab_mode(eps[i_src], d, 1.0)
    b = np.zeros((1, nx, ny), complex)
    b[0, i_src] = -phi / d
    w = W.Workload("guide", nx, ny, d, d, 1.0, eps, b, npml=(npml,) * 4)
    u = Problem.from_workload(w).solve(b[0].ravel()).reshape(nx, ny)
    jc = int(round(yc / d))
    i1, i2 = i_src + 40, nx - npml - 30
    a1, a2 = u[i1, jc], u[i2, jc]
    assert abs(abs(a2) / abs(a1) - 1) < 2e-2
    beta2d = 2 / d * math.asin(beta * d / 2)
    dphase = np.angle(a2 / a1)
    want = (beta2d * (i2 - i1) * d + math.pi) % (2 * math.pi) - math.pi
    assert abs(dphase - want) < 2e-2
    # the profile across the guide is the mode's
    prof = u[i2] / u[i2, jc]
    assert np.linalg.norm(prof - phi / phi[jc]) < 3e-2 * np.linalg.norm(phi / phi[jc])


@pytest.mark.parametrize("shape,seed", [((512, 512), 3_000_000), ((1024, 512), 3_000_007), ((256, 256), 3_000_011)])
def test_ellipse_geometry_properties(shape, seed):
    """The batched / learned geometries: fill fraction drawn from [15 %, 30 %]
    of the non-PML area (the area painted, measured on the node grid, is close
    to the ellipses' summed area), permittivity only in {1} u [2, 12.1], vacuum
    within half a wavelength of the PML, strips in [2, min(8, nx / 128)] and
    every source at least half a wavelength inside the PML."""
    nx, ny = shape
    w = W.ellipses(nx, ny, seed=seed, nrhs=8, sources="mixed")
    npml, d = w.npml[0], w.dx
    area = ((nx - 1 - 2 * npml) * d) * ((ny - 1 - 2 * npml) * d)
    fill = w.meta["fill"]
    assert w.meta["n_ellipses"] >= 1
    assert fill <= 0.30 + 1e-12
    # the drawn target is at least 15 %; the loop stops once it is reached, or
    # after 400 attempts on small grids where big ellipses no longer fit
    painted = (w.eps_node > 1.0 + 1e-12).sum() * d * d / area
    assert abs(painted - fill) < 0.25 * fill + 0.01
    e = w.eps_node
    assert e.min() == pytest.approx(1.0) and e.max() <= 12.1 + 1e-12
    keep = int(np.ceil(0.5 / d))
    margin = npml + keep - 2          # subcell averaging reaches one cell past the edge
    core = np.zeros_like(e, bool)
    core[margin:nx - margin, margin:ny - margin] = True
    assert np.all(np.abs(e[~core] - 1.0) < 1e-12)
    assert 2 <= w.nsub <= max(2, min(8, nx // 128))
    for q in range(w.nrhs):
        nz = np.argwhere(w.b[q] != 0)
        if w.meta["sources"][q] == "point":
            assert len(nz) == 1
            i, j = nz[0]
            assert npml + keep <= i <= nx - 1 - npml - keep and npml + keep <= j <= ny - 1 - npml - keep
        else:
            js = set(nz[:, 1])
            assert len(js) == 1 and len(nz) == nx
            j = js.pop()
            assert npml + keep <= j <= ny - 1 - npml - keep


def test_metalens_structure():
    """The metalens workload as stated: substrate eps 2.085 on the lower 20 %
    of the rows, pillars of eps 12.1, 14 cells high (0.6 lambda at lambda/24),
    at a 0.5 lambda period with widths in [0.1, 0.4] lambda, and the line
    source 10 rows above the bottom PML."""
    w = W.metalens()
    d, npml = w.dx, w.npml[0]
    j_sub = w.meta["j_substrate"]
    assert j_sub == round(0.2 * w.ny)
    e = w.eps_node
    assert np.allclose(e[:, 5:j_sub - 2], 2.085)           # substrate rows (away from the top interface)
    # pillar rows: count the eps 12.1 runs along a row in the middle of the pillars
    row = e[:, j_sub + 7]
    m = row > 0.5 * (12.1 + 1.0)
    starts = np.flatnonzero(m[1:] & ~m[:-1]) + 1
    ends = np.flatnonzero(m[:-1] & ~m[1:]) + 1
    assert len(starts) == w.meta["n_pillars"]
    widths = (ends - starts) * d
    assert widths.min() >= 0.1 - 2 * d and widths.max() <= 0.4 + 2 * d
    period = np.diff(0.5 * (starts + ends)) * d
    assert np.allclose(period, 0.5, atol=2 * d)
    # pillar height: 14 rows above the substrate, vacuum further up
    col = e[int(0.5 * (starts[0] + ends[0])), :]
    assert np.all(col[j_sub + 1:j_sub + 13] > 6.0) and np.all(np.abs(col[j_sub + 16:w.ny - npml] - 1.0) < 1e-12)
    nz = np.argwhere(w.b[0] != 0)
    assert set(nz[:, 1]) == {npml + 10} and len(nz) == w.nx


def _mutated_mode(eps_line, dy, mutation):
    """slab_mode with one planted mistake (test-local copy of the eigenproblem)."""
    from scipy.linalg import eigh_tridiagonal
    k0 = 2 * math.pi
    n = eps_line.size
    diag = (-1.0 if mutation == "half-diagonal" else -2.0) / dy ** 2 + \
        (-1.0 if mutation == "k0-sign" else 1.0) * k0 ** 2 * eps_line
    off = np.full(n - 1, 1.0 / dy ** 2)
    pick = n - 2 if mutation == "second-mode" else n - 1
    val, vec = eigh_tridiagonal(diag, off, select="i", select_range=(pick, pick))
    phi = vec[:, 0] / vec[np.argmax(np.abs(vec[:, 0])), 0]
    return math.sqrt(abs(val[0])), phi


@pytest.mark.parametrize("mutation", ["half-diagonal", "second-mode", "k0-sign"])
def test_mode_pins_catch_planted_mistakes(mutation):
    """Each planted mistake in the mode eigenproblem fails a pin above: the
    dispersion relation (within 2e-3 at lambda/48 for an off-grid core) or the
    fundamental mode's shape (no sign change, peak on the core)."""
    eps, d, yc = cross_section(48)
    exact = slab_beta(0.45)
    beta, phi = _mutated_mode(eps, d, mutation)
    y = np.arange(eps.size) * d
    dispersion_ok = abs(beta - exact) < 2e-3 * exact
    shape_ok = phi.min() > -1e-12 and abs(y[np.argmax(phi)] - yc) <= d
    assert not (dispersion_ok and shape_ok)
    # the unmutated solver passes both
    b0, p0 = W.slab_mode(eps, d, 1.0)
    assert abs(b0 - exact) < 2e-3 * exact and p0.min() > -1e-12
