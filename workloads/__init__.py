"""Seeded synthetic inputs: node permittivity maps and source vectors.

This module is shared by the CPU oracle (``oracle/``) and by the GPU library's
tests and benchmark. It holds no arithmetic of the method itself (no stencil,
no PML, no decomposition, no solver): it only turns a geometry description and
a seed into the two arrays the solver consumes,

* ``eps_node``: real (nx, ny) array, node-averaged relative permittivity.
  Cells are the squares between nodes; each cell gets the subcell-averaged
  permittivity of Eq. 8 (8 x 8 subcells, a subcell belongs to the medium that
  contains its centre) and each node the mean of the four cells that touch it
  (Eq. 3).  Cells just outside the grid are evaluated from the same geometry.
* ``b``: complex (nx, ny) right-hand side.  A unit point source at node s is
  b_s = -1/(dx*dy), so that the discrete field approximates (i/4) H0^(1)(k r)
  with the e^{-i w t} time convention; an x-directed line source on row js is
  b_{i,js} = -1/dy for every column i.

Arrays are indexed [i, j] with i along x and j along y, so their C-order
flattening is the solver's node index g = i*ny + j.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SUBCELLS = 8


@dataclasses.dataclass
class Workload:
    """One synthetic FDFD problem (grid, materials, sources, decomposition)."""

    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    wavelength: float
    eps_node: np.ndarray            # (nx, ny) float64
    b: np.ndarray                   # (nrhs, nx, ny) complex128
    npml: tuple = (20, 20, 20, 20)  # x0, x1, y0, y1 cells
    pml_order: int = 3
    pml_R: float = 1e-8
    nsub: int = 2
    overlap: int = 8
    interface_pml: int = 20
    restart: int = 30
    rtol: float = 1e-10
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def nrhs(self) -> int:
        return self.b.shape[0]


# --------------------------------------------------------------------------
# geometry primitives: each returns a boolean "inside" test on point arrays
# --------------------------------------------------------------------------

def _circle(cx, cy, r):
    return (lambda x, y: (x - cx) ** 2 + (y - cy) ** 2 <= r * r,
            (cx - r, cx + r, cy - r, cy + r))


def _rect(xa, xb, ya, yb):
    return (lambda x, y: (x >= xa) & (x <= xb) & (y >= ya) & (y <= yb),
            (xa, xb, ya, yb))


def _ellipse(cx, cy, a, b, theta):
    ct, st = math.cos(theta), math.sin(theta)

    def inside(x, y):
        u = (x - cx) * ct + (y - cy) * st
        v = -(x - cx) * st + (y - cy) * ct
        return (u / a) ** 2 + (v / b) ** 2 <= 1.0

    r = max(a, b)
    return inside, (cx - r, cx + r, cy - r, cy + r)


def cell_permittivity(nx, ny, dx, dy, background, objects):
    """Subcell-averaged permittivity of the cells (i, j), i in [-1, nx-1],
    j in [-1, ny-1]; cell (i, j) spans [i dx, (i+1) dx] x [j dy, (j+1) dy].

    ``objects`` is a list of ((inside, bbox), eps); later objects are painted
    over earlier ones (they are not expected to overlap except on purpose,
    e.g. a pillar standing on a substrate)."""
    cells = np.full((nx + 1, ny + 1), float(background))
    off = (np.arange(SUBCELLS) + 0.5) / SUBCELLS
    for (inside, bbox), eps in objects:
        xa, xb, ya, yb = bbox
        i0 = max(-1, int(math.floor(xa / dx)) - 1)
        i1 = min(nx - 1, int(math.ceil(xb / dx)) + 1)
        j0 = max(-1, int(math.floor(ya / dy)) - 1)
        j1 = min(ny - 1, int(math.ceil(yb / dy)) + 1)
        if i1 < i0 or j1 < j0:
            continue
        ii = np.arange(i0, i1 + 1)
        jj = np.arange(j0, j1 + 1)
        # subcell centres of every cell in the bounding box, chunked by rows
        for c0 in range(0, len(ii), 256):
            isub = ii[c0:c0 + 256]
            xs = (isub[:, None] + off[None, :]) * dx           # (ci, S)
            ys = (jj[:, None] + off[None, :]) * dy             # (cj, S)
            X = xs[:, None, :, None]
            Y = ys[None, :, None, :]
            inn = inside(X, Y)                                 # (ci, cj, S, S)
            n_in = inn.reshape(len(isub), len(jj), -1).sum(axis=2)
            frac = n_in / float(SUBCELLS * SUBCELLS)
            blk = cells[isub[0] + 1:isub[-1] + 2, j0 + 1:j1 + 2]
            blk[...] = eps * frac + blk * (1.0 - frac)
    return cells


def node_permittivity(cells):
    """Mean of the four cells touching each node (Eq. 3)."""
    return 0.25 * (cells[:-1, :-1] + cells[1:, :-1] + cells[:-1, 1:] + cells[1:, 1:])


def point_source(nx, ny, dx, dy, i, j):
    b = np.zeros((nx, ny), np.complex128)
    b[i, j] = -1.0 / (dx * dy)
    return b


def line_source_x(nx, ny, dy, j):
    b = np.zeros((nx, ny), np.complex128)
    b[:, j] = -1.0 / dy
    return b


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def cylinder(nx=200, ny=200, ppw=20, eps_cyl=4.0, radius=0.5, src_gap=1.0,
             npml=20, nsub=2, overlap=8, interface_pml=20, wavelength=1.0):
    """Dielectric cylinder at the grid centre lit by a unit point source
    ``src_gap`` wavelengths left of its surface (the small plain-method case:
    200 x 200 nodes at lambda/20, eps 4, r = 0.5 lambda, 20-cell PML,
    2 strips with 8-cell overlap and 20-cell interface PML)."""
    d = wavelength / ppw
    cx, cy = (nx - 1) * d / 2.0, (ny - 1) * d / 2.0
    objs = []
    if eps_cyl != 1.0 and radius > 0:
        objs.append((_circle(cx, cy, radius * wavelength), eps_cyl))
    cells = cell_permittivity(nx, ny, d, d, 1.0, objs)
    eps = node_permittivity(cells)
    xs = cx - (radius + src_gap) * wavelength
    si = int(round(xs / d))
    sj = int(round(cy / d))
    b = point_source(nx, ny, d, d, si, sj)[None]
    return Workload("cylinder", nx, ny, d, d, wavelength, eps, b,
                    npml=(npml,) * 4, nsub=nsub, overlap=overlap,
                    interface_pml=interface_pml, restart=30, rtol=1e-10,
                    meta=dict(center=(cx, cy), radius=radius * wavelength,
                              eps_cyl=eps_cyl, src=(si, sj)))


def plane_wave_source(eps_node, dx, dy, wavelength, angle=0.0):
    """Scattered-field source of a plane wave in air (Eq. 7):
    b = -k0^2 (eps - 1) E_inc at every node, E_inc = exp(i k0 (x cos a +
    y sin a)) with node (i, j) at (i dx, j dy).  Zero wherever eps = 1, so the
    scatterer must stay out of the PML."""
    k0 = 2 * math.pi / wavelength
    nx, ny = eps_node.shape
    x = np.arange(nx)[:, None] * dx
    y = np.arange(ny)[None, :] * dy
    einc = np.exp(1j * k0 * (x * math.cos(angle) + y * math.sin(angle)))
    return -(k0 ** 2) * (eps_node - 1.0) * einc


def cylinder_scattering(n=6000, ppw=40, radius=9.0, eps_cyl=4.0, npml=20, nsub=64, overlap=8,
                        interface_pml=20, wavelength=1.0, restart=30, rtol=1e-8):
    """The paper's first example: plane-wave (along +x) scattering by a
    dielectric cylinder of radius ``radius`` wavelengths, eps 4, at the centre
    of an n x n grid at lambda/ppw, solved for the scattered field (Eq. 7).
    The default 6000 x 6000 grid at 40 points per wavelength is the paper's
    ~36 million unknowns; PML 20 cells, overlap 8, interface PML 20 cells."""
    d = wavelength / ppw
    cx = cy = (n - 1) * d / 2.0
    if radius * wavelength > cx - (npml + 1) * d:
        raise ValueError("cylinder reaches the PML")
    cells = cell_permittivity(n, n, d, d, 1.0, [(_circle(cx, cy, radius * wavelength), eps_cyl)])
    eps = node_permittivity(cells)
    b = plane_wave_source(eps, d, d, wavelength)[None]
    return Workload("cylinder-scattering", n, n, d, d, wavelength, eps, b,
                    npml=(npml,) * 4, nsub=nsub, overlap=overlap, interface_pml=interface_pml,
                    restart=restart, rtol=rtol,
                    meta=dict(center=(cx, cy), radius=radius * wavelength, eps_cyl=eps_cyl))


def metalens(nx=4096, ny=1024, ppw=24, seed=1, npml=30, nsub=16, overlap=12,
             interface_pml=30, wavelength=1.0, nrhs=1):
    """Metalens-like strip: substrate eps 2.085 over the lower 20 % of the
    rows, a row of eps 12.1 pillars (period 0.5 lambda, height 0.6 lambda
    rounded to whole cells, seeded widths U[0.1, 0.4] lambda) standing on it,
    and an x-directed line source inside the substrate 10 cells above the
    bottom PML (the plain-FP64 metalens case is 4096 x 1024 at lambda/24,
    30-cell PML, 16 strips, 12-cell overlap).  With nrhs > 1 the extra
    right-hand sides are line sources on the next rows, 3 cells apart."""
    rng = np.random.default_rng(seed)
    d = wavelength / ppw
    j_sub = int(round(0.2 * ny))
    y_sub = j_sub * d
    height = round(0.6 * ppw) * d
    period = 0.5 * wavelength
    objs = [(_rect(-2 * d, (nx + 1) * d, -2 * d, y_sub), 2.085)]
    x_lo, x_hi = npml * d, (nx - 1 - npml) * d
    n_pillars = int((x_hi - x_lo) / period)
    widths = rng.uniform(0.1, 0.4, size=n_pillars) * wavelength
    for k in range(n_pillars):
        xc = x_lo + (k + 0.5) * period
        objs.append((_rect(xc - widths[k] / 2, xc + widths[k] / 2, y_sub, y_sub + height), 12.1))
    cells = cell_permittivity(nx, ny, d, d, 1.0, objs)
    eps = node_permittivity(cells)
    b = np.stack([line_source_x(nx, ny, d, npml + 10 + 3 * k) for k in range(nrhs)])
    return Workload("metalens", nx, ny, d, d, wavelength, eps, b,
                    npml=(npml,) * 4, nsub=nsub, overlap=overlap,
                    interface_pml=interface_pml, restart=50, rtol=1e-8,
                    meta=dict(seed=seed, n_pillars=n_pillars, j_substrate=j_sub))


def random_medium(nx, ny, ppw=20, seed=0, eps_range=(1.0, 4.0), npml=10,
                  nsub=2, overlap=4, interface_pml=10, nsrc=1, wavelength=1.0):
    """Smooth random permittivity with seeded point sources away from the PML
    (small parity and reciprocity cases)."""
    rng = np.random.default_rng(seed)
    d = wavelength / ppw
    cells = rng.uniform(eps_range[0], eps_range[1], size=(nx + 1, ny + 1))
    eps = node_permittivity(cells)
    b = np.zeros((nsrc, nx, ny), np.complex128)
    for r in range(nsrc):
        i = int(rng.integers(npml + 1, nx - npml - 1))
        j = int(rng.integers(npml + 1, ny - npml - 1))
        b[r] = point_source(nx, ny, d, d, i, j)
    return Workload("random", nx, ny, d, d, wavelength, eps, b,
                    npml=(npml,) * 4, nsub=nsub, overlap=overlap,
                    interface_pml=interface_pml, restart=30, rtol=1e-10,
                    meta=dict(seed=seed))


def ellipses(nx, ny, seed, ppw=24, npml=20, overlap=8, interface_pml=20, nsub=None, nrhs=1,
             sources="mixed", fill=(0.15, 0.30), eps_range=(2.0, 12.1), axes=(0.2, 1.0),
             keep=0.5, wavelength=1.0, rtol=1e-8, restart=30):
    """Vacuum with seeded non-overlapping dielectric ellipses (the batched and
    learned-guess geometries): semi-axes U[axes] wavelengths, random angle,
    eps U[eps_range] each, painted until the ellipses' total area reaches a
    fill fraction drawn from U[fill] of the non-PML area (or 400 placement
    attempts run out).  Ellipses are kept ``keep`` wavelengths from the PML
    and are separated by their circumscribed circles.  The number of strips
    is drawn from [2, max(2, min(8, nx // 128))] unless given.  Sources:
    ``"point"`` (unit point sources at random nodes at least ``keep`` from
    the PML), ``"line"`` (x-directed line sources on random rows) or
    ``"mixed"`` (each right-hand side one or the other, equally likely)."""
    rng = np.random.default_rng(seed)
    d = wavelength / ppw
    x_lo, x_hi = npml * d + keep * wavelength, (nx - 1 - npml) * d - keep * wavelength
    y_lo, y_hi = npml * d + keep * wavelength, (ny - 1 - npml) * d - keep * wavelength
    area = max(0.0, ((nx - 1 - 2 * npml) * d)) * max(0.0, ((ny - 1 - 2 * npml) * d))
    target = rng.uniform(*fill) * area
    placed, objs, got = [], [], 0.0
    for _ in range(400):
        if got >= target or x_hi <= x_lo or y_hi <= y_lo:
            break
        a, b = rng.uniform(*axes, size=2) * wavelength
        r = max(a, b)
        if x_hi - x_lo <= 2 * r or y_hi - y_lo <= 2 * r:
            continue
        cx = rng.uniform(x_lo + r, x_hi - r)
        cy = rng.uniform(y_lo + r, y_hi - r)
        th = rng.uniform(0, math.pi)
        if any((cx - px) ** 2 + (cy - py) ** 2 < (r + pr) ** 2 for px, py, pr in placed):
            continue
        placed.append((cx, cy, r))
        objs.append((_ellipse(cx, cy, a, b, th), float(rng.uniform(*eps_range))))
        got += math.pi * a * b
    cells = cell_permittivity(nx, ny, d, d, 1.0, objs)
    eps = node_permittivity(cells)
    if nsub is None:
        nsub = int(rng.integers(2, max(2, min(8, nx // 128)) + 1))
    i_lo, i_hi = npml + int(math.ceil(keep * ppw)), nx - 1 - npml - int(math.ceil(keep * ppw))
    j_lo, j_hi = npml + int(math.ceil(keep * ppw)), ny - 1 - npml - int(math.ceil(keep * ppw))
    b = np.zeros((nrhs, nx, ny), np.complex128)
    kinds = []
    for q in range(nrhs):
        kind = sources if sources != "mixed" else ("point" if rng.random() < 0.5 else "line")
        if kind == "point":
            b[q] = point_source(nx, ny, d, d, int(rng.integers(i_lo, i_hi + 1)), int(rng.integers(j_lo, j_hi + 1)))
        else:
            b[q] = line_source_x(nx, ny, d, int(rng.integers(j_lo, j_hi + 1)))
        kinds.append(kind)
    return Workload("ellipses", nx, ny, d, d, wavelength, eps, b,
                    npml=(npml,) * 4, nsub=nsub, overlap=overlap,
                    interface_pml=interface_pml, restart=restart, rtol=rtol,
                    meta=dict(seed=seed, n_ellipses=len(objs), fill=got / area if area else 0.0,
                              sources=kinds))


def _sbend(y0, dy, xs, length):
    """Centre line of a raised-cosine S-bend: y0 for x <= xs, y0 + dy for
    x >= xs + length, y0 + dy (1 - cos(pi t)) / 2 with t = (x - xs) / length
    in between (dy = 0: a straight guide).  Returns (y(x), dy/dx, ymin, ymax)."""
    length = max(length, 1e-12)

    def yc(x):
        t = np.clip((x - xs) / length, 0.0, 1.0)
        return y0 + dy * 0.5 * (1.0 - np.cos(np.pi * t))

    def slope(x):
        t = np.clip((x - xs) / length, 0.0, 1.0)
        return dy * 0.5 * np.pi / length * np.sin(np.pi * t)

    return yc, slope, min(y0, y0 + dy), max(y0, y0 + dy)


def _guides(xa, xb, arms, half):
    """Union of waveguide cores along the arms' centre lines for xa <= x < xb:
    a point belongs to a core if its vertical distance to a centre line is at
    most half * sqrt(1 + slope^2) (half the width measured normal to the
    line).  One object per x slab, so where arms overlap (a splitter's two
    branches leaving one guide) the subcell average sees their union."""
    def inside(x, y):
        m = np.zeros(np.broadcast(x, y).shape, bool)
        for yc, sl, _, _ in arms:
            m |= np.abs(y - yc(x)) <= half * np.sqrt(1.0 + sl(x) ** 2)
        return m & (x >= xa) & (x < xb)

    smax = max(float(np.max(np.abs(sl(np.linspace(xa, xb, 257))))) for _, sl, _, _ in arms)
    pad = half * math.sqrt(1.0 + smax ** 2) + 1e-9
    return inside, (xa, xb, min(a[2] for a in arms) - pad, max(a[3] for a in arms) + pad)


def slab_mode(eps_line, dy, wavelength):
    """Fundamental mode of a 1-D cross-section for an Ez field travelling
    along x: the eigenvector of largest eigenvalue beta^2 of
    (E[j+1] - 2 E[j] + E[j-1]) / dy^2 + k0^2 eps[j] E[j] = beta^2 E[j] with
    E = 0 beyond both ends (the guided mode has decayed there).  Returns beta
    and the profile scaled to a positive peak of 1."""
    from scipy.linalg import eigh_tridiagonal
    k0 = 2 * math.pi / wavelength
    eps_line = np.asarray(eps_line, float)
    n = eps_line.size
    diag = -2.0 / dy ** 2 + k0 ** 2 * eps_line
    off = np.full(n - 1, 1.0 / dy ** 2)
    val, vec = eigh_tridiagonal(diag, off, select="i", select_range=(n - 1, n - 1))
    phi = vec[:, 0]
    phi = phi / phi[np.argmax(np.abs(phi))]
    return math.sqrt(val[0]), phi


def waveguide_network(nx=8192, ny=2048, ppw=24, seed=2, npml=32, nsub=32, overlap=16, interface_pml=32,
                      width=0.45, eps_core=12.1, eps_clad=2.085, wavelength=1.0, rtol=1e-8, restart=50):
    """Silicon-like waveguide network: eps_core cores ``width`` wavelengths
    wide in eps_clad cladding, guides running along x from the left PML to the
    right one.  An input guide on the centre row splits at four seeded Y
    splitters (1 -> 2 -> 4 -> 5 branches: two branches leave one guide as
    raised-cosine S-bends of opposite offsets) and eight seeded S-bends shift
    single branches (four between the second and third splitter stage, four
    after the last).  The layout scales with the grid (positions and offsets
    are fractions of its size; the full case is 8192 x 2048 at lambda/24,
    32-cell PML, 32 strips, overlap 16).  The source is the guide's
    fundamental mode: ``slab_mode`` of the permittivity column 12 cells right
    of the left PML, placed on that column as a y-directed line current
    b[i, j] = -phi_j / dx (it radiates the mode both ways; the left-going
    half leaves through the PML)."""
    rng = np.random.default_rng(seed)
    d = wavelength / ppw
    Lx, Ly = (nx - 1) * d, (ny - 1) * d
    half = 0.5 * width * wavelength

    def at(f, jit):  # an x position on a cell edge
        return round((f + rng.uniform(-jit, jit)) * Lx / d) * d

    x1, x2, x3, x4, x5 = (at(0.088, 0.015), at(0.264, 0.015), at(0.41, 0.015), at(0.586, 0.015),
                          at(0.732, 0.015))
    xend = (nx + 2) * d
    d1, d2, d3 = 0.1875 * Ly, 0.094 * Ly, 0.047 * Ly
    ys = [round(0.5 * Ly / d) * d]
    slabs = [(-2 * d, x1, [_sbend(ys[0], 0.0, 0.0, 1.0)])]
    # splitter 1 and the two splitters of stage 2
    arms = [_sbend(y, s * d1, x1, 0.117 * Lx) for y in ys for s in (-1, 1)]
    slabs.append((x1, x2, arms))
    ys = sorted(y + s * d1 for y in ys for s in (-1, 1))
    arms = [_sbend(y, s * d2, x2, 0.088 * Lx) for y in ys for s in (-1, 1)]
    slabs.append((x2, x3, arms))
    ys = sorted(y + s * d2 for y in ys for s in (-1, 1))
    # four S-bends
    arms, nys = [], []
    for y in ys:
        xs = x3 + rng.uniform(0.0, 0.03) * Lx
        length = min(rng.uniform(0.073, 0.117) * Lx, x4 - xs - d)
        off = rng.uniform(-1.0, 1.0) * 0.035 * Ly
        arms.append(_sbend(y, off, xs, length))
        nys.append(y + off)
    slabs.append((x3, x4, arms))
    ys = nys
    # splitter 4 on one branch
    k3 = int(rng.integers(len(ys)))
    arms, nys = [], []
    for k, y in enumerate(ys):
        if k == k3:
            arms += [_sbend(y, s * d3, x4, 0.073 * Lx) for s in (-1, 1)]
            nys += [y - d3, y + d3]
        else:
            arms.append(_sbend(y, 0.0, x4, 1.0))
            nys.append(y)
    slabs.append((x4, x5, arms))
    ys = sorted(nys)
    # four S-bends on four of the five branches
    pick = set(int(v) for v in rng.choice(len(ys), 4, replace=False))
    arms, nys = [], []
    for k, y in enumerate(ys):
        if k in pick:
            xs = x5 + rng.uniform(0.0, 0.03) * Lx
            off = rng.uniform(-1.0, 1.0) * 0.023 * Ly
            arms.append(_sbend(y, off, xs, rng.uniform(0.073, 0.117) * Lx))
            nys.append(y + off)
        else:
            arms.append(_sbend(y, 0.0, x5, 1.0))
            nys.append(y)
    slabs.append((x5, xend, arms))
    ys = sorted(nys)
    gap = min(b - a for a, b in zip(ys, ys[1:])) - width * wavelength
    if gap <= 0 or ys[0] - half <= (npml + 1) * d or ys[-1] + half >= Ly - (npml + 1) * d:
        raise ValueError("grid too small for the waveguide network")
    objs = [(_guides(xa, xb, arms, half), eps_core) for xa, xb, arms in slabs]
    cells = cell_permittivity(nx, ny, d, d, eps_clad, objs)
    eps = node_permittivity(cells)
    i_src = npml + 12
    beta, phi = slab_mode(eps[i_src], d, wavelength)
    b = np.zeros((1, nx, ny), np.complex128)
    b[0, i_src, :] = -phi / d
    return Workload("waveguide-network", nx, ny, d, d, wavelength, eps, b,
                    npml=(npml,) * 4, nsub=nsub, overlap=overlap, interface_pml=interface_pml,
                    restart=restart, rtol=rtol,
                    meta=dict(seed=seed, splitters=4, sbends=8, branches=len(ys), outputs=ys,
                              min_gap=gap, x_stages=(x1, x2, x3, x4, x5), i_src=i_src, beta=beta,
                              neff=beta / (2 * math.pi / wavelength)))


def random_vector(n, seed, nrhs=1):
    """Seeded complex test vector(s) of length n (operator parity inputs)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))).astype(np.complex128)
