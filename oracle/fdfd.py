"""2-D TM FDFD with stretched-coordinate PML: the plain definition.

Oracle module (test infrastructure; see the package docstring).

Unknowns are the field E_z at every node of an nx x ny grid, PML included;
node (i, j) has flat index g = i*ny + j.  Outside the grid the field is zero
(Dirichlet termination behind the PML).

Row (i, j) of A applies the stretched Helmholtz operator of Eq. 9 discretised
on the 5-point stencil of Eq. 2:

  1/(sx_i dx^2) * [ (u_{i+1,j}-u_{i,j})/sx_{i+1/2} - (u_{i,j}-u_{i-1,j})/sx_{i-1/2} ]
+ 1/(sy_j dy^2) * [ (u_{i,j+1}-u_{i,j})/sy_{j+1/2} - (u_{i,j}-u_{i,j-1})/sy_{j-1/2} ]
+ k0^2 epsbar_{i,j} u_{i,j}

which is Eq. 2 exactly where s = 1.  The PML stretch s = 1 + i sigma/(w eps0)
(Eq. 10) uses the e^{-i w t} convention (the paper's "j" is read as the
physicist's i so that outgoing e^{+ikr} waves decay).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def sigma_hat_max(L, delta, k0, m, R):
    """sigma_max/(w eps0) of Eq. 13 in dimensionless form.

    Eq. 13 prints sigma_max = (m+1) ln R(0) / (2 eta d); ln R < 0 makes that
    negative, so the sign is read as sigma_max = -(m+1) ln R / (2 eta d).
    With eta*eps0 = 1/c, sigma_max/(w eps0) = (m+1)(-ln R)/(2 k0 d),
    d = L*delta the physical PML depth."""
    d = L * delta
    return (m + 1) * (-math.log(R)) / (2.0 * k0 * d)


def stretch_profile(n, L_lo, L_hi, delta, k0, m, R):
    """Stretch factors on a line of n nodes with an L_lo-cell PML at the low
    end and an L_hi-cell PML at the high end (Eqs. 10-12).

    Returns (s_node[n], s_half[n+1]); half node h lies between nodes h-1 and
    h (position h - 1/2 in cell units).  Reading of Eqs. 11-12: counted from
    the PML/interior interface, PML node u = 1..L sits at depth (u - 1/2)
    cells and half node u + 1/2 (u = 0..L) at depth u cells, so sigma is 0 at
    the interface half node and sigma_max at the outermost half node; the
    /Delta of Eqs. 11-12 is absorbed into the normalisation of Eq. 13."""
    pos_node = np.arange(n, dtype=np.float64)
    pos_half = np.arange(n + 1, dtype=np.float64) - 0.5

    def sig(pos):
        out = np.zeros_like(pos)
        if L_lo > 0:
            depth = np.maximum(0.0, (L_lo - 0.5) - pos)
            out += sigma_hat_max(L_lo, delta, k0, m, R) * (depth / L_lo) ** m
        if L_hi > 0:
            depth = np.maximum(0.0, pos - (n - L_hi - 0.5))
            out += sigma_hat_max(L_hi, delta, k0, m, R) * (depth / L_hi) ** m
        return out

    return 1.0 + 1j * sig(pos_node), 1.0 + 1j * sig(pos_half)


def assemble(nx, ny, dx, dy, k0, eps_node, sx, sxh, sy, syh):
    """Sparse A (CSR, complex128) of the stretched 5-point operator.

    sx[nx], sxh[nx+1], sy[ny], syh[ny+1] are node / half-node stretches as
    returned by stretch_profile; eps_node is (nx, ny)."""
    n = nx * ny
    I, J = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    I = I.ravel()
    J = J.ravel()
    g = I * ny + J
    cxm = 1.0 / (sx[I] * sxh[I] * dx * dx)          # coupling to (i-1, j)
    cxp = 1.0 / (sx[I] * sxh[I + 1] * dx * dx)      # coupling to (i+1, j)
    cym = 1.0 / (sy[J] * syh[J] * dy * dy)          # coupling to (i, j-1)
    cyp = 1.0 / (sy[J] * syh[J + 1] * dy * dy)      # coupling to (i, j+1)
    diag = k0 * k0 * eps_node.ravel() - cxm - cxp - cym - cyp
    rows = [g]
    cols = [g]
    vals = [diag]
    for mask, dg, c in ((I > 0, -ny, cxm), (I < nx - 1, ny, cxp),
                        (J > 0, -1, cym), (J < ny - 1, 1, cyp)):
        rows.append(g[mask])
        cols.append(g[mask] + dg)
        vals.append(c[mask])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n), dtype=np.complex128)
    return A


class Problem:
    """Global FDFD problem: grid, materials, PML; builds the global A.

    npml = (x0, x1, y0, y1) PML cells; pml_order m; pml_R = R(0)."""

    def __init__(self, nx, ny, dx, dy, wavelength, eps_node, npml=(20, 20, 20, 20),
                 pml_order=3, pml_R=1e-8):
        self.nx, self.ny = int(nx), int(ny)
        self.dx, self.dy = float(dx), float(dy)
        self.wavelength = float(wavelength)
        self.k0 = 2.0 * math.pi / self.wavelength
        self.eps = np.asarray(eps_node, dtype=np.float64).reshape(self.nx, self.ny)
        self.npml = tuple(int(v) for v in npml)
        self.m = int(pml_order)
        self.R = float(pml_R)
        self.sx, self.sxh = stretch_profile(self.nx, self.npml[0], self.npml[1], self.dx,
                                            self.k0, self.m, self.R)
        self.sy, self.syh = stretch_profile(self.ny, self.npml[2], self.npml[3], self.dy,
                                            self.k0, self.m, self.R)
        self._A = None
        self._lu = None

    @classmethod
    def from_workload(cls, w):
        return cls(w.nx, w.ny, w.dx, w.dy, w.wavelength, w.eps_node, w.npml,
                   w.pml_order, w.pml_R)

    @property
    def n(self):
        return self.nx * self.ny

    @property
    def A(self):
        if self._A is None:
            self._A = assemble(self.nx, self.ny, self.dx, self.dy, self.k0, self.eps,
                               self.sx, self.sxh, self.sy, self.syh)
        return self._A

    def matvec(self, x):
        return self.A @ x

    def solve(self, b):
        """Plain definition of the solution e = A^-1 b (Eq. 4) by a sparse
        direct LU with partial pivoting (SuperLU)."""
        if self._lu is None:
            self._lu = spla.splu(self.A.tocsc())
        return self._lu.solve(np.asarray(b, dtype=np.complex128))
