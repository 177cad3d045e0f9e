"""Two-dimensional (checkerboard) partitions of the overlapping PML-based
source-transfer DDM: plain CPU form.

Oracle module (test infrastructure; see the package docstring).

The paper cuts the grid into strips along x (Sec. 2.3).  This module extends
the same construction to boxes: the x-strip partition of ``oracle.stddm`` is
applied along x and, independently, along y, and box (kx, ky) owns the nodes
of x-strip kx's owned columns and y-strip ky's owned rows.  Its local box adds
overlap + interface_pml nodes on each side that has a neighbour, in x and in
y, with an interface_pml-cell local PML in the outer cells of that extension
(the strips' construction of Sec. 2.3 applied per axis); on the domain's sides
it keeps the global PML.  Outside its box a local problem is Dirichlet.

The preconditioner keeps the strips' definition, M^-1 = sum_k E_k A_k^-1 R_k^I
(one Jacobi source-transfer sweep followed by the synthesis of Eq. 21 with
full local fields), now summed over boxes.  With one box row it is the strip
method itself.

Parity status: pinned by its reduction to the strip oracle (one box row or
one box column), by one box being the direct solve, by the transpose symmetry
of the construction (the transposed problem with transposed boxes gives the
transposed M^-1) and by FGMRES reaching the direct solution.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .fdfd import Problem, assemble, stretch_profile
from .stddm import partition


class Box:
    """Box (kx, ky): owned columns [c0, c1) x rows [r0, r1); local box
    [x0, x1) x [y0, y1) with PML widths (Lx_lo, Lx_hi, Ly_lo, Ly_hi)."""

    def __init__(self, sx, sy):
        self.kx, self.ky = sx.k, sy.k
        self.c0, self.c1, self.x0, self.x1 = sx.c0, sx.c1, sx.x0, sx.x1
        self.r0, self.r1, self.y0, self.y1 = sy.c0, sy.c1, sy.x0, sy.x1
        self.Lx_lo, self.Lx_hi, self.Ly_lo, self.Ly_hi = sx.L_lo, sx.L_hi, sy.L_lo, sy.L_hi

    @property
    def width(self):
        return self.x1 - self.x0

    @property
    def height(self):
        return self.y1 - self.y0


class CheckerboardDDM:
    """px x py boxes of a Problem; local operators, their LU factors,
    restriction to owned nodes and zero extension of full local fields."""

    def __init__(self, prob: Problem, px, py, overlap, interface_pml):
        self.prob = prob
        self.px, self.py = int(px), int(py)
        xs = partition(prob.nx, self.px, overlap, interface_pml, prob.npml[0], prob.npml[1])
        ys = partition(prob.ny, self.py, overlap, interface_pml, prob.npml[2], prob.npml[3])
        self.boxes = [Box(sx, sy) for sx in xs for sy in ys]
        self._lu = {}

    def local_A(self, k):
        """A_k: the stretched stencil on box k's local box, local PML on its
        interior sides, global PML on the domain's sides, Dirichlet outside."""
        p, b = self.prob, self.boxes[k]
        sx, sxh = stretch_profile(b.width, b.Lx_lo, b.Lx_hi, p.dx, p.k0, p.m, p.R)
        sy, syh = stretch_profile(b.height, b.Ly_lo, b.Ly_hi, p.dy, p.k0, p.m, p.R)
        return assemble(b.width, b.height, p.dx, p.dy, p.k0, p.eps[b.x0:b.x1, b.y0:b.y1], sx, sxh, sy, syh)

    def local_solve(self, k, t):
        if k not in self._lu:
            self._lu[k] = spla.splu(self.local_A(k).tocsc())
        return self._lu[k].solve(np.asarray(t, dtype=np.complex128))

    def _view(self, k, v):
        b = self.boxes[k]
        return np.asarray(v).reshape(self.prob.nx, self.prob.ny)[b.x0:b.x1, b.y0:b.y1]

    def restrict_owned(self, k, v):
        """R_k^I v as a local vector: v on the owned nodes, 0 elsewhere."""
        b = self.boxes[k]
        t = np.zeros((b.width, b.height), np.complex128)
        sl = (slice(b.c0 - b.x0, b.c1 - b.x0), slice(b.r0 - b.y0, b.r1 - b.y0))
        t[sl] = self._view(k, v)[sl]
        return t.ravel()

    def extend(self, k, e):
        """E_k e: zero extension of the full local field to the grid."""
        b = self.boxes[k]
        out = np.zeros((self.prob.nx, self.prob.ny), np.complex128)
        out[b.x0:b.x1, b.y0:b.y1] = np.asarray(e).reshape(b.width, b.height)
        return out.ravel()

    def apply_Minv(self, v):
        """M^-1 v = sum_k E_k A_k^-1 R_k^I v."""
        out = np.zeros(self.prob.n, np.complex128)
        for k in range(len(self.boxes)):
            out += self.extend(k, self.local_solve(k, self.restrict_owned(k, v)))
        return out
