"""Overlapping PML-based source-transfer DDM (Sec. 2.3, Algorithm 1): plain CPU form.

Oracle module (test infrastructure; see the package docstring).

Partition (Sec. 2.3, Fig. 3).  The grid is cut along x into ``nsub`` strips
of node columns; strip k owns columns [c_k, c_{k+1}) (equal widths, the
remainder going one column each to the first strips).  The owned sets are
disjoint and cover the grid (the paper's non-overlapping interiors).  The
local box of strip k adds ext = overlap + interface_pml columns on each side
that has a neighbour: ``overlap`` physical columns and then an
``interface_pml``-cell PML whose interface half node is where the overlap band
ends.  At the domain ends the strip keeps the global x-PML.  Every strip keeps
the global y-PML.  Outside its box a local problem is Dirichlet.

Unknown split (Eq. 15): I_k = owned nodes (this includes global PML at the
domain ends), F_k = local nodes not owned (overlap band + interface PML),
which lie in the neighbouring strips' owned columns.

Readings of the paper used here:

* Transfer operator (Eqs. 16-17): T_pi(e_i) = R_p^I A (E_i e_i): the global
  stencil applied to strip i's zero-extended local field (PML part included),
  restricted to strip p's owned nodes.  It is non-zero only near the cut.
* Sign (Eqs. 18-19): the update source is t_p = -sum_{i != p} T_pi(e_i), which
  equals the global residual restricted to I_p; with the printed "+" the sum
  of Eq. 21 would not solve A e = b.
* Order: Jacobi -- every strip uses the other strips' previous iterate.
* Stopping test (Eq. 20, Algorithm 1's WHILE): iterate while
  sum_i ||e_i^F|| >= TOL (the printed "<" is read as ">=").
* Synthesis (Eq. 21): e_g = sum_n sum_i E_i e_i^(n), full local fields.

With these readings one sweep is x <- x + M^-1 (b - A x) with
M^-1 = sum_i E_i A_i^-1 R_i^I (Richardson on the one-sweep preconditioner).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse.linalg as spla

from .fdfd import Problem, assemble, stretch_profile


@dataclasses.dataclass
class Strip:
    k: int
    c0: int      # first owned column
    c1: int      # one past the last owned column
    x0: int      # first column of the local box
    x1: int      # one past the last column of the local box
    L_lo: int    # PML cells at the low-x end of the box
    L_hi: int    # PML cells at the high-x end of the box

    @property
    def width(self):
        return self.x1 - self.x0


def partition(nx, nsub, overlap, interface_pml, npml_x0, npml_x1):
    """Strip decomposition along x (see module docstring)."""
    if nsub < 1 or nsub > nx:
        raise ValueError("bad nsub")
    ext = overlap + interface_pml
    base, rem = divmod(nx, nsub)
    widths = [base + (1 if k < rem else 0) for k in range(nsub)]
    cuts = np.concatenate([[0], np.cumsum(widths)]).astype(int)
    strips = []
    for k in range(nsub):
        c0, c1 = int(cuts[k]), int(cuts[k + 1])
        x0 = c0 - ext if k > 0 else 0
        x1 = c1 + ext if k < nsub - 1 else nx
        # the extension must stay inside the neighbour's owned columns
        if k > 0 and ext > widths[k - 1]:
            raise ValueError("overlap + interface PML wider than a neighbouring strip")
        if k < nsub - 1 and ext > widths[k + 1]:
            raise ValueError("overlap + interface PML wider than a neighbouring strip")
        strips.append(Strip(k, c0, c1, x0, x1,
                            interface_pml if k > 0 else npml_x0,
                            interface_pml if k < nsub - 1 else npml_x1))
    return strips


class DDM:
    """The decomposed problem: local operators A_i, their factorizations,
    restriction R_i^I and zero extension E_i."""

    def __init__(self, prob: Problem, nsub, overlap, interface_pml):
        self.prob = prob
        self.nsub = int(nsub)
        self.overlap = int(overlap)
        self.interface_pml = int(interface_pml)
        self.strips = partition(prob.nx, self.nsub, self.overlap, self.interface_pml,
                                prob.npml[0], prob.npml[1])
        self._A_loc = [None] * self.nsub
        self._lu = [None] * self.nsub

    @classmethod
    def from_workload(cls, w, prob=None):
        prob = prob or Problem.from_workload(w)
        return cls(prob, w.nsub, w.overlap, w.interface_pml)

    # ---- local operators -------------------------------------------------
    def local_stretch_x(self, s: Strip):
        p = self.prob
        return stretch_profile(s.width, s.L_lo, s.L_hi, p.dx, p.k0, p.m, p.R)

    def local_A(self, k):
        """A_k: the stretched stencil on strip k's local box, local x-PML at
        interior sides, global PML elsewhere, Dirichlet outside the box
        (Algorithm 1, preprocessing)."""
        if self._A_loc[k] is None:
            p, s = self.prob, self.strips[k]
            sx, sxh = self.local_stretch_x(s)
            self._A_loc[k] = assemble(s.width, p.ny, p.dx, p.dy, p.k0, p.eps[s.x0:s.x1],
                                      sx, sxh, p.sy, p.syh)
        return self._A_loc[k]

    def factor(self, k=None):
        ks = range(self.nsub) if k is None else [k]
        for kk in ks:
            if self._lu[kk] is None:
                self._lu[kk] = spla.splu(self.local_A(kk).tocsc())

    def local_solve(self, k, t):
        """A_k^-1 t by the sparse direct LU (the exact local inverse)."""
        self.factor(k)
        return self._lu[k].solve(np.asarray(t, dtype=np.complex128))

    # ---- restriction / extension ----------------------------------------
    def restrict_owned(self, k, v):
        """R_k^I v as a local vector: v on owned columns, 0 on F columns."""
        s, ny = self.strips[k], self.prob.ny
        t = np.zeros(s.width * ny, np.complex128)
        a = (s.c0 - s.x0) * ny
        t[a:a + (s.c1 - s.c0) * ny] = v[s.c0 * ny:s.c1 * ny]
        return t

    def extend(self, k, e):
        """E_k e: zero extension of the full local field to the global grid."""
        s, ny = self.strips[k], self.prob.ny
        out = np.zeros(self.prob.n, np.complex128)
        out[s.x0 * ny:s.x1 * ny] = e
        return out

    def f_part(self, k, e):
        """e_k^F: the local field on the non-owned (overlap + PML) columns."""
        s, ny = self.strips[k], self.prob.ny
        lo = e[:(s.c0 - s.x0) * ny]
        hi = e[(s.c1 - s.x0) * ny:]
        return np.concatenate([lo, hi])

    # ---- the preconditioner and the paper's iteration --------------------
    def local_solutions(self, v):
        """[A_i^-1 R_i^I v for every strip i]."""
        return [self.local_solve(k, self.restrict_owned(k, v)) for k in range(self.nsub)]

    def apply_Minv(self, v):
        """M^-1 v = sum_i E_i A_i^-1 R_i^I v: one Jacobi source-transfer sweep
        followed by synthesis (Eq. 21)."""
        out = np.zeros(self.prob.n, np.complex128)
        for k, z in enumerate(self.local_solutions(v)):
            out += self.extend(k, z)
        return out

    def apply_Minv_multiplicative(self, v, order=None):
        """A multiplicative order of the same local solves (the layer-by-layer
        source transfer the method comes from, Sec. 1): strips one after
        another, each solving for the residual left by the previous ones,
        z <- z + E_k A_k^-1 R_k^I (v - A z), from z = 0.  Default order: the
        symmetric sweep k = 0..n-1, n-2..0; "red-black": the even strips, then
        the odd strips."""
        v = np.asarray(v, dtype=np.complex128)
        z = np.zeros(self.prob.n, np.complex128)
        if order is None:
            order = list(range(self.nsub)) + list(range(self.nsub - 2, -1, -1))
        elif order == "red-black":
            order = list(range(0, self.nsub, 2)) + list(range(1, self.nsub, 2))
        for k in order:
            r = v - self.prob.A @ z
            z = z + self.extend(k, self.local_solve(k, self.restrict_owned(k, r)))
        return z

    def transfer(self, p, i, e_i):
        """T_pi(e_i) = R_p^I A (E_i e_i) (Eq. 17 under the reading above), as
        a local vector of strip p."""
        return self.restrict_owned(p, self.prob.A @ self.extend(i, e_i))

    def algorithm1(self, b, tol, maxit):
        """Algorithm 1 as printed (with the readings above): initial local
        solves on each strip's own source, then Jacobi source transfer through
        the overlapping PML until sum_i ||e_i^F|| < tol.

        Returns (e_g, history) where history[n] = (sum_i ||e_i^F,(n)||, the
        partial synthesis sum_{n' <= n} sum_i E_i e_i^(n'))."""
        b = np.asarray(b, dtype=np.complex128)
        e = self.local_solutions(b)                       # e_i^(0)
        eg = sum(self.extend(k, e[k]) for k in range(self.nsub))
        fnorm = sum(np.linalg.norm(self.f_part(k, e[k])) for k in range(self.nsub))
        history = [(fnorm, eg.copy())]
        n = 0
        while fnorm >= tol and n < maxit:
            n += 1
            new = []
            for p in range(self.nsub):
                t = np.zeros(self.strips[p].width * self.prob.ny, np.complex128)
                for i in range(self.nsub):
                    if i != p:
                        t -= self.transfer(p, i, e[i])
                new.append(self.local_solve(p, t))
            e = new
            eg = eg + sum(self.extend(k, e[k]) for k in range(self.nsub))
            fnorm = sum(np.linalg.norm(self.f_part(k, e[k])) for k in range(self.nsub))
            history.append((fnorm, eg.copy()))
        return eg, history

    def richardson(self, b, nit, x0=None):
        """x_{n+1} = x_n + M^-1 (b - A x_n), the residual form of Algorithm 1.
        Returns the list of iterates x_1 .. x_nit (x_0 = 0 unless given)."""
        b = np.asarray(b, dtype=np.complex128)
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
        out = []
        for _ in range(nit):
            x = x + self.apply_Minv(b - self.prob.A @ x)
            out.append(x.copy())
        return out
