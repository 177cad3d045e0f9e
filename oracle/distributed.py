"""The strip method split over processes: plain CPU form of its one exchange
step (test infrastructure; see the package docstring).

Rank r of W owns a contiguous group of strips, strips [k0, k1) with
k0 = r * nsub // W, and keeps every global vector only on its owned columns
[C0, C1) (the union of its strips' owned columns).  The method then needs, per
preconditioner application and per matrix-vector product:

* synthesis (Eq. 21): a strip's full local field reaches ext = overlap +
  interface_pml columns past its owned columns, so the part of the rank's
  summed local fields on [C0 - ext, C0) belongs to rank r - 1 and the part on
  [C1, C1 + ext) to rank r + 1: ext x ny values cross each cut in each
  direction and are added to the receiver's owned columns;
* the stencil: rows of the owned columns read one column on each side, so
  one boundary column crosses each cut in each direction;
* the Krylov iteration: every inner product is a sum of the ranks' partial
  products (one all-reduce).

``comm`` is ``torch.distributed`` (any backend with send / recv and
all_reduce on CPU tensors, e.g. gloo); complex vectors travel as float64
pairs.  Everything else is the single-process oracle: the same partition,
local operators and local solves (``oracle.stddm.DDM``) and the same
textbook FGMRES (``oracle.krylov.gmres`` with a summed inner product).
"""
from __future__ import annotations

import numpy as np

from .fdfd import Problem
from .krylov import gmres
from .stddm import DDM


class RankStrips:
    def __init__(self, prob: Problem, nsub, overlap, interface_pml, rank, world, comm):
        if world > nsub:
            raise ValueError("more ranks than strips")
        self.p, self.rank, self.world, self.comm = prob, int(rank), int(world), comm
        self.ddm = DDM(prob, nsub, overlap, interface_pml)
        self.k0, self.k1 = rank * nsub // world, (rank + 1) * nsub // world
        st = self.ddm.strips
        # a local field spills ext columns past its strip; the exchange hands
        # each spill to the adjacent rank only, so every rank must own at
        # least ext columns (else the spill would reach two ranks away)
        ext = overlap + interface_pml
        for r in range(world):
            a, b = r * nsub // world, (r + 1) * nsub // world
            if world > 1 and st[b - 1].c1 - st[a].c0 < ext:
                raise ValueError(f"rank {r} owns {st[b - 1].c1 - st[a].c0} columns, fewer than overlap + "
                                 f"interface PML = {ext}: its neighbours' fields would reach past it")
        self.C0, self.C1 = st[self.k0].c0, st[self.k1 - 1].c1
        self.L0, self.L1 = st[self.k0].x0, st[self.k1 - 1].x1   # columns the rank's local fields reach
        self.sent_values = 0                                   # complex values sent so far
        A = prob.A.tocsr()
        ny = prob.ny
        lo, hi = max(self.C0 - 1, 0), min(self.C1 + 1, prob.nx)
        self._hl, self._hh = lo, hi
        self._rows = A[self.C0 * ny:self.C1 * ny][:, lo * ny:hi * ny]

    # ---- point-to-point exchange with the neighbouring ranks -------------
    def _exchange(self, send_lo, send_hi, n_lo, n_hi):
        """Send send_lo to rank - 1 and send_hi to rank + 1; receive n_lo
        values from rank - 1 and n_hi from rank + 1 (complex)."""
        import torch
        c = self.comm
        reqs, bufs = [], {}
        if self.rank > 0:
            t = torch.from_numpy(np.ascontiguousarray(send_lo).view(np.float64).copy())
            reqs.append(c.isend(t, self.rank - 1))
            self.sent_values += send_lo.size
            bufs["lo"] = torch.empty(2 * n_lo, dtype=torch.float64)
            reqs.append(c.irecv(bufs["lo"], self.rank - 1))
        if self.rank < self.world - 1:
            t = torch.from_numpy(np.ascontiguousarray(send_hi).view(np.float64).copy())
            reqs.append(c.isend(t, self.rank + 1))
            self.sent_values += send_hi.size
            bufs["hi"] = torch.empty(2 * n_hi, dtype=torch.float64)
            reqs.append(c.irecv(bufs["hi"], self.rank + 1))
        for r in reqs:
            r.wait()
        return ({k: v.numpy().view(np.complex128) for k, v in bufs.items()})

    # ---- vectors held on the owned columns --------------------------------
    def owned(self, v):
        ny = self.p.ny
        return np.asarray(v)[self.C0 * ny:self.C1 * ny].copy()

    def matvec(self, z):
        """(A z) on the owned columns; one boundary column from each neighbour."""
        ny = self.p.ny
        got = self._exchange(z[:ny], z[-ny:], ny, ny)
        parts = []
        if self._hl < self.C0:
            parts.append(got["lo"])
        parts.append(z)
        if self._hh > self.C1:
            parts.append(got["hi"])
        return self._rows @ np.concatenate(parts)

    def precond(self, v):
        """(M^-1 v) on the owned columns: the rank's local solves, their full
        local fields summed, the spill past the cuts exchanged and added."""
        ny = self.p.ny
        buf = np.zeros((self.L1 - self.L0) * ny, np.complex128)
        for k in range(self.k0, self.k1):
            s = self.ddm.strips[k]
            t = np.zeros(s.width * ny, np.complex128)
            a = (s.c0 - s.x0) * ny
            t[a:a + (s.c1 - s.c0) * ny] = v[(s.c0 - self.C0) * ny:(s.c1 - self.C0) * ny]
            z = self.ddm.local_solve(k, t)
            buf[(s.x0 - self.L0) * ny:(s.x1 - self.L0) * ny] += z
        lo_n, hi_n = (self.C0 - self.L0) * ny, (self.L1 - self.C1) * ny
        own = buf[lo_n:lo_n + (self.C1 - self.C0) * ny].copy()
        # the neighbours' spills onto this rank's columns: rank - 1 sends the
        # part of its fields right of its cut, rank + 1 the part left of its cut
        n_from_lo = self._spill(self.rank - 1, hi=True) if self.rank > 0 else 0
        n_from_hi = self._spill(self.rank + 1, hi=False) if self.rank < self.world - 1 else 0
        got = self._exchange(buf[:lo_n], buf[len(buf) - hi_n:], n_from_lo, n_from_hi)
        if "lo" in got:
            own[:got["lo"].size] += got["lo"]
        if "hi" in got:
            own[own.size - got["hi"].size:] += got["hi"]
        return own

    def _spill(self, r, hi):
        """Values rank r's local fields put past its high (hi) or low cut."""
        st, ny, W, n = self.ddm.strips, self.p.ny, self.world, self.ddm.nsub
        k0, k1 = r * n // W, (r + 1) * n // W
        return (st[k1 - 1].x1 - st[k1 - 1].c1) * ny if hi else (st[k0].c0 - st[k0].x0) * ny

    def dot(self, a, b):
        """conj(a) . b summed over the ranks."""
        import torch
        part = np.vdot(a, b)
        t = torch.tensor([part.real, part.imag], dtype=torch.float64)
        self.comm.all_reduce(t)
        return complex(t[0].item(), t[1].item())

    def solve(self, b_owned, **kw):
        """FGMRES on the owned parts (every rank calls it with its part)."""
        return gmres(self.matvec, self.precond, b_owned, dot=self.dot, **kw)
