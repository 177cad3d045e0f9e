"""The working matrix of the blocked Gauss-Jordan sweep on a complex
symmetric front (the symmetric form, D A_k of the oracle's local operator):
after every block step it is symmetric within the eliminated indices and
within the remaining ones and antisymmetric between them, which is what lets
the GPU update compute one triangle and take the pivot rows as the signed
transpose of the pivot columns.  The sweep here is the plain blocked
Gauss-Jordan of Sec. 2.4 in numpy (diagonal block inverted, column panel
C <- -C D^-1, update A <- A + C R, row panel R <- D^-1 R), on a front taken
from the oracle's strip operator; its end state is checked against the
block formulas [X^-1, X^-1 M_ER; -M_RE X^-1, S]."""
import numpy as np
import scipy.sparse as sp

import workloads as W
from oracle.fdfd import Problem
from oracle.stddm import DDM


def _front():
    w = W.random_medium(60, 24, ppw=16, seed=5, npml=6, nsub=2, overlap=3, interface_pml=6, nsrc=1)
    P = Problem.from_workload(w)
    D = DDM.from_workload(w, P)
    st = D.strips[0]
    sx, _ = D.local_stretch_x(st)
    d = np.outer(sx, P.sy).ravel()
    B = (sp.diags(d) @ D.local_A(0)).toarray()
    idx = np.arange(40)            # a front: the PML corner's first 40 nodes, coupled in x and y
    F = B[np.ix_(idx, idx)]
    F = F + 3.0 * np.eye(40) * np.abs(F).max()                  # well-conditioned pivots
    assert np.abs(F - F.T).max() <= 1e-14 * np.abs(F).max()
    return F


def _gj_blocked(F, p, nb, check):
    Wm = F.copy()
    n = Wm.shape[0]
    for k in range(0, p, nb):
        P = np.arange(k, min(k + nb, p))
        Rr = np.setdiff1d(np.arange(n), P)
        Dinv = np.linalg.inv(Wm[np.ix_(P, P)])
        C = -Wm[np.ix_(Rr, P)] @ Dinv                 # column panel
        Rw = Wm[np.ix_(P, Rr)].copy()                 # row panel, before its product
        Wm[np.ix_(Rr, Rr)] += C @ Rw                  # update (unscaled row panel)
        Wm[np.ix_(Rr, P)] = C
        Wm[np.ix_(P, Rr)] = Dinv @ Rw
        Wm[np.ix_(P, P)] = Dinv
        check(Wm, P[-1] + 1)
    return Wm


def test_working_matrix_sign_pattern_after_every_block_step():
    F = _front()
    n, p = F.shape[0], 28
    scale = np.abs(F).max()

    def check(Wm, kdone):
        elim = np.arange(n) < kdone
        sigma = np.where(elim[:, None] != elim[None, :], -1.0, 1.0)
        assert np.abs(Wm.T - sigma * Wm).max() <= 1e-12 * max(scale, np.abs(Wm).max())
        # the pivot rows are the signed transpose of the pivot columns (the mirror kernel)
        assert np.abs(Wm[:kdone, kdone:] + Wm[kdone:, :kdone].T).max() <= 1e-12 * np.abs(Wm).max()

    for nb in (1, 4, 7):
        Wm = _gj_blocked(F, p, nb, check)
        # end state: the block Gauss-Jordan formulas
        X, MER, MRE, MRR = F[:p, :p], F[:p, p:], F[p:, :p], F[p:, p:]
        Xi = np.linalg.inv(X)
        ref = np.block([[Xi, Xi @ MER], [-MRE @ Xi, MRR - MRE @ Xi @ MER]])
        assert np.abs(Wm - ref).max() <= 1e-10 * np.abs(ref).max()


def test_sign_pattern_fails_for_a_nonsymmetric_front():
    """The same sweep on the operator without D: the pattern does not hold
    (the pin tells the symmetric form from the assembled operator)."""
    w = W.random_medium(60, 24, ppw=16, seed=5, npml=6, nsub=2, overlap=3, interface_pml=6, nsrc=1)
    P = Problem.from_workload(w)
    D = DDM.from_workload(w, P)
    A = D.local_A(0).toarray()
    idx = np.arange(40)
    F = A[np.ix_(idx, idx)] + 3.0 * np.eye(40) * np.abs(A).max()
    seen = []

    def check(Wm, kdone):
        elim = np.arange(40) < kdone
        sigma = np.where(elim[:, None] != elim[None, :], -1.0, 1.0)
        seen.append(np.abs(Wm.T - sigma * Wm).max() / np.abs(Wm).max())

    _gj_blocked(F, 28, 4, check)
    assert max(seen) > 1e-6
