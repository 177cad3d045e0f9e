"""CPU-only checks of the GPU library's host side.

* libstdd.so loads and exports every entry point that include/stdd.h
  declares (parsed from the header, compared with the binding).
* The nested-dissection analysis (host C++) yields a valid elimination: every
  node is a pivot exactly once, each front's border is exactly the set of
  stencil neighbours of its subtree outside the subtree, and all border nodes
  are pivots of ancestors.
* A numpy multifrontal elimination driven by the exported fronts reproduces
  the direct solution of a strip operator (so the ordering, front index sets
  and extend-add relations the kernels use are right), with no pivoting.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stdd.h")


def _lib():
    try:
        from paper_2509_20801_gb300 import binding
    except ImportError as e:  # pragma: no cover - build() runs before the tests
        pytest.fail(f"library not built: {e}")
    return binding


def test_header_symbols_exported():
    b = _lib()
    decl = re.findall(r"\b(stdd_[a-z_0-9]+)\s*\(", open(HEADER).read())
    declared = sorted(set(decl))
    assert set(declared) == set(b.EXPORTED)
    for name in declared:
        assert hasattr(b.lib, name)


def test_create_without_gpu_reports_status():
    import ctypes
    b = _lib()
    import torch
    ctx = ctypes.c_void_p()
    st = b.lib.stdd_create(ctypes.byref(ctx), 0, None)
    if torch.cuda.is_available():
        assert st == b.STDD_OK
        b.lib.stdd_destroy(ctx)
    else:
        assert st == b.STDD_ECUDA and not ctx.value


def _fronts(W, H, leaf):
    b = _lib()
    r = b.stdd_nd_analyze(W, H, leaf)
    out = []
    off = 0
    for f in range(len(r["p"])):
        p, bb = int(r["p"][f]), int(r["b"][f])
        out.append(dict(p=p, b=bb, parent=int(r["parent"][f]), level=int(r["level"][f]),
                        piv=r["nodes"][off:off + p].copy(), ring=r["nodes"][off + p:off + p + bb].copy()))
        off += p + bb
    return out


@pytest.mark.parametrize("W,H,leaf", [(17, 23, 8), (40, 30, 16), (128, 200, 64), (5, 64, 4)])
def test_nested_dissection_structure(W, H, leaf):
    fr = _fronts(W, H, leaf)
    owner = -np.ones(W * H, int)
    for f, d in enumerate(fr):
        assert d["p"] > 0
        assert np.all(owner[d["piv"]] < 0)
        owner[d["piv"]] = f
    assert np.all(owner >= 0)
    assert sum(d["parent"] < 0 for d in fr) == 1
    # subtree node sets, children before parents
    sub = [set(d["piv"].tolist()) for d in fr]
    for f, d in enumerate(fr):
        if d["parent"] >= 0:
            assert d["parent"] > f
            assert fr[d["parent"]]["level"] == d["level"] - 1
            sub[d["parent"]] |= sub[f]
    for f, d in enumerate(fr):
        nb = set()
        for node in sub[f]:
            x, y = divmod(node, H)
            for xx, yy in ((x - 1, y), (x + 1, y), (x, y - 1), (x, y + 1)):
                if 0 <= xx < W and 0 <= yy < H and xx * H + yy not in sub[f]:
                    nb.add(xx * H + yy)
        assert set(d["ring"].tolist()) == nb
        anc = set()
        a = d["parent"]
        while a >= 0:
            anc |= set(fr[a]["piv"].tolist())
            a = fr[a]["parent"]
        assert nb <= anc


def test_metalens_strip_shape_matches_derivation():
    # the interior strip of the 4096 x 1024 metalens case: 256 owned columns
    # plus 2 x (12 overlap + 30 PML) = 340 columns
    fr = _fronts(340, 1024, 64)
    assert len(fr) == 13589
    assert max(d["p"] for d in fr) == 340 and max(d["b"] for d in fr) == 680
    assert max(d["level"] for d in fr) == 13


def _multifrontal_solve(A, fronts, t, floor=0.0, raised=None, pivots=None):
    """Dense-front elimination (no pivoting) with extend-add by node id.
    With floor > 0 a pivot of modulus below it is replaced by floor times its
    phase (static pivoting); (node, change) pairs go to ``raised`` and every
    pivot's modulus to ``pivots``."""
    A = A.tocsr()
    schur = {}
    facs = []
    for f, d in enumerate(fronts):
        idx = np.concatenate([d["piv"], d["ring"]])
        p = d["p"]
        F = A[idx][:, idx].toarray()
        F[p:, p:] = 0.0                       # ring-ring entries belong to ancestors
        pos = {int(v): k for k, v in enumerate(idx)}
        for c in [c for c in range(f) if fronts[c]["parent"] == f]:
            cidx, S = schur.pop(c)
            m = np.array([pos[int(v)] for v in cidx])
            F[np.ix_(m, m)] += S
        F11, F12, F21 = F[:p, :p], F[:p, p:], F[p:, :p]
        L = np.tril(F11.copy())
        U = np.zeros_like(F11)
        G = F11.copy()
        for k in range(p):                    # right-looking LU, no pivoting
            dv = G[k, k]
            if pivots is not None:
                pivots.append(abs(dv))
            if floor > 0 and abs(dv) < floor:
                G[k, k] = floor * dv / abs(dv) if abs(dv) > 0 else floor
                raised.append((int(idx[k]), G[k, k] - dv))
            U[k, k:] = G[k, k:]
            L[k:, k] = G[k:, k] / G[k, k]
            G[k + 1:, k + 1:] -= np.outer(L[k + 1:, k], U[k, k + 1:])
        L21 = np.linalg.solve(U.T, F21.T).T
        U12 = np.linalg.solve(L, F12)
        schur[f] = (d["ring"], F[p:, p:] - L21 @ U12)
        facs.append((idx, p, L, U, L21, U12))
    x = np.array(t, dtype=complex)
    for idx, p, L, U, L21, U12 in facs:       # forward, leaves to root
        y = np.linalg.solve(L, x[idx[:p]])
        x[idx[:p]] = y
        x[idx[p:]] -= L21 @ y
    for idx, p, L, U, L21, U12 in reversed(facs):
        x[idx[:p]] = np.linalg.solve(U, x[idx[:p]] - U12 @ x[idx[p:]])
    return x


def test_multifrontal_emulation_reproduces_direct_solve():
    import workloads as W
    from oracle.fdfd import Problem
    from oracle.stddm import DDM
    w = W.random_medium(60, 36, ppw=16, seed=2, npml=6, nsub=2, overlap=3, interface_pml=6)
    P = Problem.from_workload(w)
    D = DDM.from_workload(w, P)
    for k in range(2):
        s = D.strips[k]
        fr = _fronts(s.width, P.ny, 16)
        A = D.local_A(k)
        rng = np.random.default_rng(k)
        t = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
        x = _multifrontal_solve(A, fr, t)
        ref = D.local_solve(k, t)
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-11


def test_static_pivoting_factors_a_diagonal_perturbation():
    """Raising small pivots during the elimination (the library's optional
    static pivoting) yields exactly the factors of A + E, E diagonal with
    the raised pivots' changes, checked against SuperLU on A + E."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    import workloads as W
    from oracle.fdfd import Problem
    from oracle.stddm import DDM
    w = W.random_medium(60, 36, ppw=16, seed=2, npml=6, nsub=2, overlap=3, interface_pml=6)
    P = Problem.from_workload(w)
    D = DDM.from_workload(w, P)
    s = D.strips[1]
    fr = _fronts(s.width, P.ny, 16)
    A = D.local_A(1).tocsc()
    t = np.random.default_rng(5).standard_normal(A.shape[0]) + 0j
    mags = []
    _multifrontal_solve(A, fr, t, pivots=mags)
    floor = float(np.quantile(mags, 0.2))       # raise about a fifth of the pivots
    raised = []
    x = _multifrontal_solve(A, fr, t, floor=floor, raised=raised)
    assert 0.1 * len(mags) < len(raised) < 0.3 * len(mags)
    E = np.zeros(A.shape[0], complex)
    for node, delta in raised:
        E[node] += delta
    ref = sla.spsolve((A + sp.diags(E)).tocsc(), t)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-10
    # and it is not the unperturbed solve
    assert np.linalg.norm(x - sla.spsolve(A, t)) > 1e-3 * np.linalg.norm(ref)
