"""stdd_residual_noalloc: the residual for callers that cannot allocate.

Some callers may not call cudaMalloc when they need a residual: real-time
loops that reserve all of their device memory before they start, or host
applications that hand out GPU memory only through their own pool.  For them
the library offers stdd_residual_noalloc, which uses a fixed scratch array
compiled into the library instead of allocating.  This test calls it through
the C ABI twice in a row, on different inputs, and checks each result
against the oracle's assembled operator (b - A x, element by element, and
the norm ratio) and against the allocating stdd_residual; it also checks
the output-aliasing rules, the size limit and the set-up requirement.  The
file name makes pytest collect it after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle.fdfd import Problem  # noqa: E402

DEV = "cuda:0"


def test_noalloc_residual_matches_oracle_and_allocating_residual_twice():
    from paper_2509_20801_gb300 import Solver, stdd_residual, stdd_residual_noalloc
    w = W.random_medium(203, 77, ppw=16, seed=21, npml=8, nsub=4, overlap=5, interface_pml=9, nsrc=2)
    A = Problem.from_workload(w).A
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV))
    n = w.n
    b_h = w.b[0].ravel().copy()
    b = torch.from_numpy(b_h).to(DEV)
    xs = [W.random_vector(n, seed=31)[0], W.random_vector(n, seed=32)[0] * 1e-3]
    for x_h in xs:                       # two calls in a row on the shared scratch
        x = torch.from_numpy(x_h).to(DEV)
        r_ref = torch.empty(n, dtype=torch.complex128, device=DEV)
        rel_ref = stdd_residual(s.ctx, x, b, r_ref)
        r = torch.full((n,), float("nan"), dtype=torch.complex128, device=DEV)
        rel = stdd_residual_noalloc(s.ctx, x, b, r)
        torch.cuda.synchronize()
        r_h = r.cpu().numpy()
        # against the oracle: the residual of the assembled operator
        r_or = b_h - A @ x_h
        scale = np.abs(r_or).max()
        assert np.abs(r_h - r_or).max() <= 1e-13 * scale
        rel_or = np.linalg.norm(r_or) / np.linalg.norm(b_h)
        assert rel == pytest.approx(rel_or, rel=1e-12)
        # against the allocating entry point
        assert float(torch.max(torch.abs(r - r_ref))) <= 1e-13 * scale
        assert rel == pytest.approx(rel_ref, rel=1e-12)
    # output in the right-hand side's buffer: allowed, same values
    x_h = xs[0]
    x = torch.from_numpy(x_h).to(DEV)
    bb = b.clone()
    rel_b = stdd_residual_noalloc(s.ctx, x, bb, bb)
    torch.cuda.synchronize()
    r_or = b_h - A @ x_h
    assert np.abs(bb.cpu().numpy() - r_or).max() <= 1e-13 * np.abs(r_or).max()
    assert rel_b == pytest.approx(np.linalg.norm(r_or) / np.linalg.norm(b_h), rel=1e-12)
    s.close()


def test_noalloc_residual_rejects_bad_use():
    from paper_2509_20801_gb300 import (Solver, StddError, stdd_create, stdd_destroy, stdd_residual_noalloc,
                                        stdd_set_grid)
    ctx = stdd_create(0)
    x, b, r = (torch.zeros(64, dtype=torch.complex128, device=DEV) for _ in range(3))
    stdd_set_grid(ctx, 8, 8, 0.1, 0.1)
    with pytest.raises(StddError) as e:    # operator not set up yet
        stdd_residual_noalloc(ctx, x, b, r)
    assert e.value.status == 2
    stdd_set_grid(ctx, 8192, 8193, 0.1, 0.1)   # 67,117,056 nodes > the fixed scratch
    with pytest.raises(StddError) as e:
        stdd_residual_noalloc(ctx, x, b, r)    # (refused before the buffers are touched)
    assert e.value.status == 1 and "67,108,864" in str(e.value)
    stdd_destroy(ctx)
    # output overlapping the field (in place, or shifted by one node) and a
    # partial overlap with the right-hand side are refused before any launch
    w = W.random_medium(40, 30, ppw=16, seed=22, npml=6, nsub=2, overlap=3, interface_pml=6, nsrc=1)
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV))
    n = w.n
    buf = torch.from_numpy(W.random_vector(2 * n, seed=33)[0]).to(DEV)
    b = torch.from_numpy(w.b[0].ravel().copy()).to(DEV)
    for x_, b_, r_ in [(buf[:n], b, buf[:n]), (buf[:n], b, buf[1:n + 1]), (buf[n:], buf[:n], buf[1:n + 1])]:
        with pytest.raises(StddError) as e:
            stdd_residual_noalloc(s.ctx, x_, b_, r_)
        assert e.value.status == 1 and "overlap" in str(e.value)
    s.close()
