"""stdd_residual_noalloc: the residual for callers that cannot allocate.

Some callers may not call cudaMalloc when they need a residual (work built
into a CUDA graph, real-time loops with all memory reserved up front, hosts
that hand out GPU memory only from their own pool).  For them the library
offers stdd_residual_noalloc, which uses a fixed scratch array compiled into
the library instead of allocating.  This test calls it through the C ABI
twice in a row, on different inputs, and checks each result against the
allocating stdd_residual; it also checks the size limit and the set-up
requirement.  The file name makes pytest collect it after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402

DEV = "cuda:0"


def test_noalloc_residual_matches_allocating_residual_twice():
    from paper_2509_20801_gb300 import Solver, stdd_residual, stdd_residual_noalloc
    w = W.random_medium(203, 77, ppw=16, seed=21, npml=8, nsub=4, overlap=5, interface_pml=9, nsrc=2)
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV))
    n = w.n
    b = torch.from_numpy(w.b[0].ravel().copy()).to(DEV)
    inputs = [torch.from_numpy(W.random_vector(n, seed=31)[0]).to(DEV),
              torch.from_numpy(W.random_vector(n, seed=32)[0] * 1e-3).to(DEV)]
    for x in inputs:                       # two calls in a row on the shared scratch
        r_ref = torch.empty(n, dtype=torch.complex128, device=DEV)
        rel_ref = stdd_residual(s.ctx, x, b, r_ref)
        r = torch.full((n,), float("nan"), dtype=torch.complex128, device=DEV)
        rel = stdd_residual_noalloc(s.ctx, x, b, r)
        torch.cuda.synchronize()
        scale = float(torch.max(torch.abs(r_ref)))
        assert float(torch.max(torch.abs(r - r_ref))) <= 1e-13 * scale
        assert rel == pytest.approx(rel_ref, rel=1e-12)
        assert np.isfinite(rel) and rel > 0
    s.close()


def test_noalloc_residual_rejects_bad_use():
    from paper_2509_20801_gb300 import StddError, stdd_create, stdd_destroy, stdd_residual_noalloc, stdd_set_grid
    ctx = stdd_create(0)
    x = torch.zeros(4, dtype=torch.complex128, device=DEV)
    stdd_set_grid(ctx, 8, 8, 0.1, 0.1)
    with pytest.raises(StddError) as e:    # operator not set up yet
        stdd_residual_noalloc(ctx, x, x, x)
    assert e.value.status == 2
    stdd_set_grid(ctx, 8192, 8193, 0.1, 0.1)   # 67,117,056 nodes > the fixed scratch
    with pytest.raises(StddError) as e:
        stdd_residual_noalloc(ctx, x, x, x)
    assert e.value.status == 1 and "67,108,864" in str(e.value)
    stdd_destroy(ctx)
