"""GPU parity of the symmetric multiplicative order (STDD_OPT_ORDER = 1)
against the oracle's plain sequential definition, and its use inside FGMRES
(same solution as the direct solve, fewer iterations than the additive
order)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle.fdfd import Problem  # noqa: E402
from oracle.krylov import gmres  # noqa: E402
from oracle.stddm import DDM  # noqa: E402

DEV = "cuda:0"


def _solver(w, precision=0, order=1):
    from paper_2509_20801_gb300 import STDD_OPT_ORDER, Solver, stdd_set_option
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV), precision=precision)
    stdd_set_option(s.ctx, STDD_OPT_ORDER, order)
    return s


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def rnd():
    # ragged: nx not a multiple of nsub, odd ny, 4 strips of different widths
    w = W.random_medium(203, 77, ppw=16, seed=21, npml=8, nsub=4, overlap=5, interface_pml=9, nsrc=2)
    P = Problem.from_workload(w)
    return w, P, DDM.from_workload(w, P)


@pytest.fixture(scope="module")
def strip6():
    w = W.cylinder(nx=240, ny=60, ppw=20, npml=10, nsub=6, overlap=4, interface_pml=10, radius=0.4)
    P = Problem.from_workload(w)
    return w, P, DDM.from_workload(w, P)


@pytest.mark.parametrize("order,graphs", [(1, 1), (1, 0), (2, 1), (2, 0), (3, 1), (3, 0)])
def test_multiplicative_preconditioner_matches_oracle(rnd, order, graphs):
    from paper_2509_20801_gb300 import STDD_OPT_GRAPHS, stdd_apply_preconditioner, stdd_set_option
    w, P, D = rnd
    s = _solver(w, order=order)
    stdd_set_option(s.ctx, STDD_OPT_GRAPHS, graphs)
    s.factor()
    v = W.random_vector(P.n, seed=6)[0]
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    stdd_apply_preconditioner(s.ctx, torch.from_numpy(v).to(DEV), z)
    ref = D.apply_Minv_multiplicative(v, order={1: None, 2: "red-black", 3: list(range(w.nsub))}[order])
    assert _rel(z.cpu().numpy(), ref) < 1e-10
    s.close()


def test_order_switch_back_and_forth(rnd):
    from paper_2509_20801_gb300 import STDD_OPT_ORDER, stdd_apply_preconditioner, stdd_set_option
    w, P, D = rnd
    s = _solver(w, order=0)
    s.factor()
    v = torch.from_numpy(W.random_vector(P.n, seed=7)[0]).to(DEV)
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    outs = []
    for order in (0, 1, 0, 1):
        stdd_set_option(s.ctx, STDD_OPT_ORDER, order)
        stdd_apply_preconditioner(s.ctx, v, z)
        outs.append(z.cpu().numpy().copy())
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])
    assert _rel(outs[0], D.apply_Minv(v.cpu().numpy())) < 1e-10
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_fgmres_with_multiplicative_order(strip6, precision):
    w, P, D = strip6
    b = torch.from_numpy(w.b).to(DEV)
    ref = P.solve(w.b[0].ravel())
    its = {}
    for order in (0, 1, 2, 3):
        s = _solver(w, precision=precision, order=order)
        s.factor()
        s.set_sources(b)
        x = torch.empty_like(b)
        s.solve(x, restart=40, rtol=1e-12, maxit=300)
        err = _rel(x[0].cpu().numpy().ravel(), ref)
        assert err <= (1e-9 if precision == 0 else 1e-7), (order, err)
        its[order] = len(s.history(0)) - 1
        s.close()
    # the oracle's FGMRES with the same order takes the same count
    _, oh, _ = gmres(P.matvec, D.apply_Minv_multiplicative, w.b[0].ravel(), restart=40, rtol=1e-12, maxit=300,
                     flexible=True)
    if precision == 0:
        assert abs(its[1] - (len(oh) - 1)) <= 1
    assert its[1] < its[2] < its[0]
    # the forward sweep alone: fewer iterations than the additive order, at
    # most twice the symmetric sweep's (each application does half its work)
    assert its[3] < its[0] and its[3] <= 2 * its[1] + 1


@pytest.mark.parametrize("order", [1, 3])
def test_persistent_sweeps_equal_per_level_launches(rnd, order):
    """The persistent one-strip sweep (one cooperative launch per strip solve,
    levels separated by grid barriers) runs the same device code as the
    per-level launches: bitwise equal results, with and without graphs."""
    from paper_2509_20801_gb300 import (STDD_OPT_GRAPHS, STDD_OPT_PERSISTENT, stdd_apply_preconditioner,
                                        stdd_set_option)
    w, P, D = rnd
    v = torch.from_numpy(W.random_vector(P.n, seed=15)[0]).to(DEV)
    outs = []
    for persistent, graphs in ((1, 1), (0, 1), (1, 0)):
        s = _solver(w, order=order)
        stdd_set_option(s.ctx, STDD_OPT_PERSISTENT, persistent)
        stdd_set_option(s.ctx, STDD_OPT_GRAPHS, graphs)
        s.factor()
        z = torch.empty_like(v)
        for _ in range(2):
            stdd_apply_preconditioner(s.ctx, v, z)
        outs.append(z.cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_persistent_sweep_wait_gives_up_and_recovers(rnd):
    """A grid-barrier wait that runs out (one poll allowed) makes the
    application return STDD_ETIMEOUT without faulting; with the default limit
    the same context then applies the preconditioner correctly."""
    from paper_2509_20801_gb300 import (STDD_OPT_PERSISTENT, STDD_OPT_SWEEP_WAIT, StddError, stdd_apply_preconditioner,
                                        stdd_set_option)
    w, P, D = rnd
    s = _solver(w, order=1)
    stdd_set_option(s.ctx, STDD_OPT_PERSISTENT, 2)   # complex128 factors default to per-level launches
    s.factor()
    v_h = W.random_vector(P.n, seed=16)[0]
    v = torch.from_numpy(v_h).to(DEV)
    z = torch.empty_like(v)
    stdd_set_option(s.ctx, STDD_OPT_SWEEP_WAIT, 1)
    with pytest.raises(StddError) as e:
        stdd_apply_preconditioner(s.ctx, v, z)
    assert e.value.status == 8
    stdd_set_option(s.ctx, STDD_OPT_SWEEP_WAIT, 0)
    stdd_apply_preconditioner(s.ctx, v, z)
    assert _rel(z.cpu().numpy(), D.apply_Minv_multiplicative(v_h)) < 1e-10
    s.close()
