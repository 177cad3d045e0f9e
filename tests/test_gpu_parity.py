"""GPU parity: every step of the hot path against the CPU oracle.

All inputs are seeded (workloads); the oracle computes every expected value
on the CPU.  Tolerances:
* stencil A x: element-wise relative 1e-13 (same arithmetic, FMA order only);
* local solve A_k^-1 t and M^-1 v (complex128 factors): relative 1e-10 -- a
  different elimination order and no pivoting against SuperLU, on operators
  whose condition numbers reach ~1e3-1e4;
* the whole FGMRES solve (FP64): relative L2 error <= 1e-9 against the global
  direct solution, the spec bar;
* complex64 factors: the FP64 FGMRES still reaches the residual, the error
  against the oracle is bounded by the measured error/residual ratio.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle.fdfd import Problem  # noqa: E402
from oracle.krylov import gmres  # noqa: E402
from oracle.stddm import DDM  # noqa: E402

DEV = "cuda:0"


def _solver(w, precision=0, **kw):
    from paper_2509_20801_gb300 import Solver
    return Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(DEV), precision=precision, **kw)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def cyl():
    w = W.cylinder()
    P = Problem.from_workload(w)
    return w, P, DDM.from_workload(w, P)


@pytest.fixture(scope="module")
def rnd():
    # ragged: nx not a multiple of nsub, odd ny, 4 strips, different widths
    w = W.random_medium(203, 77, ppw=16, seed=21, npml=8, nsub=4, overlap=5, interface_pml=9, nsrc=2)
    P = Problem.from_workload(w)
    return w, P, DDM.from_workload(w, P)


def test_stencil_matches_oracle(cyl, rnd):
    from paper_2509_20801_gb300 import stdd_apply_operator
    for w, P, _ in (cyl, rnd):
        s = _solver(w)
        x = W.random_vector(P.n, seed=3)[0]
        y = torch.empty(P.n, dtype=torch.complex128, device=DEV)
        stdd_apply_operator(s.ctx, torch.from_numpy(x).to(DEV), y)
        ref = P.A @ x
        got = y.cpu().numpy()
        assert np.max(np.abs(got - ref) / (np.abs(ref) + 1e-300)) < 1e-13 or _rel(got, ref) < 1e-15
        # host buffers through the same entry point
        yh = np.empty(P.n, np.complex128)
        stdd_apply_operator(s.ctx, x, yh)
        assert np.array_equal(yh, got)
        s.close()


@pytest.mark.parametrize("which", ["cyl", "rnd"])
def test_local_solves_match_oracle(which, cyl, rnd):
    from paper_2509_20801_gb300 import stdd_local_solve, stdd_strip_info
    w, P, D = {"cyl": cyl, "rnd": rnd}[which]
    s = _solver(w)
    s.factor()
    for k in range(w.nsub):
        info = stdd_strip_info(s.ctx, k)
        st = D.strips[k]
        assert (info["c0"], info["c1"], info["x0"], info["x1"]) == (st.c0, st.c1, st.x0, st.x1)
        t = W.random_vector(st.width * P.ny, seed=10 + k)[0]
        z = torch.empty(st.width * P.ny, dtype=torch.complex128, device=DEV)
        stdd_local_solve(s.ctx, k, torch.from_numpy(t).to(DEV), z)
        ref = D.local_solve(k, t)
        assert _rel(z.cpu().numpy(), ref) < 1e-10
    s.close()


@pytest.mark.parametrize("which", ["cyl", "rnd"])
def test_preconditioner_matches_oracle(which, cyl, rnd):
    from paper_2509_20801_gb300 import stdd_apply_preconditioner
    w, P, D = {"cyl": cyl, "rnd": rnd}[which]
    s = _solver(w)
    s.factor()
    v = W.random_vector(P.n, seed=5)[0]
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    stdd_apply_preconditioner(s.ctx, torch.from_numpy(v).to(DEV), z)
    assert _rel(z.cpu().numpy(), D.apply_Minv(v)) < 1e-10
    s.close()


def test_fgmres_fp64_matches_direct_solution(cyl):
    w, P, D = cyl
    s = _solver(w)
    s.factor()
    b = torch.from_numpy(w.b).to(DEV)
    s.set_sources(b)
    x = torch.empty_like(b)
    s.solve(x, restart=30, rtol=1e-12, maxit=300)
    ref = P.solve(w.b[0].ravel())
    assert _rel(x[0].cpu().numpy().ravel(), ref) <= 1e-9
    hist = s.history(0)
    _, ohist, oits = gmres(P.matvec, D.apply_Minv, w.b[0].ravel(), restart=30, rtol=1e-12)
    assert abs((len(hist) - 1) - oits) <= 1
    assert np.allclose(hist[:4], ohist[:4], rtol=1e-6)
    st = s.stats()
    assert st["final_residual"] <= 1e-12
    s.close()


def test_multiple_rhs_and_ragged_partition(rnd):
    w, P, D = rnd
    s = _solver(w)
    s.factor()
    s.set_sources(torch.from_numpy(w.b).to(DEV))
    x = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, restart=20, rtol=1e-12, maxit=400)
    for r in range(w.nrhs):
        assert _rel(x[r].cpu().numpy().ravel(), P.solve(w.b[r].ravel())) <= 1e-9
    s.close()


def test_explicit_cuts_and_single_strip(cyl):
    w, P, D = cyl
    b = w.b[0].ravel()
    ref = P.solve(b)
    # single strip: M^-1 = A^-1, FGMRES stops after one iteration
    s = _solver(w)
    from paper_2509_20801_gb300 import stdd_set_decomposition
    stdd_set_decomposition(s.ctx, 1, None, 0, 0)
    s.factor()
    s.set_sources(torch.from_numpy(w.b).to(DEV))
    x = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, restart=10, rtol=1e-11, maxit=10)
    assert len(s.history(0)) == 2
    assert _rel(x[0].cpu().numpy().ravel(), ref) <= 1e-10
    # uneven explicit cuts
    stdd_set_decomposition(s.ctx, 3, [0, 50, 130, 200], 6, 12)
    s.factor()
    s.solve(x, restart=30, rtol=1e-12, maxit=300)
    assert _rel(x[0].cpu().numpy().ravel(), ref) <= 1e-9
    s.close()


def test_paper_richardson_matches_algorithm1(cyl):
    w, P, D = cyl
    b = w.b[0].ravel()
    s = _solver(w)
    s.factor()
    s.set_sources(torch.from_numpy(w.b).to(DEV))
    x = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, rtol=1e-12, maxit=3, paper_richardson=True)
    # three sweeps of the residual form == Algorithm 1's partial synthesis
    xs = D.richardson(b, 3)
    assert _rel(x[0].cpu().numpy().ravel(), xs[2]) < 1e-10
    h = s.history(0)
    assert len(h) == 4
    assert abs(h[3] - np.linalg.norm(b - P.A @ xs[2]) / np.linalg.norm(b)) <= 1e-6 * h[3] + 1e-14
    s.close()


def test_complex64_factors_reach_fp64_residual(cyl):
    w, P, D = cyl
    s = _solver(w, precision=1)
    s.factor()
    s.set_sources(torch.from_numpy(w.b).to(DEV))
    x = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x, restart=30, rtol=1e-10, maxit=300)
    got = x[0].cpu().numpy().ravel()
    b = w.b[0].ravel()
    res = np.linalg.norm(b - P.A @ got) / np.linalg.norm(b)
    assert res <= 1.5e-10
    ref = P.solve(b)
    assert _rel(got, ref) <= 1e-7
    s.close()


def test_state_errors():
    from paper_2509_20801_gb300 import StddError, stdd_set_decomposition
    w = W.cylinder()
    s = _solver(w)
    x = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
    with pytest.raises(StddError) as e:
        s.solve(x)
    assert e.value.status in (2,)
    with pytest.raises(StddError) as e:
        stdd_set_decomposition(s.ctx, 4, None, 30, 30)   # extension wider than a strip
    assert e.value.status == 1
    s.factor()
    s.set_sources(torch.from_numpy(w.b).to(DEV))
    st = s.solve(x, restart=5, rtol=1e-14, maxit=2, allow_noconv=True)
    assert st == 7
    s.close()


def test_deterministic(rnd):
    w, P, D = rnd
    outs = []
    for _ in range(2):
        s = _solver(w)
        s.factor()
        s.set_sources(torch.from_numpy(w.b).to(DEV))
        x = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
        s.solve(x, restart=20, rtol=1e-10, maxit=200)
        outs.append(x.cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_graphs_and_autotune_do_not_change_results(rnd):
    """CUDA-graph replay of M^-1 and the autotuned substitution launch shapes
    only change speed: results are bitwise identical with and without them."""
    from paper_2509_20801_gb300 import (STDD_OPT_AUTOTUNE, STDD_OPT_GRAPHS, stdd_apply_preconditioner,
                                        stdd_set_option)
    w, P, D = rnd
    v = torch.from_numpy(W.random_vector(P.n, seed=8)[0]).to(DEV)
    outs = []
    for graphs, tune in ((1, 1), (0, 1), (1, 0), (0, 0)):
        s = _solver(w)
        stdd_set_option(s.ctx, STDD_OPT_GRAPHS, graphs)
        stdd_set_option(s.ctx, STDD_OPT_AUTOTUNE, tune)
        s.factor()
        z = torch.empty_like(v)
        for _ in range(2):                 # second call replays the captured graph
            stdd_apply_preconditioner(s.ctx, v, z)
        s.set_sources(torch.from_numpy(w.b).to(DEV))
        x = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
        s.solve(x, restart=20, rtol=1e-10, maxit=200)
        outs.append((z.cpu().numpy(), x.cpu().numpy()))
        s.close()
    for z, x in outs[1:]:
        assert np.array_equal(z, outs[0][0]) and np.array_equal(x, outs[0][1])


@pytest.mark.parametrize("leaf", [4, 64])
def test_other_leaf_sizes_match_oracle(leaf, cyl):
    from paper_2509_20801_gb300 import STDD_OPT_LEAF, stdd_apply_preconditioner, stdd_set_option
    w, P, D = cyl
    s = _solver(w)
    stdd_set_option(s.ctx, STDD_OPT_LEAF, leaf)
    s.factor()
    v = W.random_vector(P.n, seed=6)[0]
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    stdd_apply_preconditioner(s.ctx, torch.from_numpy(v).to(DEV), z)
    assert _rel(z.cpu().numpy(), D.apply_Minv(v)) < 1e-10
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_rhs_equal_single_rhs(precision):
    """Right-hand sides solved together (lockstep FGMRES, every factor entry
    read once for all of them) give bitwise the same fields as each solved
    alone, and the FP64 ones match the direct solution."""
    w = W.random_medium(150, 64, ppw=16, seed=23, npml=8, nsub=3, overlap=4, interface_pml=8, nsrc=5)
    P = Problem.from_workload(w)
    s = _solver(w, precision=precision)
    s.factor()
    s.set_sources(torch.from_numpy(w.b).to(DEV))
    x_all = torch.empty(w.b.shape, dtype=torch.complex128, device=DEV)
    s.solve(x_all, restart=15, rtol=1e-11, maxit=300)
    for r in range(w.nrhs):
        s.set_sources(torch.from_numpy(w.b[r:r + 1].copy()).to(DEV))
        x1 = torch.empty((1,) + w.b.shape[1:], dtype=torch.complex128, device=DEV)
        s.solve(x1, restart=15, rtol=1e-11, maxit=300)
        assert torch.equal(x1[0], x_all[r])
        if precision == 0:
            assert _rel(x1[0].cpu().numpy().ravel(), P.solve(w.b[r].ravel())) <= 1e-9
    s.close()


@pytest.mark.parametrize("which,leaf", [("cyl", 16), ("rnd", 16), ("rnd", 64), ("cyl", 4)])
def test_pivoting_local_solves_and_preconditioner_match_oracle(which, leaf, cyl, rnd):
    """Partial pivoting within the fronts (STDD_OPT_PIVOTING): the factors
    are those of the same A_k, so every local solve and M^-1 still equal the
    oracle's (SuperLU, 1e-10), for small fronts swept in shared memory (warp
    and CTA per front) and blocked large fronts; rows were interchanged."""
    from paper_2509_20801_gb300 import (STDD_OPT_LEAF, STDD_OPT_PIVOTING, stdd_apply_preconditioner,
                                        stdd_local_solve, stdd_set_option)
    w, P, D = {"cyl": cyl, "rnd": rnd}[which]
    s = _solver(w)
    stdd_set_option(s.ctx, STDD_OPT_LEAF, leaf)
    stdd_set_option(s.ctx, STDD_OPT_PIVOTING, 1)
    s.factor()
    for k in range(w.nsub):
        st = D.strips[k]
        t = W.random_vector(st.width * P.ny, seed=20 + k)[0]
        z = torch.empty(st.width * P.ny, dtype=torch.complex128, device=DEV)
        stdd_local_solve(s.ctx, k, torch.from_numpy(t).to(DEV), z)
        assert _rel(z.cpu().numpy(), D.local_solve(k, t)) < 1e-10
    v = W.random_vector(P.n, seed=6)[0]
    z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
    stdd_apply_preconditioner(s.ctx, torch.from_numpy(v).to(DEV), z)
    assert _rel(z.cpu().numpy(), D.apply_Minv(v)) < 1e-10
    # FGMRES reaches the direct solution
    b = torch.from_numpy(w.b).to(DEV)
    s.set_sources(b)
    x = torch.empty_like(b)
    s.solve(x, restart=30, rtol=1e-12, maxit=400)
    assert _rel(x[0].cpu().numpy().ravel(), P.solve(w.b[0].ravel())) <= 1e-9
    s.close()


def test_pivoting_interchanges_rows_and_is_deterministic(cyl):
    """With pivoting on, the eliminated fronts differ from the unpivoted ones
    (rows were interchanged: M^-1 agrees only to rounding, not bitwise) and
    two factorizations give bitwise equal results."""
    from paper_2509_20801_gb300 import STDD_OPT_PIVOTING, stdd_apply_preconditioner, stdd_set_option
    w, P, D = cyl
    v = torch.from_numpy(W.random_vector(P.n, seed=7)[0]).to(DEV)
    outs = []
    for piv in (0, 1, 1):
        s = _solver(w)
        stdd_set_option(s.ctx, STDD_OPT_PIVOTING, piv)
        s.factor()
        z = torch.empty(P.n, dtype=torch.complex128, device=DEV)
        stdd_apply_preconditioner(s.ctx, v, z)
        outs.append(z.cpu().numpy())
        s.close()
    assert not np.array_equal(outs[0], outs[1]) and _rel(outs[1], outs[0]) < 1e-10
    assert np.array_equal(outs[1], outs[2])


def test_factorization_graph_follows_configuration_changes(rnd):
    """The factorization replays a captured graph; after the permittivity
    (same buffer, new values), the frequency (a value baked into the
    launches) or the pivoting option changes, the next factorization still
    gives the oracle's local solves for the new problem, and repeated
    factorizations are bitwise equal to one without graphs."""
    from paper_2509_20801_gb300 import (STDD_OPT_GRAPHS, STDD_OPT_PIVOTING, stdd_apply_preconditioner,
                                        stdd_set_frequency, stdd_set_option, stdd_set_permittivity)
    w, P, D = rnd
    v_h = W.random_vector(P.n, seed=9)[0]
    v = torch.from_numpy(v_h).to(DEV)
    s = _solver(w)
    ref = _solver(w)
    stdd_set_option(ref.ctx, STDD_OPT_GRAPHS, 0)
    z, zr = torch.empty_like(v), torch.empty_like(v)
    for _ in range(3):                      # capture, then replays
        s.factor()
        stdd_apply_preconditioner(s.ctx, v, z)
    ref.factor()
    stdd_apply_preconditioner(ref.ctx, v, zr)
    assert torch.equal(z, zr)
    # new permittivity values in the same device buffer, then a new frequency
    eps2 = w.eps_node * 1.1
    stdd_set_permittivity(s.ctx, torch.from_numpy(eps2).to(DEV))
    for wl in (w.wavelength, w.wavelength * 1.07):
        stdd_set_frequency(s.ctx, wl)
        for piv in (0, 1):
            stdd_set_option(s.ctx, STDD_OPT_PIVOTING, piv)
            s.factor()
            stdd_apply_preconditioner(s.ctx, v, z)
            P2 = Problem(P.nx, P.ny, P.dx, P.dy, wl, eps2, w.npml, w.pml_order, w.pml_R)
            D2 = DDM(P2, w.nsub, w.overlap, w.interface_pml)
            assert _rel(z.cpu().numpy(), D2.apply_Minv(v_h)) < 1e-10, (wl, piv)
    s.close()
    ref.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_update_tile_shapes_give_identical_factors(cyl, precision):
    """The front update on 64 x 64 and on 32 x 32 tiles (and whatever the
    autotuner picks per level) sums every entry's products in the same order:
    M^-1 bitwise equal, and equal to the oracle's (FP64)."""
    from paper_2509_20801_gb300 import STDD_OPT_LEAF, STDD_OPT_UPDATE_TILE, stdd_apply_preconditioner, stdd_set_option
    w, P, D = cyl
    v_h = W.random_vector(P.n, seed=17)[0]
    v = torch.from_numpy(v_h).to(DEV)
    outs = []
    for tile in (64, 32, 0):
        s = _solver(w, precision=precision)
        stdd_set_option(s.ctx, STDD_OPT_LEAF, 64)       # more blocked (n > 64) fronts
        stdd_set_option(s.ctx, STDD_OPT_UPDATE_TILE, tile)
        s.factor()
        z = torch.empty_like(v)
        stdd_apply_preconditioner(s.ctx, v, z)
        outs.append(z.cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    if precision == 0:
        assert _rel(outs[0], D.apply_Minv(v_h)) < 1e-10


@pytest.mark.parametrize("order", [0, 1])
def test_sweep_splits_give_identical_results(cyl, order):
    """The substitution products summed by one warp per item, by up to eight
    warps of a block, or by one warp per 128-column segment anywhere on the
    GPU (partial sums added by a second launch) add the same segment sums in
    the same order: M^-1 bitwise equal across the forced splits and the
    tuned one, and equal to the oracle's (additive and multiplicative
    orders, per-level and persistent sweeps)."""
    from paper_2509_20801_gb300 import (STDD_OPT_ORDER, STDD_OPT_PERSISTENT, STDD_OPT_SWEEP_SPLIT, StddError,
                                        stdd_apply_preconditioner, stdd_set_option)
    w, P, D = cyl
    v_h = W.random_vector(P.n, seed=18)[0]
    v = torch.from_numpy(v_h).to(DEV)
    outs = []
    for split, persistent in ((1, 0), (8, 0), (16, 0), (0, 0), (16, 2)):
        if persistent and order == 0:
            continue
        s = _solver(w)
        stdd_set_option(s.ctx, STDD_OPT_ORDER, order)
        stdd_set_option(s.ctx, STDD_OPT_PERSISTENT, persistent)
        stdd_set_option(s.ctx, STDD_OPT_SWEEP_SPLIT, split)
        s.factor()
        z = torch.empty_like(v)
        stdd_apply_preconditioner(s.ctx, v, z)
        outs.append(z.cpu().numpy())
        if split == 16:
            with pytest.raises(StddError):
                stdd_set_option(s.ctx, STDD_OPT_SWEEP_SPLIT, 3)
        s.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    ref = D.apply_Minv(v_h) if order == 0 else D.apply_Minv_multiplicative(v_h)
    assert _rel(outs[0], ref) < 1e-10
