"""The batched uneven workload driver: several ellipse geometries of
different sizes with several point sources each, complex64 factors; every
field reaches the tolerance (library residual), and fields of four
geometries of four sizes match the oracle's direct solve to 1e-7."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_batched_driver_small():
    from oracle.fdfd import Problem
    from paper_2509_20801_gb300 import batched
    shapes = ((256, 256), (384, 256))
    rows, summ = batched.run(count=3, nrhs=3, precision="c64", shapes=shapes)
    assert summ["geometries"] == 3 and summ["all_converged"]
    assert summ["max_true_residual"] <= 1e-8
    assert summ["mdof_per_s"] > 0
    # geometry 0, first source: against the oracle (complex64 factors, FP64 Krylov)
    w = batched.geometries(3, 3, shapes)[0]
    from paper_2509_20801_gb300 import STDD_PREC_C64, Solver
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).cuda(), precision=STDD_PREC_C64)
    s.factor()
    b = torch.from_numpy(w.b).cuda()
    s.set_sources(b)
    x = torch.empty_like(b)
    s.solve(x, restart=30, rtol=1e-8, maxit=1000)
    ref = Problem.from_workload(w).solve(w.b[0].ravel())
    assert np.linalg.norm(x[0].cpu().numpy().ravel() - ref) <= 1e-6 * np.linalg.norm(ref)
    s.close()


def test_batched_driver_concurrent_streams_match_sequential():
    """Geometries in flight at once (own contexts and streams, host threads)
    converge like the one-after-another run, with the same iteration counts
    (the same arithmetic per context; the autotuners' launch-shape choices do
    not change results), and with partial pivoting in the fronts."""
    from paper_2509_20801_gb300 import batched
    shapes = ((256, 256), (384, 256), (512, 256))
    rows_s, summ_s = batched.run(count=4, nrhs=2, precision="c64", shapes=shapes, pivoting=1)
    rows_c, summ_c = batched.run_concurrent(count=4, nrhs=2, precision="c64", shapes=shapes, pivoting=1,
                                            workers=3)
    assert summ_c["all_converged"] and summ_c["max_true_residual"] <= 1e-8
    assert [r["g"] for r in rows_c] == [r["g"] for r in rows_s]
    for a, b in zip(rows_s, rows_c):
        assert (a["nx"], a["ny"], a["iterations_max"]) == (b["nx"], b["ny"], b["iterations_max"])
        assert abs(a["max_true_residual"] - b["max_true_residual"]) <= 1e-3 * a["max_true_residual"]


def test_batched_four_sizes_match_oracle_direct_solve():
    """One seeded geometry of each of four grid sizes (the generator of the
    48-geometry workload), complex64 factors with partial pivoting in the
    fronts, FP64 FGMRES to 1e-10: every source's field against the oracle's
    direct solve of the assembled operator, 1e-7."""
    from oracle.fdfd import Problem
    from paper_2509_20801_gb300 import STDD_OPT_PIVOTING, STDD_PREC_C64, Solver, stdd_set_option
    from paper_2509_20801_gb300 import batched
    shapes = ((192, 192), (256, 192), (256, 256), (320, 256))
    for k, sh in enumerate(shapes):
        w = batched.geometries(1, 2, (sh,), seed=11 + k)[0]
        assert (w.nx, w.ny) == sh
        s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).cuda(), precision=STDD_PREC_C64)
        stdd_set_option(s.ctx, STDD_OPT_PIVOTING, 1)
        s.factor()
        b = torch.from_numpy(w.b).cuda()
        s.set_sources(b)
        x = torch.empty_like(b)
        s.solve(x, restart=40, rtol=1e-10, maxit=1000)
        P = Problem.from_workload(w)
        for q in range(w.nrhs):
            ref = P.solve(w.b[q].ravel())
            got = x[q].cpu().numpy().ravel()
            assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref), (sh, q)
        s.close()
