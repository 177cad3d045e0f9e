"""The mixed-precision waveguide-network case on the GPU.  Small network
(768 x 384, 4 strips): every precision against the oracle's direct solve
(FP64 to 1e-9; complex64 factors, SIMT or BF16 / FP16 tensor-core updates,
to 1e-7 at a final residual of 1e-8), and static pivoting, which changes
the preconditioner but not the solution.  Full size (8192 x 2048, 32
strips): the complex64 solve with static pivoting (the driver's default),
its residual recomputed with the oracle's own assembled operator, and its
field against the FP64 GPU field."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle.fdfd import Problem  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small():
    w = W.waveguide_network(768, 384, nsub=4, npml=24, overlap=8, interface_pml=24)
    P = Problem.from_workload(w)
    return w, P, P.solve(w.b[0].ravel())


@pytest.mark.parametrize("order", ["red-black", "additive"])
def test_small_network_fp64_matches_oracle(small, order):
    from paper_2509_20801_gb300 import waveguide
    w, P, ref = small
    rows, fields, _ = waveguide.run(workload=w, precisions=("fp64",), order=order, rtol=1e-12, maxit=400,
                                    keep_fields=True, out=open("/dev/null", "w"))
    assert rows[0]["converged"]
    assert _rel(fields["fp64"].ravel(), ref) <= 1e-9


def test_small_network_mixed_matches_oracle(small):
    from paper_2509_20801_gb300 import waveguide
    w, P, ref = small
    rows, fields, _ = waveguide.run(workload=w, precisions=("c64", "fp16", "bf16"), order="red-black",
                                    rtol=1e-8, maxit=400, keep_fields=True, out=open("/dev/null", "w"))
    for r in rows:
        assert r["converged"] and r["final_residual"] <= 1e-8, r
        got = fields[r["precision"]].ravel()
        rel_res = np.linalg.norm(w.b[0].ravel() - P.A @ got) / np.linalg.norm(w.b[0])
        assert rel_res <= 1e-8 * (1 + 1e-6), (r["precision"], rel_res)
        assert _rel(got, ref) <= 1e-7, (r["precision"], _rel(got, ref))


@pytest.mark.parametrize("precision,k,tol", [("fp64", 1, 1e-9), ("c64", 2, 1e-7), ("fp16", 2, 1e-7)])
def test_static_pivoting_keeps_the_solution(small, precision, k, tol):
    from paper_2509_20801_gb300 import waveguide
    w, P, ref = small
    rtol = 1e-12 if precision == "fp64" else 1e-8
    rows, fields, _ = waveguide.run(workload=w, precisions=(precision,), order="multiplicative", rtol=rtol,
                                    maxit=400, keep_fields=True, out=open("/dev/null", "w"), static_pivot=k)
    r = rows[0]
    assert r["converged"] and r["static_pivot"] == (k if precision != "fp64" else 0)
    assert _rel(fields[precision].ravel(), ref) <= tol


@pytest.mark.parametrize("order", ["red-black", "multiplicative"])
def test_small_network_pivoting_without_floor(small, order):
    """Partial pivoting within the fronts, no static-pivot floor: complex64
    factors with FP32, FP16 and BF16 updates reach a true residual of 1e-8
    and the oracle's direct solution within 1e-7; FP64 factors within 1e-9."""
    from paper_2509_20801_gb300 import waveguide
    w, P, ref = small
    rows, fields, _ = waveguide.run(workload=w, precisions=("fp64", "c64", "fp16", "bf16"), order=order,
                                    rtol=1e-8, maxit=400, keep_fields=True, out=open("/dev/null", "w"),
                                    static_pivot=0, pivoting=1)
    for r in rows:
        assert r["pivoting"] == 1 and r["static_pivot"] == 0 and r["raised_pivots"] == 0
        assert r["converged"] and r["final_residual"] <= 1e-8, r
        got = fields[r["precision"]].ravel()
        rel_res = np.linalg.norm(w.b[0].ravel() - P.A @ got) / np.linalg.norm(w.b[0])
        assert rel_res <= 1e-8 * (1 + 1e-6), (r["precision"], rel_res)
        tol = 1e-9 if r["precision"] == "fp64" else 1e-7
        assert _rel(got, ref) <= max(tol, 20 * rel_res), (r["precision"], _rel(got, ref))


def test_pivoting_option_checks():
    from paper_2509_20801_gb300 import STDD_OPT_PIVOTING, Solver, StddError, stdd_set_option
    w = W.waveguide_network(768, 384, nsub=4, npml=24, overlap=8, interface_pml=24)
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to("cuda:0"), precision=1)
    for bad in (-1, 2):
        with pytest.raises(StddError) as e:
            stdd_set_option(s.ctx, STDD_OPT_PIVOTING, bad)
        assert e.value.status == 1
    s.close()


def test_static_pivot_option_and_count():
    from paper_2509_20801_gb300 import STDD_OPT_STATIC_PIVOT, Solver, StddError, stdd_set_option
    w = W.waveguide_network(768, 384, nsub=4, npml=24, overlap=8, interface_pml=24)
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to("cuda:0"), precision=1)
    with pytest.raises(StddError):
        stdd_set_option(s.ctx, STDD_OPT_STATIC_PIVOT, 16)
    s.factor()
    assert s.stats()["raised_pivots"] == 0            # off by default
    counts = []
    for k in (3, 2, 1):
        stdd_set_option(s.ctx, STDD_OPT_STATIC_PIVOT, k)
        s.factor()
        counts.append(s.stats()["raised_pivots"])
    # a higher floor raises at least the pivots a lower one did
    assert counts[0] <= counts[1] <= counts[2] and counts[2] > 0
    s.close()


def test_fullsize_network_mixed_precision():
    from paper_2509_20801_gb300 import waveguide
    w = W.waveguide_network()
    assert (w.nx, w.ny, w.nsub, w.overlap, w.interface_pml, w.npml[0]) == (8192, 2048, 32, 16, 32, 32)
    rows, fields, _ = waveguide.run(workload=w, precisions=("fp64", "c64"), rtol=1e-8,
                                    keep_fields=True, out=open("/dev/null", "w"))
    P = Problem.from_workload(w)
    b = w.b[0].ravel()
    for r in rows:
        assert r["converged"], r
        rel_res = np.linalg.norm(b - P.A @ fields[r["precision"]].ravel()) / np.linalg.norm(b)
        assert rel_res <= 1e-8 * (1 + 1e-6), (r["precision"], rel_res)
    assert rows[1]["diff_vs_fp64"] <= 1e-7
