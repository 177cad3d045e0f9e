"""The batched uneven workload: many seeded ellipse geometries of different
sizes, each with several point sources, solved one geometry after another on
one stream (within a geometry the kernels are batched over all strips, fronts
and right-hand sides and the preconditioner is replayed as a CUDA graph).

Geometry g uses seed 3 * 1_000_000 + g; its size is drawn (seed 3) from the
given shapes, its strips from [2, min(8, nx / 128)].  Per geometry: factor and
solve times (CUDA events), iterations, and the true residual of every field
(library residual call).  The summary reports the throughput over the whole
batch, MDoF/s = sum of nx * ny * nrhs / total time.

    python -m paper_2509_20801_gb300.batched [--count 48] [--nrhs 8] [--precision c64]
        [--order additive|multiplicative|red-black] [--restart m] [--maxit k] [--static-pivot k]
        [--pivoting 0|1] [--workers k]

With --workers k > 1 the geometries run k at a time, each on its own context
and CUDA stream driven by its own host thread, so that the GPU overlaps them.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import binding as _b

SHAPES = ((256, 256), (512, 512), (1024, 512), (2048, 512), (2048, 1024))
PRECISIONS = {"fp64": _b.STDD_PREC_FP64, "c64": _b.STDD_PREC_C64}
ORDERS = {"additive": 0, "multiplicative": 1, "red-black": 2}


def geometries(count=48, nrhs=8, shapes=SHAPES, seed=3):
    import workloads as W
    rng = np.random.default_rng(seed)
    picks = rng.integers(0, len(shapes), count)
    return [W.ellipses(shapes[k][0], shapes[k][1], seed=seed * 1_000_000 + g, nrhs=nrhs, sources="point")
            for g, k in enumerate(picks)]


def _solve_one(g, w, precision, rtol, restart, maxit, device, order, static_pivot, pivoting):
    """Factor and solve geometry g on its own context (and so its own CUDA
    stream); host wall times of both phases (each library call returns when
    its work is done)."""
    import torch
    from . import Solver
    dev = torch.device("cuda", device)
    s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(dev), precision=PRECISIONS[precision],
                             device=device)
    _b.stdd_set_option(s.ctx, _b.STDD_OPT_ORDER, ORDERS[order])
    _b.stdd_set_option(s.ctx, _b.STDD_OPT_STATIC_PIVOT, static_pivot)
    _b.stdd_set_option(s.ctx, _b.STDD_OPT_PIVOTING, pivoting)
    _b.stdd_set_option(s.ctx, _b.STDD_OPT_PERSISTENT, 0)   # concurrent contexts: no co-residency needs
    try:
        b = torch.from_numpy(w.b).to(dev)      # a pageable copy: complete on return
        x = torch.empty_like(b)
        t0 = time.perf_counter()
        s.factor()
        t1 = time.perf_counter()
        s.set_sources(b)
        st = s.solve(x, restart=restart, rtol=rtol, maxit=maxit, allow_noconv=True)
        t2 = time.perf_counter()
        r = torch.empty(w.n, dtype=torch.complex128, device=dev)
        res = [_b.stdd_residual(s.ctx, x[q].reshape(-1).contiguous(), b[q].reshape(-1).contiguous(), r)
               for q in range(w.nrhs)]
        its = [len(s.history(q)) - 1 for q in range(w.nrhs)]
        return dict(g=g, nx=w.nx, ny=w.ny, nsub=w.nsub, nrhs=w.nrhs, factor_ms=(t1 - t0) * 1e3,
                    solve_ms=(t2 - t1) * 1e3, iterations_max=max(its), iterations_mean=float(np.mean(its)),
                    converged=st == _b.STDD_OK, max_true_residual=float(max(res)),
                    raised_pivots=s.stats()["raised_pivots"])
    finally:
        s.close()


def run_concurrent(count=48, nrhs=8, precision="c64", rtol=1e-8, restart=30, maxit=1000, device=0,
                   shapes=SHAPES, out=None, log=None, order="additive", static_pivot=0, pivoting=1, workers=4):
    """The same batch with `workers` geometries in flight at once: each on
    its own context and CUDA stream, driven by its own host thread (the
    library's calls release the Python interpreter), largest geometries
    first, so the GPU overlaps the small geometries' kernels with the large
    ones'.  Throughput = sum of nx * ny * nrhs / wall time of the batch."""
    import concurrent.futures as cf

    import torch
    ws = geometries(count, nrhs, shapes)
    torch.cuda.synchronize(device)
    order_g = sorted(range(len(ws)), key=lambda g: -ws[g].n)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(_solve_one, g, ws[g], precision, rtol, restart, maxit, device, order, static_pivot,
                          pivoting) for g in order_g]
        rows = [f.result() for f in futs]
    torch.cuda.synchronize(device)
    wall = time.perf_counter() - t0
    rows.sort(key=lambda r: r["g"])
    if out:
        for row in rows:
            print(json.dumps(row), file=out, flush=True)
    dof = sum(r["nx"] * r["ny"] * r["nrhs"] for r in rows)
    summary = dict(geometries=len(rows), rhs_per_geometry=nrhs, precision=precision, order=order, restart=restart,
                   static_pivot=static_pivot, pivoting=pivoting, workers=workers, maxit=maxit, rtol=rtol,
                   unknowns=sum(r["nx"] * r["ny"] for r in rows), dof_rhs=dof, wall_ms=wall * 1e3,
                   mdof_per_s=dof / wall / 1e6, all_converged=all(r["converged"] for r in rows),
                   max_true_residual=max(r["max_true_residual"] for r in rows),
                   iterations_mean=float(np.mean([r["iterations_mean"] for r in rows])))
    return rows, summary


def run(count=48, nrhs=8, precision="c64", rtol=1e-8, restart=30, maxit=1000, device=0, shapes=SHAPES,
        out=None, log=None, order="additive", static_pivot=0, pivoting=0):
    import torch
    from . import Solver
    dev = torch.device("cuda", device)
    t0 = time.perf_counter()
    ws = geometries(count, nrhs, shapes)
    if log:
        log(f"{len(ws)} geometries: {time.perf_counter() - t0:.1f} s")
    rows = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for g, w in enumerate(ws):
        s = Solver.from_workload(w, eps=torch.from_numpy(w.eps_node).to(dev), precision=PRECISIONS[precision],
                                 device=device)
        _b.stdd_set_option(s.ctx, _b.STDD_OPT_ORDER, ORDERS[order])
        _b.stdd_set_option(s.ctx, _b.STDD_OPT_STATIC_PIVOT, static_pivot)
        _b.stdd_set_option(s.ctx, _b.STDD_OPT_PIVOTING, pivoting)
        try:
            b = torch.from_numpy(w.b).to(dev)
            x = torch.empty_like(b)
            torch.cuda.synchronize(dev)
            ev[0].record()
            s.factor()
            ev[1].record()
            s.set_sources(b)
            st = s.solve(x, restart=restart, rtol=rtol, maxit=maxit, allow_noconv=True)
            ev[2].record()
            torch.cuda.synchronize(dev)
            r = torch.empty(w.n, dtype=torch.complex128, device=dev)
            res = [_b.stdd_residual(s.ctx, x[q].reshape(-1).contiguous(), b[q].reshape(-1).contiguous(), r)
                   for q in range(w.nrhs)]
            its = [len(s.history(q)) - 1 for q in range(w.nrhs)]
            row = dict(g=g, nx=w.nx, ny=w.ny, nsub=w.nsub, nrhs=w.nrhs, factor_ms=ev[0].elapsed_time(ev[1]),
                       solve_ms=ev[1].elapsed_time(ev[2]), iterations_max=max(its),
                       iterations_mean=float(np.mean(its)), converged=st == _b.STDD_OK,
                       max_true_residual=float(max(res)), raised_pivots=s.stats()["raised_pivots"])
        finally:
            s.close()
        rows.append(row)
        if out:
            print(json.dumps(row), file=out, flush=True)
    dof = sum(r["nx"] * r["ny"] * r["nrhs"] for r in rows)
    tms = sum(r["factor_ms"] + r["solve_ms"] for r in rows)
    summary = dict(geometries=len(rows), rhs_per_geometry=nrhs, precision=precision, order=order, restart=restart,
                   static_pivot=static_pivot, pivoting=pivoting,
                   maxit=maxit, rtol=rtol,
                   unknowns=sum(r["nx"] * r["ny"] for r in rows), dof_rhs=dof, total_ms=tms,
                   factor_ms=sum(r["factor_ms"] for r in rows), solve_ms=sum(r["solve_ms"] for r in rows),
                   mdof_per_s=dof / (tms * 1e-3) / 1e6, all_converged=all(r["converged"] for r in rows),
                   max_true_residual=max(r["max_true_residual"] for r in rows),
                   iterations_mean=float(np.mean([r["iterations_mean"] for r in rows])))
    return rows, summary


if __name__ == "__main__":
    import argparse
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="batched uneven workload: many geometries, several sources each")
    ap.add_argument("--count", type=int, default=48)
    ap.add_argument("--nrhs", type=int, default=8)
    ap.add_argument("--precision", default="c64", choices=sorted(PRECISIONS))
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--order", default="additive", choices=sorted(ORDERS))
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--maxit", type=int, default=1000)
    ap.add_argument("--static-pivot", type=int, default=0)
    ap.add_argument("--pivoting", type=int, default=0, choices=[0, 1])
    ap.add_argument("--workers", type=int, default=1,
                    help="geometries in flight at once (each on its own context and stream); 1: one after another")
    a = ap.parse_args()
    if a.workers > 1:
        _, summ = run_concurrent(a.count, a.nrhs, a.precision, a.rtol, a.restart, a.maxit, out=sys.stderr,
                                 order=a.order, static_pivot=a.static_pivot, pivoting=a.pivoting, workers=a.workers)
    else:
        _, summ = run(a.count, a.nrhs, a.precision, a.rtol, a.restart, a.maxit, out=sys.stderr,
                      log=lambda m: print(m, file=sys.stderr, flush=True), order=a.order,
                      static_pivot=a.static_pivot, pivoting=a.pivoting)
    print(json.dumps(summ))
