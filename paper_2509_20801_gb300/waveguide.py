"""The mixed-precision single large instance: a silicon-like waveguide network
(8192 x 2048 nodes, 16.8 million unknowns at lambda/24, 32-cell PML, 32
strips with overlap 16, four Y splitters and eight S-bends, excited by the
input guide's fundamental mode) solved to a relative residual of 1e-8 with
complex64 factors (FP32 SIMT or BF16 / FP16 tensor-core front updates) and
the FP64 Krylov iteration, next to the plain FP64 path on the same problem.

For each precision: factorization and solve times (CUDA events around the
library calls; the first factorization of a context includes the one-time
tuning of the substitution launch shapes, so a second factorization is timed
too), FGMRES iterations, the true final residual, MDoF/s over the
whole solve (factor + iterations), the device memory the context held, the
pivots raised by static pivoting and the relative L2 difference of the field
from the FP64 path's field.  One JSON line per precision on stdout.

The complex64 factors use static pivoting with a floor of 1e-2 of the
stencil's diagonal scale by default (``--static-pivot 2``): without it the
unpivoted elimination's growth on this geometry's interior strips leaves the
complex64 local solves with O(1) errors and FGMRES stalls; FP64 factors keep
the plain elimination.  The default order is the symmetric multiplicative
one, which carries the guided waves across all strips in one sweep.

    python -m paper_2509_20801_gb300.waveguide [--nx 8192 --ny 2048 --nsub 32]
        [--precisions fp64,c64,fp16,bf16] [--order additive|multiplicative|red-black]
        [--static-pivot k]
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import binding as _b

PRECISIONS = {"fp64": _b.STDD_PREC_FP64, "c64": _b.STDD_PREC_C64, "bf16": _b.STDD_PREC_C64_BF16,
              "fp16": _b.STDD_PREC_C64_FP16}
ORDERS = {"additive": 0, "multiplicative": 1, "red-black": 2, "forward": 3}


def run(nx=8192, ny=2048, nsub=32, precisions=("fp64", "c64", "fp16"), order="multiplicative", rtol=1e-8,
        restart=50, maxit=600, seed=2, device=0, out=sys.stdout, log=None, workload=None, keep_fields=False,
        static_pivot=2, pivoting=0):
    import torch
    import workloads as W
    from . import Solver
    dev = torch.device("cuda", device)
    t0 = time.perf_counter()
    w = workload if workload is not None else W.waveguide_network(nx, ny, seed=seed, nsub=nsub, rtol=rtol,
                                                                   restart=restart)
    if log:
        log(f"waveguide network {w.nx}x{w.ny}: {time.perf_counter() - t0:.1f} s, n_eff {w.meta['neff']:.4f}")
    eps = torch.from_numpy(w.eps_node).to(dev)
    b = torch.from_numpy(w.b).to(dev)
    x = torch.empty_like(b)
    rows, fields = [], {}
    ref = None
    for prec in precisions:
        s = Solver(w.nx, w.ny, w.dx, w.dy, w.wavelength, eps, npml=w.npml, pml_order=w.pml_order,
                   pml_R=w.pml_R, nsub=w.nsub, overlap=w.overlap, interface_pml=w.interface_pml,
                   precision=PRECISIONS[prec], device=device)
        _b.stdd_set_option(s.ctx, _b.STDD_OPT_ORDER, ORDERS[order])
        sp = 0 if prec == "fp64" else static_pivot
        _b.stdd_set_option(s.ctx, _b.STDD_OPT_STATIC_PIVOT, sp)
        _b.stdd_set_option(s.ctx, _b.STDD_OPT_PIVOTING, pivoting)
        try:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize(dev)
            ev[0].record()
            s.factor()
            ev[1].record()
            s.set_sources(b)
            st = s.solve(x, restart=w.restart, rtol=rtol, maxit=maxit, allow_noconv=True)
            ev[2].record()
            torch.cuda.synchronize(dev)
            hist = s.history(0)
            stats = s.stats()
            # the first factorization of a context also tunes the substitution
            # launch shapes; a second one gives the steady-state time
            ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev2[0].record()
            s.factor()
            ev2[1].record()
            torch.cuda.synchronize(dev)
            row = dict(workload="waveguide-network", nx=w.nx, ny=w.ny, unknowns=w.n, nsub=w.nsub,
                       overlap=w.overlap, interface_pml=w.interface_pml, precision=prec, order=order,
                       restart=w.restart, static_pivot=sp, pivoting=pivoting,
                       raised_pivots=stats["raised_pivots"],
                       factor_s=ev[0].elapsed_time(ev[1]) / 1e3,
                       factor_again_s=ev2[0].elapsed_time(ev2[1]) / 1e3,
                       solve_s=ev[1].elapsed_time(ev[2]) / 1e3, iterations=len(hist) - 1,
                       converged=st == _b.STDD_OK, final_residual=float(hist[-1]),
                       device_gb=stats["device_bytes"] / 1e9, factor_entries=stats["factor_entries"],
                       factor_tflop=stats["factor_flops"] / 1e12)
            row["total_s"] = row["factor_s"] + row["solve_s"]
            row["mdofs"] = w.n / row["total_s"] / 1e6
            xf = x[0].clone()
            if prec == "fp64":
                ref = xf
            if ref is not None:
                row["diff_vs_fp64"] = float(torch.linalg.vector_norm(xf - ref) / torch.linalg.vector_norm(ref))
            if keep_fields:
                fields[prec] = xf.cpu().numpy()
        finally:
            s.close()
            torch.cuda.empty_cache()
        rows.append(row)
        print(json.dumps(row), file=out, flush=True)
    return (rows, fields, w) if keep_fields else rows


if __name__ == "__main__":
    import argparse
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="waveguide network, mixed precision against FP64")
    ap.add_argument("--nx", type=int, default=8192)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--nsub", type=int, default=32)
    ap.add_argument("--precisions", default="fp64,c64,fp16")
    ap.add_argument("--order", default="multiplicative", choices=sorted(ORDERS))
    ap.add_argument("--static-pivot", type=int, default=2)
    ap.add_argument("--pivoting", type=int, default=0, choices=[0, 1],
                    help="1: partial pivoting within each front's pivot rows")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--restart", type=int, default=50)
    ap.add_argument("--maxit", type=int, default=600)
    a = ap.parse_args()
    run(a.nx, a.ny, a.nsub, tuple(a.precisions.split(",")), a.order, a.rtol, a.restart, a.maxit,
        log=lambda m: print(m, file=sys.stderr, flush=True), static_pivot=a.static_pivot, pivoting=a.pivoting)
