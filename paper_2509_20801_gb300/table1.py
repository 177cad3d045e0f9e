"""The paper's first example at full size on one GPU: plane-wave scattering by
a dielectric cylinder (r = 9 wavelengths, eps 4, 40 points per wavelength,
6000 x 6000 nodes, about 36 million unknowns; Sec. 3.1, Table 1), solved for
the scattered field (Eq. 7) with a growing number of strips.

For each strip count: factorization and solve times (CUDA events around the
library calls), inner iterations of FGMRES to the tolerance, optionally the
iterations of the paper's own stationary iteration (Algorithm 1), the device
memory the context holds, and the relative L2 error of the field against the
Mie series on seeded sample nodes in the ring a + lambda/4 <= r <= a + 2 lambda
clear of the PML (the series is evaluated here, outside the library).  One JSON line per strip
count on stdout.

    python -m paper_2509_20801_gb300.table1 [--n 6000] [--nsub 2,4,8,16,32,64]
        [--precision fp64|c64] [--order additive|multiplicative|red-black] [--restart m]
        [--richardson]
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import binding as _b

PRECISIONS = {"fp64": _b.STDD_PREC_FP64, "c64": _b.STDD_PREC_C64, "fp16": _b.STDD_PREC_C64_FP16}
ORDERS = {"additive": 0, "multiplicative": 1, "red-black": 2}


def mie_scattered(x, y, cx, cy, a, eps1, k0):
    """Scattered field of exp(i k0 x) on a dielectric cylinder (TM): the
    separation-of-variables series with exp(i k0 x) = exp(i k0 cx) sum_n i^n
    J_n(k0 r) e^{i n phi} and continuity of E and dE/dr at r = a."""
    import scipy.special as ss
    m = math.sqrt(eps1)
    r = np.hypot(x - cx, y - cy)
    ph = np.arctan2(y - cy, x - cx)
    x0, x1 = k0 * a, m * k0 * a
    u = np.zeros(np.shape(r), complex)
    for n in range(-(int(x1) + 20), int(x1) + 21):
        bn = (m * ss.jvp(n, x1) * ss.jv(n, x0) - ss.jv(n, x1) * ss.jvp(n, x0)) / (
            ss.jv(n, x1) * ss.h1vp(n, x0) - m * ss.jvp(n, x1) * ss.hankel1(n, x0))
        u += (1j ** n) * bn * ss.hankel1(n, k0 * r) * np.exp(1j * n * ph)
    return u * np.exp(1j * k0 * cx)


def sample_ring(w, count, seed=0):
    """Seeded node indices (i, j) with a + lambda/4 <= r <= a + 2 lambda,
    kept a quarter wavelength clear of the PML."""
    rng = np.random.default_rng(seed)
    cx, cy = w.meta["center"]
    a = w.meta["radius"]
    r_hi = min(a + 2.0 * w.wavelength, cx - w.npml[0] * w.dx - 0.25 * w.wavelength)
    if r_hi <= a + 0.25 * w.wavelength:
        raise ValueError("no room between the cylinder and the PML")
    r = rng.uniform(a + 0.25 * w.wavelength, r_hi, count)
    t = rng.uniform(0, 2 * math.pi, count)
    i = np.clip(np.rint((cx + r * np.cos(t)) / w.dx).astype(int), 0, w.nx - 1)
    j = np.clip(np.rint((cy + r * np.sin(t)) / w.dy).astype(int), 0, w.ny - 1)
    return i, j


def run(n=6000, ppw=40, radius=9.0, nsubs=(2, 4, 8, 16, 32, 64), precision="fp64", rtol=1e-8, restart=30,
        maxit=1000, richardson=False, samples=4000, device=0, out=sys.stdout, log=None, order="additive"):
    import torch
    import workloads as W
    from . import Solver
    dev = torch.device("cuda", device)
    t0 = time.perf_counter()
    w = W.cylinder_scattering(n=n, ppw=ppw, radius=radius, nsub=nsubs[0], rtol=rtol, restart=restart)
    if log:
        log(f"geometry {n}x{n}: {time.perf_counter() - t0:.1f} s")
    si, sj = sample_ring(w, samples)
    cx, cy = w.meta["center"]
    mie = mie_scattered(si * w.dx, sj * w.dy, cx, cy, w.meta["radius"], w.meta["eps_cyl"], 2 * math.pi / w.wavelength)
    eps = torch.from_numpy(w.eps_node).to(dev)
    b = torch.from_numpy(w.b).to(dev)
    x = torch.empty_like(b)
    rows = []
    for ns in nsubs:
        s = Solver(w.nx, w.ny, w.dx, w.dy, w.wavelength, eps, npml=w.npml, pml_order=w.pml_order,
                   pml_R=w.pml_R, nsub=ns, overlap=w.overlap, interface_pml=w.interface_pml,
                   precision=PRECISIONS[precision], device=device)
        _b.stdd_set_option(s.ctx, _b.STDD_OPT_ORDER, ORDERS[order])
        try:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize(dev)
            ev[0].record()
            s.factor()
            ev[1].record()
            s.set_sources(b)
            st = s.solve(x, restart=restart, rtol=rtol, maxit=maxit, allow_noconv=True)
            ev[2].record()
            torch.cuda.synchronize(dev)
            hist = s.history(0)
            stats = s.stats()
            got = x[0].cpu().numpy()[si, sj]
            row = dict(nsub=ns, unknowns=w.n, unknowns_per_strip=w.n // ns, precision=precision, order=order,
                       restart=restart,
                       factor_s=ev[0].elapsed_time(ev[1]) / 1e3, solve_s=ev[1].elapsed_time(ev[2]) / 1e3,
                       iterations=len(hist) - 1, converged=st == _b.STDD_OK, final_residual=float(hist[-1]),
                       device_gb=stats["device_bytes"] / 1e9, factor_entries=stats["factor_entries"],
                       factor_tflop=stats["factor_flops"] / 1e12,
                       mie_error=float(np.linalg.norm(got - mie) / np.linalg.norm(mie)))
            row["total_s"] = row["factor_s"] + row["solve_s"]
            if richardson:
                ev[0].record()
                st = s.solve(x, rtol=rtol, maxit=maxit, paper_richardson=True, allow_noconv=True)
                ev[1].record()
                torch.cuda.synchronize(dev)
                h = s.history(0)
                row.update(richardson_sweeps=len(h) - 1, richardson_s=ev[0].elapsed_time(ev[1]) / 1e3,
                           richardson_converged=st == _b.STDD_OK)
        finally:
            s.close()
            torch.cuda.empty_cache()
        rows.append(row)
        print(json.dumps(row), file=out, flush=True)
    return rows


if __name__ == "__main__":
    import argparse
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="Table 1 of the paper on one GPU")
    ap.add_argument("--n", type=int, default=6000)
    ap.add_argument("--ppw", type=int, default=40)
    ap.add_argument("--radius", type=float, default=9.0)
    ap.add_argument("--nsub", default="2,4,8,16,32,64")
    ap.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--richardson", action="store_true")
    ap.add_argument("--order", default="additive", choices=sorted(ORDERS))
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--maxit", type=int, default=1000)
    a = ap.parse_args()
    run(a.n, a.ppw, a.radius, tuple(int(v) for v in a.nsub.split(",")), a.precision, a.rtol, a.restart,
        a.maxit, a.richardson, order=a.order, log=lambda m: print(m, file=sys.stderr, flush=True))
