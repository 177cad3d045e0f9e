"""GB300 (sm_103a) solver for 2-D TM FDFD by the PML-based overlapping
source-transfer domain decomposition of arXiv 2509.20801.

The compute path lives in libstdd.so (C ABI: include/stdd.h).  ``binding``
marshals arguments to it; ``Solver`` strings the calls together for one
problem.  Importing this package fails if libstdd.so has not been built.
"""
from __future__ import annotations

from . import binding as _b
from .binding import (STDD_PREC_C64, STDD_PREC_C64_BF16, STDD_PREC_C64_FP16, STDD_PREC_FP64, StddError, stdd_apply_operator,  # noqa: F401
                      stdd_apply_preconditioner, stdd_create, stdd_destroy, stdd_factor,
                      stdd_get_profile, stdd_get_stats, stdd_last_error, stdd_residual,
                      stdd_residual_noalloc,
                      stdd_set_profiling, stdd_set_option, STDD_OPT_GRAPHS, STDD_OPT_AUTOTUNE,
                      STDD_OPT_LEAF, STDD_OPT_ORDER, STDD_OPT_BAND, STDD_OPT_STATIC_PIVOT, STDD_OPT_PIVOTING, STDD_OPT_PERSISTENT, STDD_OPT_SWEEP_WAIT, STDD_OPT_UPDATE_TILE, STDD_OPT_SYMMETRIC, STDD_OPT_FP64_TC, STDD_OPT_SWEEP_SPLIT, stdd_local_solve, stdd_nd_analyze,
                      stdd_residual_history, stdd_set_decomposition, stdd_set_frequency,
                      stdd_set_grid, stdd_set_permittivity, stdd_set_pml, stdd_set_precision,
                      stdd_set_sources, stdd_solve, stdd_strip_info, stdd_tc_tile_product, stdd_tc_f64_tile_product, stdd_set_decomposition_2d, stdd_box_info)

LIB_PATH = _b.LIB_PATH


class Solver:
    """One FDFD problem on one GPU: configuration, factorization, solves.

    ``eps`` is a float64 (nx, ny) array or tensor; fields are complex128
    (nrhs, nx, ny) with node (i, j) at flat index i*ny + j."""

    def __init__(self, nx, ny, dx, dy, wavelength, eps, npml=(20, 20, 20, 20), pml_order=3,
                 pml_R=1e-8, nsub=2, overlap=8, interface_pml=20, precision=STDD_PREC_FP64,
                 device=0, stream=None, x_cuts=None):
        self.ctx = stdd_create(device, stream)
        self.nx, self.ny = int(nx), int(ny)
        stdd_set_grid(self.ctx, nx, ny, dx, dy)
        stdd_set_permittivity(self.ctx, eps)
        stdd_set_frequency(self.ctx, wavelength)
        stdd_set_pml(self.ctx, npml, pml_order, pml_R)
        stdd_set_decomposition(self.ctx, nsub, x_cuts, overlap, interface_pml)
        stdd_set_precision(self.ctx, precision)
        self.nsub = int(nsub)

    @classmethod
    def from_workload(cls, w, eps=None, **kw):
        return cls(w.nx, w.ny, w.dx, w.dy, w.wavelength, w.eps_node if eps is None else eps,
                   npml=w.npml, pml_order=w.pml_order, pml_R=w.pml_R, nsub=w.nsub,
                   overlap=w.overlap, interface_pml=w.interface_pml, **kw)

    def factor(self):
        stdd_factor(self.ctx)

    def set_sources(self, b):
        nrhs = 1 if b.ndim == 2 else b.shape[0]
        stdd_set_sources(self.ctx, nrhs, b)

    def solve(self, x_out, **kw):
        return stdd_solve(self.ctx, x_out, **kw)

    def history(self, rhs=0):
        return stdd_residual_history(self.ctx, rhs)

    def stats(self):
        return stdd_get_stats(self.ctx)

    def close(self):
        if self.ctx is not None:
            stdd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
