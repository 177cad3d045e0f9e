"""Thin Python binding of the C ABI in include/stdd.h (ctypes).

Argument marshalling only: every function has the name of the C entry point
it wraps, takes numpy arrays or torch tensors (complex128 for fields,
float64 for permittivity) and passes their pointers with ``is_device`` set
from the tensor's device.  All computation happens in libstdd.so; if the
library is missing this module raises on import.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstdd.so")

STDD_OK, STDD_EINVAL, STDD_ESTATE, STDD_ENOMEM, STDD_ECUDA = 0, 1, 2, 3, 4
STDD_EPIVOT, STDD_EBREAKDOWN, STDD_ENOCONV, STDD_ETIMEOUT = 5, 6, 7, 8
STDD_PREC_FP64, STDD_PREC_C64, STDD_PREC_C64_BF16, STDD_PREC_C64_FP16 = 0, 1, 2, 3
STDD_X0_ZERO, STDD_X0_USER, STDD_X0_LEARNED = 0, 1, 2
STDD_NN_FP32, STDD_NN_BF16, STDD_NN_TC = 0, 1, 2
STATUS_NAMES = {0: "STDD_OK", 1: "STDD_EINVAL", 2: "STDD_ESTATE", 3: "STDD_ENOMEM", 4: "STDD_ECUDA",
                5: "STDD_EPIVOT", 6: "STDD_EBREAKDOWN", 7: "STDD_ENOCONV", 8: "STDD_ETIMEOUT"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libstdd.so is not built ({LIB_PATH}); run __graft_entry__.build()")

lib = ctypes.CDLL(LIB_PATH)

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
P = ctypes.POINTER


class stdd_solve_opts(ctypes.Structure):
    _fields_ = [("restart", c_int), ("maxit", c_int), ("rtol", c_double), ("x0_mode", c_int),
                ("x0", c_void_p), ("x0_is_device", c_int), ("paper_richardson", c_int)]


class stdd_stats(ctypes.Structure):
    _fields_ = [("nfronts", ctypes.c_longlong), ("depth", c_int), ("max_pivots", c_int),
                ("max_border", c_int), ("factor_entries", ctypes.c_longlong),
                ("factor_flops", c_double), ("solve_flops", c_double),
                ("local_dofs", ctypes.c_longlong), ("device_bytes", ctypes.c_longlong),
                ("iterations", c_int), ("final_residual", c_double), ("min_pivot", c_double),
                ("reorth_passes", c_int), ("raised_pivots", ctypes.c_longlong),
                ("factor_flops_lu", c_double)]


class stdd_profile(ctypes.Structure):
    _fields_ = [("factor_ms", c_double), ("minv_ms", c_double), ("minv_calls", c_int),
                ("matvec_ms", c_double), ("matvec_calls", c_int), ("ortho_ms", c_double),
                ("ortho_calls", c_int), ("solve_ms", c_double), ("launches", ctypes.c_longlong),
                ("small_ms", c_double), ("small_flops", c_double), ("small_calls", c_int),
                ("update_ms", c_double), ("update_flops", c_double), ("update_calls", c_int),
                ("up_ms", c_double), ("up_bytes", c_double), ("up_calls", c_int),
                ("down_ms", c_double), ("down_bytes", c_double), ("down_calls", c_int),
                ("small_flops_executed", c_double), ("update_flops_executed", c_double),
                ("sweep_ms", c_double), ("sweep_bytes", c_double), ("sweep_calls", c_int)]


_SIGS = {
    "stdd_create": (c_int, [P(c_void_p), c_int, c_void_p]),
    "stdd_destroy": (None, [c_void_p]),
    "stdd_set_grid": (c_int, [c_void_p, c_int, c_int, c_double, c_double]),
    "stdd_set_permittivity": (c_int, [c_void_p, c_void_p, c_int]),
    "stdd_set_frequency": (c_int, [c_void_p, c_double]),
    "stdd_set_pml": (c_int, [c_void_p, P(c_int), c_int, c_double]),
    "stdd_set_decomposition": (c_int, [c_void_p, c_int, P(c_int), c_int, c_int]),
    "stdd_set_precision": (c_int, [c_void_p, c_int]),
    "stdd_set_sources": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "stdd_factor": (c_int, [c_void_p]),
    "stdd_solve": (c_int, [c_void_p, P(stdd_solve_opts), c_void_p, c_int]),
    "stdd_residual_history": (c_int, [c_void_p, c_int, P(c_double), c_int, P(c_int)]),
    "stdd_last_error": (ctypes.c_char_p, [c_void_p]),
    "stdd_apply_operator": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "stdd_apply_preconditioner": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "stdd_local_solve": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int]),
    "stdd_strip_info": (c_int, [c_void_p, c_int, P(c_int), P(c_int), P(c_int), P(c_int)]),
    "stdd_set_decomposition_2d": (c_int, [c_void_p, c_int, P(c_int), c_int, P(c_int), c_int, c_int]),
    "stdd_box_info": (c_int, [c_void_p, c_int, P(c_int)]),
    "stdd_get_stats": (c_int, [c_void_p, P(stdd_stats)]),
    "stdd_residual": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, P(c_double), c_int]),
    "stdd_residual_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, P(c_double)]),
    "stdd_set_profiling": (c_int, [c_void_p, c_int]),
    "stdd_set_option": (c_int, [c_void_p, c_int, c_int]),
    "stdd_get_profile": (c_int, [c_void_p, P(stdd_profile), c_int]),
    "stdd_tc_tile_product": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "stdd_tc_f64_tile_product": (c_int, [c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "stdd_nd_analyze": (c_int, [c_int, c_int, c_int, P(c_int), P(ctypes.c_longlong), c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p]),
    "stdd_nn_create": (c_int, [P(c_void_p), c_int, c_void_p, c_int, c_int, c_int, c_int, ctypes.c_ulonglong]),
    "stdd_nn_destroy": (None, [c_void_p]),
    "stdd_nn_num_params": (ctypes.c_longlong, [c_void_p]),
    "stdd_nn_get_params": (c_int, [c_void_p, c_void_p]),
    "stdd_nn_set_params": (c_int, [c_void_p, c_void_p]),
    "stdd_nn_forward": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "stdd_nn_gradient": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, P(ctypes.c_float), c_void_p]),
    "stdd_nn_train_step": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, ctypes.c_float,
                                   P(ctypes.c_float)]),
    "stdd_nn_make_images": (c_int, [c_void_p, c_int, c_int, c_double, c_void_p, c_void_p, c_void_p, c_int, c_int,
                                    c_void_p, c_void_p]),
    "stdd_nn_last_error": (ctypes.c_char_p, [c_void_p]),
    "stdd_set_learned_guess": (c_int, [c_void_p, c_void_p]),
    "stdd_learned_guess_info": (c_int, [c_void_p, c_int, P(c_double), P(c_double), P(c_int)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class StddError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported buffer type {type(a)}")


def _check(ctx, st, allow=()):
    if st != STDD_OK and st not in allow:
        msg = lib.stdd_last_error(ctx)
        raise StddError(st, msg.decode() if msg else "")
    return st


def stdd_create(device=0, stream=None):
    ctx = c_void_p()
    st = lib.stdd_create(ctypes.byref(ctx), int(device), c_void_p(stream) if stream else None)
    if st != STDD_OK:
        raise StddError(st, "stdd_create failed")
    return ctx


def stdd_destroy(ctx):
    lib.stdd_destroy(ctx)


def stdd_set_grid(ctx, nx, ny, dx, dy):
    return _check(ctx, lib.stdd_set_grid(ctx, int(nx), int(ny), float(dx), float(dy)))


def stdd_set_permittivity(ctx, eps):
    p, dev = _ptr(eps)
    return _check(ctx, lib.stdd_set_permittivity(ctx, c_void_p(p), dev))


def stdd_set_frequency(ctx, wavelength):
    return _check(ctx, lib.stdd_set_frequency(ctx, float(wavelength)))


def stdd_set_pml(ctx, npml, order_m, R0):
    arr = (c_int * 4)(*[int(v) for v in npml])
    return _check(ctx, lib.stdd_set_pml(ctx, arr, int(order_m), float(R0)))


def stdd_set_decomposition(ctx, nsub, x_cuts, overlap, interface_pml):
    cuts = None if x_cuts is None else (c_int * (nsub + 1))(*[int(v) for v in x_cuts])
    return _check(ctx, lib.stdd_set_decomposition(ctx, int(nsub), cuts, int(overlap), int(interface_pml)))


def stdd_set_precision(ctx, mode):
    return _check(ctx, lib.stdd_set_precision(ctx, int(mode)))


def stdd_set_sources(ctx, nrhs, b):
    p, dev = _ptr(b)
    return _check(ctx, lib.stdd_set_sources(ctx, int(nrhs), c_void_p(p), dev))


def stdd_factor(ctx):
    return _check(ctx, lib.stdd_factor(ctx))


def stdd_solve(ctx, x_out, restart=30, maxit=1000, rtol=1e-10, x0=None, paper_richardson=False,
               allow_noconv=False):
    o = stdd_solve_opts()
    o.restart, o.maxit, o.rtol = int(restart), int(maxit), float(rtol)
    o.paper_richardson = 1 if paper_richardson else 0
    if x0 is None:
        o.x0_mode, o.x0, o.x0_is_device = STDD_X0_ZERO, None, 0
    elif isinstance(x0, str):
        if x0 != "learned":
            raise ValueError("x0 must be None, 'learned' or a field array")
        o.x0_mode, o.x0, o.x0_is_device = STDD_X0_LEARNED, None, 0
    else:
        p, dev = _ptr(x0)
        o.x0_mode, o.x0, o.x0_is_device = STDD_X0_USER, p, dev
    p, dev = _ptr(x_out)
    allow = (STDD_ENOCONV,) if allow_noconv else ()
    return _check(ctx, lib.stdd_solve(ctx, ctypes.byref(o), c_void_p(p), dev), allow)


def stdd_residual_history(ctx, rhs=0):
    n = c_int(0)
    _check(ctx, lib.stdd_residual_history(ctx, int(rhs), None, 0, ctypes.byref(n)))
    out = (c_double * max(1, n.value))()
    _check(ctx, lib.stdd_residual_history(ctx, int(rhs), out, n.value, ctypes.byref(n)))
    return np.array(out[:n.value])


def stdd_last_error(ctx):
    m = lib.stdd_last_error(ctx)
    return m.decode() if m else ""


def stdd_apply_operator(ctx, x, y):
    px, dx_ = _ptr(x)
    py, dy_ = _ptr(y)
    if dx_ != dy_:
        raise ValueError("x and y must live on the same side")
    return _check(ctx, lib.stdd_apply_operator(ctx, c_void_p(px), c_void_p(py), dx_))


def stdd_apply_preconditioner(ctx, v, z):
    pv, dv = _ptr(v)
    pz, dz = _ptr(z)
    if dv != dz:
        raise ValueError("v and z must live on the same side")
    return _check(ctx, lib.stdd_apply_preconditioner(ctx, c_void_p(pv), c_void_p(pz), dv))


def stdd_local_solve(ctx, strip, t, z):
    pt, dt = _ptr(t)
    pz, dz = _ptr(z)
    if dt != dz:
        raise ValueError("t and z must live on the same side")
    return _check(ctx, lib.stdd_local_solve(ctx, int(strip), c_void_p(pt), c_void_p(pz), dt))


def stdd_strip_info(ctx, strip):
    v = [c_int() for _ in range(4)]
    _check(ctx, lib.stdd_strip_info(ctx, int(strip), *[ctypes.byref(x) for x in v]))
    c0, c1, x0, x1 = (x.value for x in v)
    return dict(c0=c0, c1=c1, x0=x0, x1=x1)


def stdd_set_decomposition_2d(ctx, px, py, overlap, interface_pml, x_cuts=None, y_cuts=None):
    """px x py boxes (checkerboard); cuts as lists of px+1 / py+1 ints or None."""
    xa = (c_int * (px + 1))(*[int(v) for v in x_cuts]) if x_cuts is not None else None
    ya = (c_int * (py + 1))(*[int(v) for v in y_cuts]) if y_cuts is not None else None
    return _check(ctx, lib.stdd_set_decomposition_2d(ctx, int(px), xa, int(py), ya, int(overlap),
                                                     int(interface_pml)))


def stdd_box_info(ctx, box):
    v = (c_int * 8)()
    _check(ctx, lib.stdd_box_info(ctx, int(box), v))
    return dict(zip(("c0", "c1", "r0", "r1", "x0", "x1", "y0", "y1"), list(v)))


def stdd_get_stats(ctx):
    s = stdd_stats()
    _check(ctx, lib.stdd_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in stdd_stats._fields_}


def stdd_residual(ctx, x, b, r):
    """r = b - A x; returns ||r|| / ||b||."""
    px, dx_ = _ptr(x)
    pb, db = _ptr(b)
    pr, dr = _ptr(r)
    if not dx_ == db == dr:
        raise ValueError("x, b and r must live on the same side")
    rel = c_double(0.0)
    _check(ctx, lib.stdd_residual(ctx, c_void_p(px), c_void_p(pb), c_void_p(pr), ctypes.byref(rel), dx_))
    return rel.value


def stdd_residual_noalloc(ctx, x, b, r):
    """r = b - A x into the caller's device buffers with no device allocation
    (fixed in-library scratch); returns ||r|| / ||b||.  All three must be
    CUDA tensors."""
    px, dx_ = _ptr(x)
    pb, db = _ptr(b)
    pr, dr = _ptr(r)
    if not (dx_ == db == dr == 1):
        raise ValueError("x, b and r must be device buffers")
    rel = c_double(0.0)
    _check(ctx, lib.stdd_residual_noalloc(ctx, c_void_p(px), c_void_p(pb), c_void_p(pr), ctypes.byref(rel)))
    return rel.value


STDD_OPT_GRAPHS, STDD_OPT_AUTOTUNE, STDD_OPT_LEAF, STDD_OPT_ORDER, STDD_OPT_BAND = 1, 2, 3, 4, 5
STDD_OPT_STATIC_PIVOT = 6
STDD_OPT_PIVOTING = 7
STDD_OPT_PERSISTENT = 8
STDD_OPT_SWEEP_WAIT = 9
STDD_OPT_UPDATE_TILE = 10
STDD_OPT_SYMMETRIC = 11
STDD_OPT_FP64_TC = 12
STDD_OPT_SWEEP_SPLIT = 13


def stdd_set_profiling(ctx, level=1):
    """0 off, 1 phase spans, 2 phase + per-launch kernel spans (graphs off)."""
    return _check(ctx, lib.stdd_set_profiling(ctx, int(level)))


def stdd_set_option(ctx, option, value):
    return _check(ctx, lib.stdd_set_option(ctx, int(option), int(value)))


def stdd_get_profile(ctx, reset=True):
    s = stdd_profile()
    _check(ctx, lib.stdd_get_profile(ctx, ctypes.byref(s), 1 if reset else 0))
    return {k: getattr(s, k) for k, _ in stdd_profile._fields_}


def stdd_tc_tile_product(C, R, fmt=1, device=0):
    """D = C R on the tensor cores (one tile of the mixed-precision front
    update): C complex (64, kc), R complex (kc, 128), 1 <= kc <= 32; returns D
    complex (64, 128)."""
    C = np.asarray(C, np.complex128)
    R = np.asarray(R, np.complex128)
    kc = C.shape[1]
    if C.shape != (64, kc) or R.shape != (kc, 128):
        raise ValueError("C must be 64 x kc and R kc x 128")
    Cf = np.ascontiguousarray(C.T)          # column-major: column j contiguous
    Rf = np.ascontiguousarray(R.T)
    D = np.empty((128, 64), np.complex128)  # column-major D
    st = lib.stdd_tc_tile_product(int(device), int(fmt), int(kc), c_void_p(Cf.ctypes.data),
                                  c_void_p(Rf.ctypes.data), c_void_p(D.ctypes.data))
    if st != STDD_OK:
        raise StddError(st, "stdd_tc_tile_product failed")
    return D.T.copy()


def stdd_tc_f64_tile_product(C, R, device=0):
    """D = C R in complex128 through the exact-splitting tensor-core path of
    the complex128 front update: C complex (64, kc), R complex (kc, 64),
    1 <= kc <= 32; returns D complex (64, 64)."""
    C = np.asarray(C, np.complex128)
    R = np.asarray(R, np.complex128)
    kc = C.shape[1]
    if C.shape != (64, kc) or R.shape != (kc, 64):
        raise ValueError("C must be 64 x kc and R kc x 64")
    Cf = np.ascontiguousarray(C.T)
    Rf = np.ascontiguousarray(R.T)
    D = np.empty((64, 64), np.complex128)   # column-major D (rows of this array are D's columns)
    st = lib.stdd_tc_f64_tile_product(int(device), int(kc), c_void_p(Cf.ctypes.data), c_void_p(Rf.ctypes.data),
                                      c_void_p(D.ctypes.data))
    if st != STDD_OK:
        raise StddError(st, "stdd_tc_f64_tile_product failed")
    return D.T.copy()


def stdd_nd_analyze(W, H, leaf_max=64):
    """Host-only nested-dissection analysis; returns dict of numpy arrays."""
    nf = c_int(0)
    nn = ctypes.c_longlong(0)
    st = lib.stdd_nd_analyze(int(W), int(H), int(leaf_max), ctypes.byref(nf), ctypes.byref(nn),
                             None, None, None, None, None)
    if st != STDD_OK:
        raise StddError(st, "stdd_nd_analyze failed")
    p = np.zeros(nf.value, np.int32)
    b = np.zeros(nf.value, np.int32)
    parent = np.zeros(nf.value, np.int32)
    level = np.zeros(nf.value, np.int32)
    nodes = np.zeros(max(1, nn.value), np.int32)
    st = lib.stdd_nd_analyze(int(W), int(H), int(leaf_max), ctypes.byref(nf), ctypes.byref(nn),
                             p.ctypes.data, b.ctypes.data, parent.ctypes.data, level.ctypes.data,
                             nodes.ctypes.data)
    if st != STDD_OK:
        raise StddError(st, "stdd_nd_analyze failed")
    return dict(p=p, b=b, parent=parent, level=level, nodes=nodes[:nn.value])


# ---- learned initial guess ------------------------------------------------

def _check_nn(nn, st):
    if st != STDD_OK:
        msg = lib.stdd_nn_last_error(nn) if nn else b"network not created"
        raise StddError(st, msg.decode() if msg else "")
    return st


def stdd_nn_create(device=0, stream=None, levels=6, base_channels=32, max_channels=256, mode=STDD_NN_TC, seed=0):
    h = c_void_p()
    st = lib.stdd_nn_create(ctypes.byref(h), int(device), stream, int(levels), int(base_channels),
                            int(max_channels), int(mode), int(seed))
    if st != STDD_OK:
        raise StddError(st, "stdd_nn_create failed")
    return h


def stdd_nn_destroy(nn):
    lib.stdd_nn_destroy(nn)


def stdd_nn_num_params(nn):
    return int(lib.stdd_nn_num_params(nn))


def stdd_nn_get_params(nn):
    out = np.empty(stdd_nn_num_params(nn), np.float32)
    _check_nn(nn, lib.stdd_nn_get_params(nn, out.ctypes.data))
    return out


def stdd_nn_set_params(nn, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != stdd_nn_num_params(nn):
        raise ValueError("parameter array has the wrong size")
    return _check_nn(nn, lib.stdd_nn_set_params(nn, a.ctypes.data))


def _dev_f32(t, name):
    p, dev = _ptr(t)
    if not dev:
        raise ValueError(f"{name} must be a device tensor")
    if getattr(t, "dtype", None) is not None and str(t.dtype) != "torch.float32":
        raise TypeError(f"{name} must be float32")
    return p


def stdd_nn_forward(nn, inp, out):
    """out[N, 2, H, W] = network(inp[N, 3, H, W]) (device float32 tensors)."""
    N, C, H, W = inp.shape
    if C != 3 or tuple(out.shape) != (N, 2, H, W):
        raise ValueError("input must be [N, 3, H, W] and output [N, 2, H, W]")
    return _check_nn(nn, lib.stdd_nn_forward(nn, N, H, W, _dev_f32(inp, "input"), _dev_f32(out, "output")))


def stdd_nn_gradient(nn, inp, target):
    """(loss, gradient array) of the mean squared error for one batch."""
    N, C, H, W = inp.shape
    if C != 3 or tuple(target.shape) != (N, 2, H, W):
        raise ValueError("input must be [N, 3, H, W] and target [N, 2, H, W]")
    loss = ctypes.c_float(0)
    g = np.empty(stdd_nn_num_params(nn), np.float32)
    _check_nn(nn, lib.stdd_nn_gradient(nn, N, H, W, _dev_f32(inp, "input"), _dev_f32(target, "target"),
                                       ctypes.byref(loss), g.ctypes.data))
    return float(loss.value), g


def stdd_nn_train_step(nn, inp, target, lr):
    N, C, H, W = inp.shape
    if C != 3 or tuple(target.shape) != (N, 2, H, W):
        raise ValueError("input must be [N, 3, H, W] and target [N, 2, H, W]")
    loss = ctypes.c_float(0)
    _check_nn(nn, lib.stdd_nn_train_step(nn, N, H, W, _dev_f32(inp, "input"), _dev_f32(target, "target"),
                                         float(lr), ctypes.byref(loss)))
    return float(loss.value)


def stdd_nn_make_images(nn, unit, eps, b, x, inp, target=None):
    """Fill inp[3, H, W] (and target[2, H, W] if x is given) from the device
    fields eps (nx, ny) float64, b and x (nx, ny) complex128."""
    nx, ny = eps.shape
    _, H, W = inp.shape
    pe, de = _ptr(eps)
    pb, db = _ptr(b)
    px, dxx = _ptr(x) if x is not None else (None, 1)
    if not (de and db and dxx):
        raise ValueError("fields must be device tensors")
    pt = _dev_f32(target, "target") if x is not None else None
    return _check_nn(nn, lib.stdd_nn_make_images(nn, nx, ny, float(unit), pe, pb, px, H, W,
                                                 _dev_f32(inp, "input"), pt))


def stdd_nn_last_error(nn):
    m = lib.stdd_nn_last_error(nn)
    return m.decode() if m else ""


def stdd_set_learned_guess(ctx, nn):
    return _check(ctx, lib.stdd_set_learned_guess(ctx, nn))


def stdd_learned_guess_info(ctx, rhs=0):
    """(raw relative residual, scaled relative residual, used) of the last
    learned guess for right-hand side rhs."""
    a, b, u = c_double(0), c_double(0), c_int(0)
    _check(ctx, lib.stdd_learned_guess_info(ctx, int(rhs), ctypes.byref(a), ctypes.byref(b), ctypes.byref(u)))
    return a.value, b.value, bool(u.value)
