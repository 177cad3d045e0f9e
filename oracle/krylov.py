"""Textbook restarted GMRES(m) and FGMRES(m), right preconditioning, complex128.

Oracle module (test infrastructure; see the package docstring).

The paper's own iteration is stationary (Algorithm 1).  The outer Krylov
solver accelerates it: with M^-1 the one-sweep source-transfer preconditioner,
right-preconditioned GMRES minimises ||b - A x|| over x0 + M^-1 K_j(A M^-1, r0),
a space that contains every Richardson / Algorithm-1 iterate.

Arnoldi uses modified Gram-Schmidt; the Hessenberg least-squares problem is
reduced by complex Givens rotations [c s; -conj(s) c] with real c.  The
relative residual is ||b - A x|| / ||b||; the true residual is recomputed at
every restart and at termination.  Flexible GMRES stores z_j = M^-1 v_j and
forms x = x0 + Z y, so the identity b - A x = V(beta e1 - H y) holds whatever
M^-1 does.
"""
from __future__ import annotations

import numpy as np


def _givens(a, b):
    """c (real), s (complex) with [c s; -conj(s) c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0
    if a == 0:
        return 0.0, complex(np.conj(b)) / abs(b)
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def gmres(matvec, precond, b, restart=30, rtol=1e-10, maxit=1000, x0=None, flexible=True, dot=None):
    """Restarted right-preconditioned (F)GMRES.

    Returns (x, history, iterations) with history the relative residual
    estimate after every inner step (history[0] = initial true residual).
    ``dot`` (default: np.vdot over the whole vector) is the inner product
    conj(a) . b; a vector split over processes passes one that sums the
    processes' partial products, and norms are then sqrt(dot(w, w))."""
    if dot is None:
        vdot, norm = np.vdot, np.linalg.norm
    else:
        vdot = dot

        def norm(w):
            return float(np.sqrt(max(dot(w, w).real, 0.0)))
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    bnorm = norm(b)
    if bnorm == 0:
        return np.zeros_like(b), [0.0], 0
    x = np.zeros(n, np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    history = []
    its = 0
    while True:
        r = b - matvec(x)
        beta = norm(r)
        if not history:
            history.append(beta / bnorm)
        if beta / bnorm <= rtol or its >= maxit:
            return x, history, its
        m = restart
        V = np.zeros((m + 1, n), np.complex128)
        Z = np.zeros((m, n), np.complex128) if flexible else None
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            z = precond(V[j])
            if flexible:
                Z[j] = z
            w = matvec(z)
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = norm(w)
            for i in range(j):                           # earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            hjj = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j, j] = hjj
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            breakdown = False
            if abs(hjj) == 0:
                breakdown = True
            else:
                nrm = norm(w)
                if nrm == 0:
                    breakdown = True
                else:
                    V[j + 1] = w / nrm
            if abs(g[j + 1]) / bnorm <= rtol or its >= maxit or breakdown:
                break
        k = j_done
        y = np.zeros(k, np.complex128)
        for i in range(k - 1, -1, -1):                   # back substitution
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        if flexible:
            x = x + y @ Z[:k]
        else:
            x = x + precond(y @ V[:k])
