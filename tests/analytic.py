"""Closed-form fields used to pin the oracle (independent of its code).

* ``discrete_line_source_1d``: the exact solution of the infinite 1-D
  three-point recurrence (u_{j+1} - 2 u_j + u_{j-1})/h^2 + k^2 u_j = -delta_{j,js}/h,
  derived by substitution: u_j = (i h / (2 sin t)) e^{i t |j - js|},
  cos t = 1 - k^2 h^2 / 2 (outgoing for e^{-i w t}).
* ``hankel_green``: the 2-D free-space Green's function (i/4) H0^(1)(k r),
  solution of (lap + k^2) G = -delta.
* ``mie_point_source``: total field of a unit line source outside a
  dielectric cylinder (TM, mu = 1) by separation of variables (Kong, 1986):
  incident coefficients d_n = (i/4) H_n(k0 r_s) e^{-i n phi_s}, scattered
  a_n = d_n [k1 J_n'(k1 a) J_n(k0 a) - k0 J_n(k1 a) J_n'(k0 a)]
          / [k0 J_n(k1 a) H_n'(k0 a) - k1 J_n'(k1 a) H_n(k0 a)],
  from continuity of u and du/dr at r = a.
* ``mie_plane_wave``: scattered field of the plane wave exp(i k0 x) on the
  same cylinder: exp(i k0 x) = exp(i k0 cx) sum_n i^n J_n(k0 r) e^{i n phi}
  (Jacobi-Anger about the centre), scattered coefficients exp(i k0 cx) i^n b_n
  b_n = [m J_n'(m k0 a) J_n(k0 a) - J_n(m k0 a) J_n'(k0 a)]
        / [J_n(m k0 a) H_n'(k0 a) - m J_n'(m k0 a) H_n(k0 a)],  m = sqrt(eps1).
"""
import math

import numpy as np
import scipy.special as ss


def discrete_line_source_1d(n, h, k, js):
    t = math.acos(1.0 - (k * h) ** 2 / 2.0)
    j = np.arange(n)
    return 1j * h / (2.0 * math.sin(t)) * np.exp(1j * t * np.abs(j - js))


def hankel_green(k, r):
    return 0.25j * ss.hankel1(0, k * r)


def mie_point_source(x, y, cx, cy, a, eps1, xs, ys, k0):
    k1 = k0 * math.sqrt(eps1)
    rs = math.hypot(xs - cx, ys - cy)
    phs = math.atan2(ys - cy, xs - cx)
    r = np.hypot(x - cx, y - cy)
    ph = np.arctan2(y - cy, x - cx)
    nmax = int(k1 * a) + 20
    u = hankel_green(k0, np.hypot(x - xs, y - ys))
    for n in range(-nmax, nmax + 1):
        dn = 0.25j * ss.hankel1(n, k0 * rs) * np.exp(-1j * n * phs)
        j0, j0p = ss.jv(n, k0 * a), ss.jvp(n, k0 * a)
        j1, j1p = ss.jv(n, k1 * a), ss.jvp(n, k1 * a)
        h0, h0p = ss.hankel1(n, k0 * a), ss.h1vp(n, k0 * a)
        an = dn * (k1 * j1p * j0 - k0 * j1 * j0p) / (k0 * j1 * h0p - k1 * j1p * h0)
        u = u + an * ss.hankel1(n, k0 * r) * np.exp(1j * n * ph)
    return u


def mie_plane_wave(x, y, cx, cy, a, eps1, k0):
    m = math.sqrt(eps1)
    r = np.hypot(x - cx, y - cy)
    ph = np.arctan2(y - cy, x - cx)
    x0, x1 = k0 * a, m * k0 * a
    nmax = int(x1) + 20
    u = np.zeros(np.shape(r), complex)
    for n in range(-nmax, nmax + 1):
        bn = (m * ss.jvp(n, x1) * ss.jv(n, x0) - ss.jv(n, x1) * ss.jvp(n, x0)) / (
            ss.jv(n, x1) * ss.h1vp(n, x0) - m * ss.jvp(n, x1) * ss.hankel1(n, x0))
        u = u + (1j ** n) * bn * ss.hankel1(n, k0 * r) * np.exp(1j * n * ph)
    return u * np.exp(1j * k0 * cx)
