"""Closed-form rays used to pin the oracle (pure numpy, independent of oracle.c).

Each function solves the ray equations exactly for a special medium, with the
parameter tau of the Hamiltonian flow dx/dtau = dD/dk = 2k,
dk/dtau = -dD/dx = w^2 grad n^2, and physical time dt/dtau = -dD/dw = 2 w n^2.
"""
from __future__ import annotations

import math

import numpy as np


def _invert_monotone(t_of, dt_dtau, T):
    """tau with t_of(tau) = T for increasing t_of: Newton steps kept inside a
    bisection bracket (plain Newton can jump branches where dt/dtau is small)."""
    lo, hi = 0.0, max(T, 1e-3)
    while t_of(hi) < T:
        hi *= 2.0
    tau = 0.5 * (lo + hi)
    for _ in range(200):
        f = t_of(tau) - T
        if f > 0:
            hi = tau
        else:
            lo = tau
        d = dt_dtau(tau)
        nt = tau - f / d if d > 0 else 0.5 * (lo + hi)
        if not (lo < nt < hi):
            nt = 0.5 * (lo + hi)
        if abs(nt - tau) <= 1e-17 * max(1.0, tau) or hi - lo < 1e-16:
            tau = nt
            break
        tau = nt
    return tau


def straight(x0, k0, n_h, t, omega=1.0):
    """Homogeneous medium: x = x0 + k0 t / (w n^2), k constant."""
    x0 = np.asarray(x0, float)
    k0 = np.asarray(k0, float)
    return x0 + k0 * (t / (omega * n_h * n_h)), k0.copy()


def grin(x0, k0, n0, a, T, omega=1.0):
    """Parabolic fibre n^2 = n0^2 (1 - a^2 (y^2 + z^2)) without blobs.

    y(tau) = y0 cos(W tau) + (2 ky0 / W) sin(W tau), W = 2 w n0 a (same for z);
    x(tau) = x0 + 2 kx tau;  t(tau) = 2 w n0^2 tau - 2 w n0^2 a^2 int_0^tau (y^2 + z^2).
    T -> tau by Newton (dt/dtau = 2 w n^2 > 0).  Returns (x, k) at physical time T.
    """
    x0 = np.asarray(x0, float)
    k0 = np.asarray(k0, float)
    W = 2.0 * omega * n0 * a

    def quad_int(A, B, tau):
        s2 = math.sin(2 * W * tau)
        c2 = math.cos(2 * W * tau)
        return (A * A * (tau / 2 + s2 / (4 * W)) + B * B * (tau / 2 - s2 / (4 * W))
                + A * B * (1 - c2) / (2 * W))

    Ay, By = x0[1], 2 * k0[1] / W
    Az, Bz = x0[2], 2 * k0[2] / W

    def t_of(tau):
        return 2 * omega * n0 ** 2 * tau - 2 * omega * n0 ** 2 * a ** 2 * (
            quad_int(Ay, By, tau) + quad_int(Az, Bz, tau))

    def pos(tau):
        y = Ay * math.cos(W * tau) + By * math.sin(W * tau)
        z = Az * math.cos(W * tau) + Bz * math.sin(W * tau)
        return y, z

    def dt_dtau(tau):
        y, z = pos(tau)
        return 2 * omega * n0 ** 2 * (1 - a ** 2 * (y * y + z * z))

    tau = _invert_monotone(t_of, dt_dtau, T)
    y, z = pos(tau)
    ky = (-Ay * W * math.sin(W * tau) + By * W * math.cos(W * tau)) / 2
    kz = (-Az * W * math.sin(W * tau) + Bz * W * math.cos(W * tau)) / 2
    return np.array([x0[0] + 2 * k0[0] * tau, y, z]), np.array([k0[0], ky, kz])


def quadratic(p, u, T):
    """n^2 = 2 - |x|^2 everywhere, w = 1, start x = p with k = u on shell (|u|^2 = 2 - |p|^2).

    x = p cos 2tau + u sin 2tau, k = -p sin 2tau + u cos 2tau,
    t = 2 tau + (|u|^2 - |p|^2) sin(4 tau)/4 - (p.u)(1 - cos 4 tau)/2.
    """
    p = np.asarray(p, float)
    u = np.asarray(u, float)
    uu, pp, pu = u @ u, p @ p, p @ u

    def t_of(tau):
        return 2 * tau + (uu - pp) * math.sin(4 * tau) / 4 - pu * (1 - math.cos(4 * tau)) / 2

    def dt_dtau(tau):
        x = p * math.cos(2 * tau) + u * math.sin(2 * tau)
        return 2 * (2 - x @ x)

    tau = _invert_monotone(t_of, dt_dtau, T)
    x = p * math.cos(2 * tau) + u * math.sin(2 * tau)
    k = -p * math.sin(2 * tau) + u * math.cos(2 * tau)
    return x, k


def luneburg_from_plane(y0, z0, T):
    """Luneburg lens (w = 1) ray launched at (-1, y0, z0) along +x, at time T.

    Straight at unit speed until the unit sphere at p = (-sqrt(1 - rho^2), y0, z0),
    reached at t_e = 1 + p_x; inside, the quadratic-law ellipse from p with k = +x;
    every ray reaches the focus (1, 0, 0) at t = 1 + pi/2.  Valid for T up to the
    focus.
    """
    px = -math.sqrt(1 - y0 * y0 - z0 * z0)
    te = 1 + px
    if T <= te:
        return np.array([-1 + T, y0, z0]), np.array([1.0, 0, 0])
    return quadratic(np.array([px, y0, z0]), np.array([1.0, 0, 0]), T - te)
