"""Plain FP64 CPU oracle for Hamiltonian ray tracing (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package.  The arithmetic lives in ``oracle.c`` (plain C, -O2
-ffp-contract=off, OpenMP over independent rays); this module only builds it
and marshals numpy arrays.  It shares nothing with the CUDA library.

Layouts: rays are (n, 6) float64 rows (x, y, z, kx, ky, kz); t, dres, dmax are
(n,) float64; status, steps, rejects are (n,) int32.  Status codes:
0 active, 1 exited, 2 cut-off, 3 non-finite, 4 max-steps, 5 step-underflow,
6 reached t_max.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KIND = {"homog": 0, "luneburg": 1, "grin": 2, "quadratic": 3, "spline": 4, "cold": 5}
ACTIVE, EXITED, CUTOFF, NONFINITE, MAX_STEPS, STEP_UNDERFLOW, DONE = range(7)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=gnu11", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Medium(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_blobs", C.c_int32), ("grid_n", C.c_int32),
                ("pad_", C.c_int32), ("n_h", C.c_double), ("n0", C.c_double),
                ("a", C.c_double), ("blobs", C.c_void_p), ("grid", C.c_void_p),
                ("n_species", C.c_int32), ("pad2_", C.c_int32), ("species", C.c_double * 8),
                ("prof", C.c_double * 4)]


class _StepCtl(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double),
                ("t_max", C.c_double), ("radius", C.c_double), ("fac_min", C.c_double),
                ("fac_max", C.c_double), ("safety", C.c_double), ("max_steps", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        I64, D = C.c_int64, C.c_double
        _lib.or_eval.argtypes = [P, I64, P, P, D, P]
        _lib.or_index_hess.argtypes = [P, I64, P, P]
        _lib.or_onshell.argtypes = [P, I64, P, P, D, P, P]
        _lib.or_trace_rk4.argtypes = [P, I64, P, P, P, P, P, P, D, D, I64, D, I64, P]
        _lib.or_newton_kx.argtypes = [P, I64, P, P, D, D, C.c_int, P, P]
        _lib.or_trace_rk4_kink.argtypes = [P, I64, P, P, P, P, P, P, D, D, I64, D, P]
        _lib.or_trace_dopri5.argtypes = [P, I64, P, P, P, P, P, P, P, P, D, P]
        _lib.or_tangent_rk4.argtypes = [P, I64, P, P, P, P, P, D, D, I64, D]
        _lib.or_loss_grad.argtypes = [I64, C.c_int, P, P, P, P]
        _lib.or_dopri5_tableau.argtypes = [P]
        _lib.or_num_threads.restype = C.c_int
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


@dataclass
class Medium:
    """Medium description; keeps the arrays alive while the C struct points at them."""
    kind: str = "homog"
    n_h: float = 1.0
    n0: float = 1.5
    a: float = 2.0
    blobs: np.ndarray | None = None
    grid: np.ndarray | None = None
    species: tuple = ()          # cold plasma: ((w_p^2, Omega), ...) at f = g = 1
    profile: tuple = (1.0, 0.0, 1.0, 0.0)   # (f0, f1, g0, g1)

    def struct(self) -> _Medium:
        self._blobs = None if self.blobs is None or len(self.blobs) == 0 else \
            np.ascontiguousarray(self.blobs, dtype=np.float64).reshape(-1, 5)
        self._grid = None if self.grid is None else np.ascontiguousarray(self.grid, dtype=np.float32)
        nb = 0 if self._blobs is None else self._blobs.shape[0]
        gn = 0 if self._grid is None else self._grid.shape[0]
        if self.kind == "spline" and self._grid is None:
            raise ValueError("spline medium needs a grid")
        sp = np.zeros(8)
        for i, (wp2, om) in enumerate(self.species):
            sp[2 * i], sp[2 * i + 1] = wp2, om
        return _Medium(KIND[self.kind], nb, gn, 0, self.n_h, self.n0, self.a,
                       _p(self._blobs), _p(self._grid), len(self.species), 0,
                       (C.c_double * 8)(*sp), (C.c_double * 4)(*self.profile))


def medium(**kw) -> Medium:
    return Medium(**kw)


def eval_dispersion(m: Medium, x, k, omega: float = 1.0) -> np.ndarray:
    """(n, 9) rows (D, Dx[3], Dk[3], Dw, eps)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    k = np.ascontiguousarray(k, dtype=np.float64).reshape(-1, 3)
    out = np.empty((x.shape[0], 9))
    s = m.struct()
    lib().or_eval(C.byref(s), x.shape[0], _p(x), _p(k), omega, _p(out))
    return out


def index_hess(m: Medium, x) -> np.ndarray:
    """(n, 13) rows (n2, grad[3], hess[9]) of an isotropic medium."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    out = np.empty((x.shape[0], 13))
    s = m.struct()
    lib().or_index_hess(C.byref(s), x.shape[0], _p(x), _p(out))
    return out


def onshell(m: Medium, x0, d, omega: float = 1.0):
    """k0 = s d with D(x0, k0, omega) = 0; returns (k0 (n,3), status (n,))."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    k0 = np.empty_like(x0)
    st = np.empty(x0.shape[0], dtype=np.int32)
    s = m.struct()
    lib().or_onshell(C.byref(s), x0.shape[0], _p(x0), _p(d), omega, _p(k0), _p(st))
    return k0, st


def newton_kx(m: Medium, x, k, omega: float = 1.0, tol: float = 1e-15, max_iter: int = 50):
    """Solve D = 0 for k_x by Newton from the k_x in k (k_y, k_z fixed).
    Returns (k (n,3), status (n,), iterations (n,))."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    k = np.array(k, dtype=np.float64).reshape(-1, 3)
    st = np.empty(x.shape[0], np.int32)
    it = np.empty(x.shape[0], np.int32)
    s = m.struct()
    lib().or_newton_kx(C.byref(s), x.shape[0], _p(x), _p(k), omega, tol, max_iter, _p(st), _p(it))
    return k, st, it


@dataclass
class Rays:
    y: np.ndarray          # (n, 6)
    t: np.ndarray
    status: np.ndarray
    steps: np.ndarray
    dres: np.ndarray
    dmax: np.ndarray
    rejects: np.ndarray | None = None

    @property
    def n(self) -> int:
        return self.y.shape[0]

    def copy(self) -> "Rays":
        return Rays(*(None if a is None else a.copy() for a in
                      (self.y, self.t, self.status, self.steps, self.dres, self.dmax, self.rejects)))


def make_rays(x0, k0, status=None, t0=None) -> Rays:
    x0 = np.asarray(x0, dtype=np.float64).reshape(-1, 3)
    n = x0.shape[0]
    y = np.ascontiguousarray(np.concatenate([x0, np.asarray(k0, np.float64).reshape(-1, 3)], axis=1))
    return Rays(y, np.zeros(n) if t0 is None else np.array(t0, dtype=np.float64),
                np.zeros(n, np.int32) if status is None else np.array(status, dtype=np.int32),
                np.zeros(n, np.int32), np.zeros(n), np.zeros(n), np.zeros(n, np.int32))


def trace_rk4(m: Medium, rays: Rays, omega: float, dt: float, n_steps: int,
              radius: float = 0.0, checkpoint_every: int = 0):
    """Advance rays in place; returns the checkpoint array (n, n_ckpt, 6) or None."""
    s = m.struct()
    ck = None
    if checkpoint_every > 0:
        nck = (n_steps + checkpoint_every - 1) // checkpoint_every
        ck = np.zeros((rays.n, nck, 6))
    lib().or_trace_rk4(C.byref(s), rays.n, _p(rays.y), _p(rays.t), _p(rays.status),
                       _p(rays.steps), _p(rays.dres), _p(rays.dmax), omega, dt, n_steps,
                       radius, checkpoint_every, _p(ck))
    return ck


def trace_rk4_kink(m: Medium, rays: Rays, omega: float, dt: float, n_steps: int,
                   radius: float = 0.0) -> np.ndarray:
    """trace_rk4 that also returns, per ray, min over stage points of ||x|^2 - 1|."""
    s = m.struct()
    kink = np.full(rays.n, np.inf)
    lib().or_trace_rk4_kink(C.byref(s), rays.n, _p(rays.y), _p(rays.t), _p(rays.status),
                            _p(rays.steps), _p(rays.dres), _p(rays.dmax), omega, dt, n_steps,
                            radius, _p(kink))
    return kink


def dopri5_tableau() -> np.ndarray:
    out = np.empty(63)
    lib().or_dopri5_tableau(_p(out))
    return out


def step_ctl(rtol=1e-9, atol=1e-9, h0=1e-3, t_max=10.0, radius=1.5, fac_min=0.2, fac_max=10.0,
             safety=0.9, max_steps=100000) -> _StepCtl:
    return _StepCtl(rtol, atol, h0, t_max, radius, fac_min, fac_max, safety, max_steps)


def trace_dopri5(media: list[Medium], offsets, rays: Rays, omega: float = 1.0, **ctl):
    """Adaptive DOPRI5 over many media; rays of medium j in [offsets[j], offsets[j+1])."""
    structs = (_Medium * len(media))(*[m.struct() for m in media])
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    c = step_ctl(**ctl)
    if rays.rejects is None:
        rays.rejects = np.zeros(rays.n, np.int32)
    lib().or_trace_dopri5(structs, len(media), _p(off), _p(rays.y), _p(rays.t), _p(rays.status),
                          _p(rays.steps), _p(rays.rejects), _p(rays.dres), _p(rays.dmax),
                          omega, C.byref(c))


def tangent_rk4(m: Medium, rays: Rays, omega: float, dt: float, n_steps: int, radius: float = 0.0):
    """Trace rays in place and return S = dy_N/dA, shape (n, 6, n_blobs)."""
    s = m.struct()
    nb = s.n_blobs
    S = np.zeros((rays.n, 6, nb))
    lib().or_tangent_rk4(C.byref(s), rays.n, _p(rays.y), _p(rays.t), _p(rays.status),
                         _p(rays.steps), _p(S), omega, dt, n_steps, radius)
    return S


def loss_grad(y_final, xstar, S) -> np.ndarray:
    y_final = np.ascontiguousarray(y_final, dtype=np.float64)
    xstar = np.ascontiguousarray(xstar, dtype=np.float64).reshape(-1, 3)
    S = np.ascontiguousarray(S, dtype=np.float64)
    nb = S.shape[2]
    g = np.empty(nb)
    lib().or_loss_grad(y_final.shape[0], nb, _p(y_final), _p(xstar), _p(S), _p(g))
    return g


def num_threads() -> int:
    return int(lib().or_num_threads())
