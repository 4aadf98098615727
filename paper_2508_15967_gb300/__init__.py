"""GB300-native Hamiltonian ray tracing -- Python binding of libgf.so.

This module only marshals arguments: torch tensors (device memory and the
caller's CUDA stream) are turned into the plain pointers and sizes of the C
ABI in ``include/gf.h``; every step of the computation runs in the library's
CUDA kernels.  Functions carry the C names.  If ``libgf.so`` has not been
built the import of the binding fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgf.so")

GF_OK, GF_ERR_INVALID_ARG, GF_ERR_CUDA, GF_ERR_OOM, GF_ERR_UNSUPPORTED, GF_ERR_TIMEOUT = range(6)
GF_F32, GF_F64, GF_F64X = 0, 1, 2
KINDS = {"homog": 0, "luneburg": 1, "grin": 2, "quadratic": 3, "spline": 4, "cold": 5}
(GF_RAY_ACTIVE, GF_RAY_EXITED, GF_RAY_CUTOFF, GF_RAY_NONFINITE, GF_RAY_MAX_STEPS,
 GF_RAY_STEP_UNDERFLOW, GF_RAY_DONE) = range(7)
GF_MAX_BLOBS = 64


class GfMediumDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_blobs", C.c_int32), ("grid_n", C.c_int32),
                ("reserved", C.c_int32), ("n_h", C.c_double), ("n0", C.c_double), ("a", C.c_double),
                ("blobs", C.c_void_p), ("grid", C.c_void_p), ("n_species", C.c_int32),
                ("reserved2", C.c_int32), ("species", C.c_double * 8), ("profile", C.c_double * 4)]


class GfRays(C.Structure):
    _fields_ = [("n", C.c_int64), ("ld", C.c_int64), ("y", C.c_void_p), ("t", C.c_void_p),
                ("status", C.c_void_p), ("steps", C.c_void_p), ("d_res", C.c_void_p),
                ("d_max", C.c_void_p)]


class GfStepCtl(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double),
                ("t_max", C.c_double), ("radius", C.c_double), ("fac_min", C.c_double),
                ("fac_max", C.c_double), ("safety", C.c_double), ("max_steps", C.c_int64)]


class GfTune(C.Structure):
    _fields_ = [("block", C.c_int32), ("rays_per_thread", C.c_int32), ("compaction", C.c_int32),
                ("chunk", C.c_int32)]

    def as_tuple(self):
        return (self.block, self.rays_per_thread, self.compaction, self.chunk)


GF_SCHED_PERSISTENT, GF_SCHED_PER_MEDIUM = 0, 1
GF_MAX_BATCH_BLOBS = 16


class GfError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """The loaded libgf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgf.so not found at {LIB_PATH}; build it with "
                               "`python -m paper_2508_15967_gb300.build`")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sigs = {
            "gf_last_error": ([], C.c_char_p),
            "gf_version": ([], I32),
            "gf_medium_create": ([P, P], I32),
            "gf_medium_destroy": ([P], I32),
            "gf_medium_set_amplitudes": ([P, P, P], I32),
            "gf_rays_onshell": ([P, I32, P, P, D, P], I32),
            "gf_trace_rk4": ([P, I32, P, D, D, I64, D, I64, P, P], I32),
            "gf_rays_newton_kx": ([P, I32, P, D, D, I32, P], I32),
            "gf_bench_fma_peak": ([I32, I64, I32, P, P], I32),
            "gf_bench_set_counters": ([P], I32),
            "gf_bench_exp": ([P, P, P, I64, P], I32),
            "gf_bench_exp_df": ([P, P, I64, P], I32),
            "gf_bench_exp_fp": ([P, P, I64, P], I32),
            "gf_bench_blob_gauss": ([P, P, P, I64, P], I32),
            "gf_bench_recip": ([P, P, P, I64, P], I32),
            "gf_fault_inject": ([I64], I32),
            "gf_bench_live_allocations": ([P], I64),
            "gf_adjoint_scratch_bytes": ([P, I64, I64], C.c_size_t),
            "gf_trace_adjoint": ([P, I64, D, D, I64, I64, P, P, P, I64, P, P, P, C.c_size_t, P], I32),
            "gf_trace_adjoint_static": ([P, I64, D, D, I64, I64, P, P, P, I64, P, P, P], I32),
            "gf_jit_medium_create": ([C.c_char_p, P], I32),
            "gf_jit_compile_check": ([C.c_char_p, C.c_char_p, C.c_char_p, C.c_size_t], I32),
            "gf_batch_create": ([P, I32, P, P], I32),
            "gf_batch_destroy": ([P], I32),
            "gf_trace_dopri5": ([P, P, P, D, P, I32, P, P], I32),
            "gf_batch_set_precision": ([P, I32], I32),
            "gf_dopri5_autotune": ([P, P, D, P, C.c_char_p, P], I32),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(fn: str, status: int) -> None:
    if status != GF_OK:
        raise GfError(fn, status, lib().gf_last_error().decode())


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


# --------------------------------------------------------------------------- media

class Medium:
    """Handle of a device-resident medium (owns it; destroyed with the object)."""

    def __init__(self, handle: int, kind: str, n_blobs: int):
        self.handle = handle
        self.kind = kind
        self.n_blobs = n_blobs

    def close(self) -> None:
        if self.handle:
            lib().gf_medium_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gf_medium_create(kind: str, *, n_h: float = 1.0, n0: float = 1.5, a: float = 2.0,
                     blobs=None, grid=None, species=(), profile=(1.0, 0.0, 1.0, 0.0)) -> Medium:
    """Copy a medium to the current device (see gf_medium_create in gf.h).
    Cold plasma: species = ((w_p^2, Omega), ...), profile = (f0, f1, g0, g1)."""
    b = None if blobs is None or len(blobs) == 0 else \
        np.ascontiguousarray(np.asarray(blobs, dtype=np.float64).reshape(-1, 5))
    g = None if grid is None else np.ascontiguousarray(np.asarray(grid, dtype=np.float32))
    sp = [0.0] * 8
    for i, (wp2, om) in enumerate(species):
        sp[2 * i], sp[2 * i + 1] = wp2, om
    desc = GfMediumDesc(KINDS[kind], 0 if b is None else b.shape[0], 0 if g is None else g.shape[0],
                        0, n_h, n0, a, None if b is None else b.ctypes.data,
                        None if g is None else g.ctypes.data, len(species), 0,
                        (C.c_double * 8)(*sp), (C.c_double * 4)(*profile))
    h = C.c_void_p()
    _check("gf_medium_create", lib().gf_medium_create(C.byref(desc), C.byref(h)))
    return Medium(h.value, kind, desc.n_blobs)


def gf_jit_medium_create(source: str) -> Medium:
    """Compile generated CUDA source of gf_user_dispersion into an RK4 medium (see gf.h)."""
    h = C.c_void_p()
    _check("gf_jit_medium_create", lib().gf_jit_medium_create(source.encode(), C.byref(h)))
    return Medium(h.value, "generated", 0)


def gf_jit_compile_check(source: str, arch: str = "sm_103a") -> tuple[int, str]:
    """(status, compiler log) of compiling generated source without loading it."""
    buf = C.create_string_buffer(1 << 16)
    st = lib().gf_jit_compile_check(source.encode(), arch.encode(), buf, len(buf))
    return st, buf.value.decode(errors="replace")


def gf_medium_destroy(m: Medium) -> None:
    m.close()


def gf_medium_set_amplitudes(m: Medium, amplitudes: torch.Tensor, stream=None) -> None:
    a = amplitudes.detach().to(dtype=torch.float64).contiguous()
    _check("gf_medium_set_amplitudes",
           lib().gf_medium_set_amplitudes(m.handle, _ptr(a), _stream(stream)))


# --------------------------------------------------------------------------- rays

@dataclass
class Rays:
    """Device ray buffers in the library's layout: y is (6, ld), rows x y z kx ky kz."""
    y: torch.Tensor
    t: torch.Tensor
    status: torch.Tensor
    steps: torch.Tensor
    d_res: torch.Tensor | None
    d_max: torch.Tensor | None

    @property
    def n(self) -> int:
        return self.t.shape[0]

    @property
    def precision(self) -> int:
        return GF_F64 if self.y.dtype == torch.float64 else GF_F32

    @classmethod
    def empty(cls, n: int, dtype=torch.float64, device="cuda", diagnostics: bool = True) -> "Rays":
        z = lambda dt: torch.zeros(n, dtype=dt, device=device)
        return cls(torch.zeros(6, n, dtype=dtype, device=device), z(torch.float64), z(torch.int32),
                   z(torch.int32), z(torch.float64) if diagnostics else None,
                   z(torch.float64) if diagnostics else None)

    @classmethod
    def from_numpy(cls, x0, k0=None, dtype=torch.float64, device="cuda") -> "Rays":
        x0 = np.asarray(x0, dtype=np.float64).reshape(-1, 3)
        r = cls.empty(x0.shape[0], dtype, device)
        state = np.zeros((6, x0.shape[0]))
        state[:3] = x0.T
        if k0 is not None:
            state[3:] = np.asarray(k0, dtype=np.float64).reshape(-1, 3).T
        r.y.copy_(torch.from_numpy(state).to(dtype))
        return r

    def struct(self) -> GfRays:
        if self.y.dim() != 2 or self.y.shape[0] != 6 or self.y.stride(1) != 1:
            raise ValueError("rays.y must be a (6, ld) tensor with unit inner stride")
        return GfRays(self.n, self.y.stride(0), _ptr(self.y), _ptr(self.t), _ptr(self.status),
                      _ptr(self.steps), _ptr(self.d_res), _ptr(self.d_max))

    def state(self) -> np.ndarray:
        """(n, 6) float64 host copy of the state."""
        return self.y[:, :self.n].double().T.cpu().numpy()

    def clone(self) -> "Rays":
        return Rays(*(None if v is None else v.clone() for v in
                      (self.y, self.t, self.status, self.steps, self.d_res, self.d_max)))


def gf_rays_onshell(m: Medium, rays: Rays, direction: torch.Tensor, omega: float = 1.0,
                    stream=None) -> None:
    """Set k on shell along `direction` ((3, ld) device tensor of the rays' dtype)."""
    if direction.dtype != rays.y.dtype or direction.stride(0) != rays.y.stride(0):
        raise ValueError("direction must be (3, ld) with the dtype and row stride of rays.y")
    s = rays.struct()
    _check("gf_rays_onshell", lib().gf_rays_onshell(m.handle, rays.precision, C.byref(s),
                                                    _ptr(direction), omega, _stream(stream)))


def gf_rays_newton_kx(m: Medium, rays: Rays, omega: float = 1.0, tol: float = 1e-15,
                      max_iter: int = 50, stream=None) -> None:
    """Solve D = 0 for k_x by Newton from the k_x in rays.y[3] (k_y, k_z fixed)."""
    s = rays.struct()
    _check("gf_rays_newton_kx", lib().gf_rays_newton_kx(m.handle, rays.precision, C.byref(s), omega, tol,
                                                        max_iter, _stream(stream)))


def gf_trace_rk4(m: Medium, rays: Rays, omega: float, dt: float, n_steps: int, radius: float = 0.0,
                 checkpoint_every: int = 0, ckpt: torch.Tensor | None = None, stream=None,
                 precision: int | None = None) -> None:
    """Advance active rays by n_steps fixed RK4 steps in place (see gf.h).
    precision: None = from the ray dtype (GF_F64 / GF_F32); GF_F64X for float64 rays."""
    s = rays.struct()
    prec = rays.precision if precision is None else precision
    if prec == GF_F64X and rays.y.dtype != torch.float64:
        raise ValueError("GF_F64X needs float64 rays")
    _check("gf_trace_rk4", lib().gf_trace_rk4(m.handle, prec, C.byref(s), omega, dt,
                                              int(n_steps), radius, int(checkpoint_every),
                                              _ptr(ckpt), _stream(stream)))


# --------------------------------------------------------------------------- adjoint

def gf_adjoint_scratch_bytes(m: Medium, n: int, checkpoint_every: int) -> int:
    return int(lib().gf_adjoint_scratch_bytes(m.handle, n, checkpoint_every))


def gf_trace_adjoint(m: Medium, n: int, omega: float, dt: float, n_steps: int, checkpoint_every: int,
                     ckpt: torch.Tensor, steps_done: torch.Tensor, lam: torch.Tensor,
                     dtheta: torch.Tensor, dy0: torch.Tensor | None = None,
                     scratch: torch.Tensor | None = None, stream=None) -> None:
    """dL/dtheta (and dL/dy0) of the RK4 trace from its checkpoints (see gf.h)."""
    need = gf_adjoint_scratch_bytes(m, n, checkpoint_every)
    if scratch is None:
        scratch = torch.empty(max(need, 1), dtype=torch.uint8, device=dtheta.device)
    if lam.stride(1) != 1 or (dy0 is not None and dy0.stride(0) != lam.stride(0)):
        raise ValueError("lam and dy0 must be (6, ld) with unit inner stride and the same ld")
    _check("gf_trace_adjoint", lib().gf_trace_adjoint(
        m.handle, n, omega, dt, int(n_steps), int(checkpoint_every), _ptr(ckpt), _ptr(steps_done),
        _ptr(lam), lam.stride(0), _ptr(dtheta), _ptr(dy0), _ptr(scratch), scratch.numel(),
        _stream(stream)))


def gf_trace_adjoint_static(m: Medium, n: int, omega: float, dt: float, n_steps: int,
                            checkpoint_every: int, ckpt: torch.Tensor, steps_done: torch.Tensor,
                            lam: torch.Tensor, dtheta: torch.Tensor, dy0: torch.Tensor | None = None,
                            stream=None) -> None:
    """gf_trace_adjoint with the library's fixed 64 MiB scratch: no device allocation (see gf.h)."""
    if lam.stride(1) != 1 or (dy0 is not None and dy0.stride(0) != lam.stride(0)):
        raise ValueError("lam and dy0 must be (6, ld) with unit inner stride and the same ld")
    _check("gf_trace_adjoint_static", lib().gf_trace_adjoint_static(
        m.handle, n, omega, dt, int(n_steps), int(checkpoint_every), _ptr(ckpt), _ptr(steps_done),
        _ptr(lam), lam.stride(0), _ptr(dtheta), _ptr(dy0), _stream(stream)))


class TraceRK4(torch.autograd.Function):
    """y_N = RK4 trace of y0 through a medium whose blob amplitudes are theta.

    forward: gf_medium_set_amplitudes + gf_trace_rk4 with checkpoints every
    `checkpoint_every` steps; backward: gf_trace_adjoint.  y0 and the output
    are (6, n) float64 device tensors (rows x y z kx ky kz)."""

    @staticmethod
    def forward(ctx, theta, y0, medium, omega, dt, n_steps, checkpoint_every):
        gf_medium_set_amplitudes(medium, theta)
        n = y0.shape[1]
        rays = Rays.empty(n, torch.float64, y0.device, diagnostics=False)
        rays.y.copy_(y0.detach())
        n_ckpt = max(1, -(-int(n_steps) // int(checkpoint_every)))
        ckpt = torch.empty((n_ckpt, 6, n), dtype=torch.float64, device=y0.device)
        gf_trace_rk4(medium, rays, omega, dt, n_steps, 0.0, checkpoint_every, ckpt)
        ctx.save_for_backward(theta.detach(), ckpt, rays.steps)
        ctx.medium, ctx.omega, ctx.dt, ctx.n_steps, ctx.every = medium, omega, dt, n_steps, checkpoint_every
        return rays.y

    @staticmethod
    def backward(ctx, grad_y):
        theta, ckpt, steps = ctx.saved_tensors
        m = ctx.medium
        gf_medium_set_amplitudes(m, theta)
        lam = grad_y.to(torch.float64).contiguous()
        n = lam.shape[1]
        dtheta = torch.empty(m.n_blobs, dtype=torch.float64, device=lam.device)
        dy0 = torch.empty_like(lam) if ctx.needs_input_grad[1] else None
        gf_trace_adjoint(m, n, ctx.omega, ctx.dt, ctx.n_steps, ctx.every, ckpt, steps, lam, dtheta, dy0)
        return dtheta, dy0, None, None, None, None, None


def trace_rk4_autograd(medium: Medium, theta: torch.Tensor, y0: torch.Tensor, omega: float, dt: float,
                       n_steps: int, checkpoint_every: int = 64) -> torch.Tensor:
    """Differentiable RK4 trace: returns y_N (6, n); gradients flow to theta and y0."""
    return TraceRK4.apply(theta, y0, medium, omega, dt, n_steps, checkpoint_every)


# --------------------------------------------------------------------------- batched DOPRI5

class Batch:
    """Handle of a device-resident batch of media (owns it)."""

    def __init__(self, handle: int, n_media: int, offsets: np.ndarray):
        self.handle = handle
        self.n_media = n_media
        self.offsets = offsets

    def close(self) -> None:
        if self.handle:
            lib().gf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gf_batch_create(media: list, offsets) -> Batch:
    """Gather media (rays of medium j at [offsets[j], offsets[j+1])) into a batch."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if off.shape[0] != len(media) + 1:
        raise ValueError("offsets must have len(media) + 1 entries")
    arr = (C.c_void_p * len(media))(*[m.handle for m in media])
    h = C.c_void_p()
    _check("gf_batch_create", lib().gf_batch_create(arr, len(media), off.ctypes.data, C.byref(h)))
    return Batch(h.value, len(media), off)


def gf_batch_set_precision(b: Batch, precision: int) -> None:
    """GF_F64 (default) or GF_F64X (double-float blob sums) for later DOPRI5 calls."""
    _check("gf_batch_set_precision", lib().gf_batch_set_precision(b.handle, precision))


def gf_batch_destroy(b: Batch) -> None:
    b.close()


def step_ctl(rtol=1e-9, atol=1e-9, h0=1e-3, t_max=10.0, radius=1.5, fac_min=0.2, fac_max=10.0,
             safety=0.9, max_steps=100000) -> GfStepCtl:
    return GfStepCtl(rtol, atol, h0, t_max, radius, fac_min, fac_max, safety, max_steps)


def gf_trace_dopri5(b: Batch, rays: Rays, rejects: torch.Tensor | None = None, omega: float = 1.0,
                    ctl: GfStepCtl | None = None, sched: int = GF_SCHED_PERSISTENT,
                    tune: GfTune | tuple | None = None, stream=None) -> None:
    """Adaptive DOPRI5 over every active ray of the batch, in place (see gf.h)."""
    s = rays.struct()
    c = ctl if ctl is not None else step_ctl()
    t = GfTune(*tune) if isinstance(tune, tuple) else tune
    _check("gf_trace_dopri5", lib().gf_trace_dopri5(b.handle, C.byref(s), _ptr(rejects), omega,
                                                    C.byref(c), sched,
                                                    None if t is None else C.byref(t), _stream(stream)))


def gf_dopri5_autotune(b: Batch, rays: Rays, omega: float = 1.0, ctl: GfStepCtl | None = None,
                       cache_path: str | None = None) -> GfTune:
    """Pick block x rays/thread x compaction x chunk for the persistent schedule."""
    s = rays.struct()
    c = ctl if ctl is not None else step_ctl()
    out = GfTune()
    _check("gf_dopri5_autotune", lib().gf_dopri5_autotune(
        b.handle, C.byref(s), omega, C.byref(c), None if cache_path is None else cache_path.encode(),
        C.byref(out)))
    return out


def trace_host(m: Medium, x0_host: torch.Tensor, dir_host: torch.Tensor, omega: float, dt: float,
               n_steps: int, rays: Rays | None = None, dirs: torch.Tensor | None = None,
               out: dict | None = None, radius: float = 0.0, precision: int | None = None) -> dict:
    """End-to-end call on host buffers: copy launch points and directions
    ((3, n) host tensors, pinned for overlap) to the device, set the rays on
    shell, trace n_steps RK4 steps, and copy every ray buffer back.  Device
    buffers may be passed in for reuse.  Returns the host dict y, t, status,
    steps, d_res, d_max."""
    n = x0_host.shape[1]
    if rays is None:
        rays = Rays.empty(n, x0_host.dtype)
    if dirs is None:
        dirs = torch.empty((3, n), dtype=x0_host.dtype, device=rays.y.device)
    rays.y[:3].copy_(x0_host, non_blocking=True)
    dirs.copy_(dir_host, non_blocking=True)
    rays.t.zero_()
    rays.status.zero_()
    rays.steps.zero_()
    rays.d_max.zero_()
    gf_rays_onshell(m, rays, dirs, omega)
    gf_trace_rk4(m, rays, omega, dt, n_steps, radius, precision=precision)
    if out is None:
        out = {k: torch.empty(getattr(rays, k).shape, dtype=getattr(rays, k).dtype).pin_memory()
               for k in ("y", "t", "status", "steps", "d_res", "d_max")}
    for k, v in out.items():
        v.copy_(getattr(rays, k), non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return out


def gf_bench_fma_peak(precision: int, iters: int = 1 << 16, blocks_per_sm: int = 8):
    """(TFLOP/s, ms) of an FMA-chain kernel in FP64 or FP32 on the current device."""
    tf, ms = C.c_double(), C.c_double()
    _check("gf_bench_fma_peak", lib().gf_bench_fma_peak(precision, iters, blocks_per_sm,
                                                        C.byref(tf), C.byref(ms)))
    return tf.value, ms.value


def gf_bench_set_counters(counters: torch.Tensor | None) -> None:
    """Route RK4 work counts (evaluations, blob terms) into a 2-element int64 device tensor."""
    _check("gf_bench_set_counters", lib().gf_bench_set_counters(_ptr(counters)))


def gf_bench_exp(a: torch.Tensor):
    """(library 2^a, CUDA exp2) of a float64 device tensor."""
    a = a.contiguous()
    o1, o2 = torch.empty_like(a), torch.empty_like(a)
    _check("gf_bench_exp", lib().gf_bench_exp(_ptr(a), _ptr(o1), _ptr(o2), a.numel(), _stream(None)))
    return o1, o2


def gf_bench_exp_fp(a: torch.Tensor) -> torch.Tensor:
    """The library's 2^a in its FP64-FMA form, of a float64 device tensor."""
    a = a.contiguous()
    o = torch.empty_like(a)
    _check("gf_bench_exp_fp", lib().gf_bench_exp_fp(_ptr(a), _ptr(o), a.numel(), _stream(None)))
    return o


def gf_bench_blob_gauss(u: torch.Tensor):
    """(integer-form, FMA-form) blob Gaussians 2^-|u|^2 of a float64 device tensor of shape (3, n)."""
    u = u.contiguous()
    n = u.shape[1]
    o1 = torch.empty(n, dtype=torch.float64, device=u.device)
    o2 = torch.empty_like(o1)
    _check("gf_bench_blob_gauss", lib().gf_bench_blob_gauss(_ptr(u), _ptr(o1), _ptr(o2), n, _stream(None)))
    return o1, o2


def gf_bench_exp_df(a: torch.Tensor) -> torch.Tensor:
    """Double-float 2^a of a float64 device tensor (hi + lo returned as float64)."""
    a = a.contiguous()
    o = torch.empty_like(a)
    _check("gf_bench_exp_df", lib().gf_bench_exp_df(_ptr(a), _ptr(o), a.numel(), _stream(None)))
    return o


def gf_bench_recip(a: torch.Tensor):
    """(FP64 evaluator's 1/a for a > 0 else 0, float truncation of a) of a float64 device tensor."""
    a = a.contiguous()
    o1 = torch.empty_like(a)
    o2 = torch.empty(a.shape, dtype=torch.float32, device=a.device)
    _check("gf_bench_recip", lib().gf_bench_recip(_ptr(a), _ptr(o1), _ptr(o2), a.numel(), _stream(None)))
    return o1, o2


def gf_fault_inject(n: int) -> None:
    """Make the n-th CUDA call the library checks from now on report an
    injected failure (n <= 0 disarms); see gf_bench.h."""
    _check("gf_fault_inject", lib().gf_fault_inject(int(n)))


def gf_bench_live_allocations() -> tuple[int, int]:
    """(number, total bytes) of the device allocations the library holds."""
    nbytes = C.c_size_t(0)
    n = lib().gf_bench_live_allocations(C.byref(nbytes))
    return int(n), int(nbytes.value)


def medium_from_workload(spec: dict) -> Medium:
    """gf_medium_create from a workload's medium dictionary (see workloads.py)."""
    return gf_medium_create(**spec)
