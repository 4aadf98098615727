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
GF_F32, GF_F64 = 0, 1
KINDS = {"homog": 0, "luneburg": 1, "grin": 2, "quadratic": 3, "spline": 4}
(GF_RAY_ACTIVE, GF_RAY_EXITED, GF_RAY_CUTOFF, GF_RAY_NONFINITE, GF_RAY_MAX_STEPS,
 GF_RAY_STEP_UNDERFLOW, GF_RAY_DONE) = range(7)
GF_MAX_BLOBS = 64


class GfMediumDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_blobs", C.c_int32), ("grid_n", C.c_int32),
                ("reserved", C.c_int32), ("n_h", C.c_double), ("n0", C.c_double), ("a", C.c_double),
                ("blobs", C.c_void_p), ("grid", C.c_void_p)]


class GfRays(C.Structure):
    _fields_ = [("n", C.c_int64), ("ld", C.c_int64), ("y", C.c_void_p), ("t", C.c_void_p),
                ("status", C.c_void_p), ("steps", C.c_void_p), ("d_res", C.c_void_p),
                ("d_max", C.c_void_p)]


class GfStepCtl(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double),
                ("t_max", C.c_double), ("radius", C.c_double), ("fac_min", C.c_double),
                ("fac_max", C.c_double), ("safety", C.c_double), ("max_steps", C.c_int64)]


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
            "gf_bench_fma_peak": ([I32, I64, I32, P, P], I32),
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
                     blobs=None, grid=None) -> Medium:
    """Copy a medium to the current device (see gf_medium_create in gf.h)."""
    b = None if blobs is None or len(blobs) == 0 else \
        np.ascontiguousarray(np.asarray(blobs, dtype=np.float64).reshape(-1, 5))
    g = None if grid is None else np.ascontiguousarray(np.asarray(grid, dtype=np.float32))
    desc = GfMediumDesc(KINDS[kind], 0 if b is None else b.shape[0], 0 if g is None else g.shape[0],
                        0, n_h, n0, a, None if b is None else b.ctypes.data,
                        None if g is None else g.ctypes.data)
    h = C.c_void_p()
    _check("gf_medium_create", lib().gf_medium_create(C.byref(desc), C.byref(h)))
    return Medium(h.value, kind, desc.n_blobs)


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


def gf_trace_rk4(m: Medium, rays: Rays, omega: float, dt: float, n_steps: int, radius: float = 0.0,
                 checkpoint_every: int = 0, ckpt: torch.Tensor | None = None, stream=None) -> None:
    """Advance active rays by n_steps fixed RK4 steps in place (see gf.h)."""
    s = rays.struct()
    _check("gf_trace_rk4", lib().gf_trace_rk4(m.handle, rays.precision, C.byref(s), omega, dt,
                                              int(n_steps), radius, int(checkpoint_every),
                                              _ptr(ckpt), _stream(stream)))


def trace_host(m: Medium, x0_host: torch.Tensor, dir_host: torch.Tensor, omega: float, dt: float,
               n_steps: int, rays: Rays | None = None, dirs: torch.Tensor | None = None,
               out: dict | None = None, radius: float = 0.0) -> dict:
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
    gf_trace_rk4(m, rays, omega, dt, n_steps, radius)
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


def medium_from_workload(spec: dict) -> Medium:
    """gf_medium_create from a workload's medium dictionary (see workloads.py)."""
    return gf_medium_create(**spec)
