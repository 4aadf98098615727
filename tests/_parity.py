"""Helpers of the GPU parity tests: run the same seeded rays through the CUDA
library (through its C ABI) and through the FP64 oracle, and compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
import paper_2508_15967_gb300 as gf


def rel_err(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-ray error of state a against reference b, both (n, 6):
    max(|dx| / max(|x_b|, 1), |dk| / max(|k_b|, 1)) in Euclidean norms."""
    ex = np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.maximum(np.linalg.norm(b[:, :3], axis=1), 1.0)
    ek = np.linalg.norm(a[:, 3:] - b[:, 3:], axis=1) / np.maximum(np.linalg.norm(b[:, 3:], axis=1), 1.0)
    return np.maximum(ex, ek)


def oracle_medium(spec: dict) -> O.Medium:
    return O.medium(**spec)


def oracle_rk4(spec, x0, k0, omega, dt, n_steps, radius=0.0, status=None, every=0):
    r = O.make_rays(x0, k0, status=status)
    ck = O.trace_rk4(oracle_medium(spec), r, omega, dt, n_steps, radius, every)
    return r, ck


class GpuResult:
    def __init__(self, rays: gf.Rays):
        torch.cuda.synchronize()
        self.y = rays.state()
        self.t = rays.t.cpu().numpy()
        self.status = rays.status.cpu().numpy()
        self.steps = rays.steps.cpu().numpy()
        self.dres = rays.d_res.cpu().numpy()
        self.dmax = rays.d_max.cpu().numpy()


def gpu_rk4(spec, x0, k0, omega, dt, n_steps, radius=0.0, dtype=torch.float64, status=None,
            ckpt_every=0):
    m = gf.gf_medium_create(**spec)
    rays = gf.Rays.from_numpy(x0, k0, dtype)
    if status is not None:
        rays.status.copy_(torch.as_tensor(status, dtype=torch.int32))
    ck = None
    if ckpt_every:
        nck = (n_steps + ckpt_every - 1) // ckpt_every
        ck = torch.full((nck, 6, rays.n), float("nan"), dtype=torch.float64, device="cuda")
    gf.gf_trace_rk4(m, rays, omega, dt, n_steps, radius, ckpt_every, ck)
    res = GpuResult(rays)
    if ck is not None:
        res.ckpt = ck.cpu().numpy()
    return res


def conditioning_mask(spec, x0, k0, omega, dt, n_steps, ref_y, floor=1e-10, rel_perturb=None):
    """Rays whose oracle result moves by more than `floor` when the launch point
    is perturbed by one ulp (FP64: nextafter; FP32 scale: rel_perturb = 2^-23):
    ill-conditioned at that precision, excluded from the gate and counted."""
    x1 = np.nextafter(x0, np.inf) if rel_perturb is None else x0 * (1 + rel_perturb)
    r, _ = oracle_rk4(spec, x1, k0, omega, dt, n_steps)
    return rel_err(r.y, ref_y) > floor


def assert_parity(g: GpuResult, o: O.Rays, tol: float, cond_mask=None, diag_atol=1e-12,
                  min_keep=0.99):
    assert np.array_equal(g.status, o.status), (np.bincount(g.status), np.bincount(o.status))
    assert np.array_equal(g.steps, o.steps)
    e = rel_err(g.y, o.y)
    keep = np.ones(len(e), bool) if cond_mask is None else ~cond_mask
    assert keep.sum() >= min_keep * len(e), f"{(~keep).sum()} ill-conditioned rays"
    worst = e[keep].max() if keep.any() else 0.0
    assert worst <= tol, f"max rel err {worst:.3e} > {tol:.1e} (ray {np.argmax(np.where(keep, e, 0))})"
    np.testing.assert_allclose(g.t, o.t, rtol=1e-15, atol=0)
    np.testing.assert_allclose(g.dres, o.dres, rtol=1e-9, atol=diag_atol)
    np.testing.assert_allclose(g.dmax, o.dmax, rtol=1e-9, atol=diag_atol)
    return worst
