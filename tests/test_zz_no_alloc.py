"""The allocation-free adjoint entry point (gf_trace_adjoint_static), for
callers that cannot allocate device memory once running (for example a
real-time control loop, where cudaMalloc/cudaFree may block or synchronise
the device, or a host code whose GPU memory is reserved up front by its own
pool).  Its scratch is a fixed 64 MiB array inside the library; it must give
the same gradient as gf_trace_adjoint, bit for bit, call after call, since
the array keeps the previous call's contents (including a larger call's
differently laid-out data), and it must allocate nothing once warmed up.
Collected last so that a failure here never hides the other tests."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _forward(n, n_steps, every):
    wl = W.adjoint(n=n, n_steps=n_steps)
    m = gf.gf_medium_create(**wl.medium)
    k0, _ = O.onshell(O.medium(**wl.medium), wl.x0, wl.d)
    rays = gf.Rays.from_numpy(wl.x0, k0)
    n_ckpt = -(-n_steps // every)
    ck = torch.empty((n_ckpt, 6, n), dtype=torch.float64, device="cuda")
    gf.gf_trace_rk4(m, rays, 1.0, wl.dt, n_steps, 0.0, every, ck)
    return wl, m, rays, ck


def _lambda(wl, rays, rng, with_k):
    xstar = torch.from_numpy(np.ascontiguousarray((wl.x0 + rng.normal(0, 0.02, wl.x0.shape)).T)).cuda()
    lam = torch.zeros_like(rays.y)
    lam[:3] = 2 * (rays.y[:3] - xstar)
    if with_k:
        lam[3:] = torch.from_numpy(rng.normal(0, 1, (3, rays.n))).cuda()
    return lam


def _both(m, wl, n_steps, every, ck, rays, lam):
    """(gf_trace_adjoint, gf_trace_adjoint_static) results on the same inputs."""
    n = rays.n
    ref_t = torch.empty(64, dtype=torch.float64, device="cuda")
    ref_y = torch.empty_like(lam)
    gf.gf_trace_adjoint(m, n, 1.0, wl.dt, n_steps, every, ck, rays.steps, lam, ref_t, ref_y)
    got_t = torch.full_like(ref_t, float("nan"))
    got_y = torch.full_like(ref_y, float("nan"))
    gf.gf_trace_adjoint_static(m, n, 1.0, wl.dt, n_steps, every, ck, rays.steps, lam, got_t, got_y)
    torch.cuda.synchronize()
    return (ref_t, ref_y), (got_t, got_y)


def test_static_scratch_adjoint_matches_allocating_entry_point():
    n, n_steps, every = 300, 700, 64
    wl, m, rays, ck = _forward(n, n_steps, every)
    assert gf.gf_adjoint_scratch_bytes(m, n, every) <= 64 << 20
    rng = np.random.default_rng(1)
    # warm-up call with no rays: loads the library's module on this device, zeroes dL/dtheta
    out = torch.full((64,), 7.0, dtype=torch.float64, device="cuda")
    empty = torch.empty((6, 0), dtype=torch.float64, device="cuda")
    gf.gf_trace_adjoint_static(m, 0, 1.0, wl.dt, n_steps, every, ck, rays.steps, empty, out)
    torch.cuda.synchronize()
    assert (out == 0).all()
    for call in range(2):                       # two calls in a row, different losses
        lam = _lambda(wl, rays, rng, with_k=call == 1)
        (ref_t, ref_y), (got_t, got_y) = _both(m, wl, n_steps, every, ck, rays, lam)
        assert torch.equal(got_t, ref_t) and torch.equal(got_y, ref_y), call
    # the static call itself allocates nothing, in the library or in torch
    lam = _lambda(wl, rays, rng, with_k=True)
    got_t = torch.empty(64, dtype=torch.float64, device="cuda")
    got_y = torch.empty_like(lam)
    torch.cuda.synchronize()
    before = (gf.gf_bench_live_allocations(), torch.cuda.memory_allocated())
    gf.gf_trace_adjoint_static(m, n, 1.0, wl.dt, n_steps, every, ck, rays.steps, lam, got_t, got_y)
    torch.cuda.synchronize()
    assert (gf.gf_bench_live_allocations(), torch.cuda.memory_allocated()) == before


def test_static_scratch_after_a_larger_call():
    """A larger call with another checkpoint interval leaves its own data in the
    array; the smaller call that follows must not read any of it."""
    wl_big, m_big, rays_big, ck_big = _forward(2400, 200, 16)
    assert gf.gf_adjoint_scratch_bytes(m_big, 2400, 16) <= 64 << 20
    rng = np.random.default_rng(2)
    lam_big = _lambda(wl_big, rays_big, rng, with_k=True)
    (rt, ry), (gt, gy) = _both(m_big, wl_big, 200, 16, ck_big, rays_big, lam_big)
    assert torch.equal(gt, rt) and torch.equal(gy, ry)
    wl, m, rays, ck = _forward(300, 700, 64)
    lam = _lambda(wl, rays, rng, with_k=False)
    (rt, ry), (gt, gy) = _both(m, wl, 700, 64, ck, rays, lam)
    assert torch.equal(gt, rt) and torch.equal(gy, ry)


def test_static_scratch_rejects_oversized_calls():
    n, n_steps, every = 4000, 64, 64
    wl, m, rays, ck = _forward(n, n_steps, every)
    lam = torch.zeros_like(rays.y)
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    assert gf.gf_adjoint_scratch_bytes(m, n, every) > 64 << 20
    with pytest.raises(gf.GfError, match="fixed array holds"):
        gf.gf_trace_adjoint_static(m, n, 1.0, wl.dt, n_steps, every, ck, rays.steps, lam, out)
