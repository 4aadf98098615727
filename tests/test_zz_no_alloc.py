"""The allocation-free adjoint entry point (gf_trace_adjoint_static), for
callers that cannot allocate device memory once running (for example a
real-time control loop, where cudaMalloc/cudaFree may block or synchronise
the device, or a host code whose GPU memory is reserved up front by its own
pool).  Its scratch is a fixed 64 MiB array inside the library; it must give
the same gradient as gf_trace_adjoint, call after call, since the array keeps
the previous call's contents.  Collected last so that a failure here never
hides the other tests."""
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


def test_static_scratch_adjoint_matches_allocating_entry_point():
    n, n_steps, every = 300, 700, 64
    wl, m, rays, ck = _forward(n, n_steps, every)
    assert gf.gf_adjoint_scratch_bytes(m, n, every) <= 64 << 20
    rng = np.random.default_rng(1)
    for call in range(2):                       # two calls in a row, different losses
        xstar = torch.from_numpy(np.ascontiguousarray((wl.x0 + rng.normal(0, 0.02, wl.x0.shape)).T)).cuda()
        lam = torch.zeros_like(rays.y)
        lam[:3] = 2 * (rays.y[:3] - xstar)
        if call == 1:
            lam[3:] = torch.from_numpy(rng.normal(0, 1, (3, n))).cuda()
        ref_t = torch.empty(64, dtype=torch.float64, device="cuda")
        ref_y = torch.empty_like(lam)
        gf.gf_trace_adjoint(m, n, 1.0, wl.dt, n_steps, every, ck, rays.steps, lam, ref_t, ref_y)
        got_t = torch.full_like(ref_t, float("nan"))
        got_y = torch.full_like(ref_y, float("nan"))
        gf.gf_trace_adjoint_static(m, n, 1.0, wl.dt, n_steps, every, ck, rays.steps, lam, got_t, got_y)
        torch.cuda.synchronize()
        assert torch.isfinite(got_t).all() and torch.isfinite(got_y).all()
        rel_t = ((got_t - ref_t).abs().max() / ref_t.abs().max()).item()
        rel_y = ((got_y - ref_y).abs().max() / ref_y.abs().max()).item()
        assert rel_t <= 1e-12 and rel_y <= 1e-12, (call, rel_t, rel_y)


def test_static_scratch_rejects_oversized_calls():
    n, n_steps, every = 1000, 64, 64
    wl, m, rays, ck = _forward(n, n_steps, every)
    lam = torch.zeros_like(rays.y)
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    assert gf.gf_adjoint_scratch_bytes(m, n, every) > 64 << 20
    with pytest.raises(gf.GfError, match="fixed array holds"):
        gf.gf_trace_adjoint_static(m, n, 1.0, wl.dt, n_steps, every, ck, rays.steps, lam, out)
