"""Failure handling of the C ABI, tested without a device fault: an injected
failure (gf_fault_inject) makes the n-th CUDA call the library checks report
an error although it succeeded, for every n along a whole sequence of calls.
Each time the entry point must return the error (never crash), release every
device allocation it took (gf_bench_live_allocations back to the baseline once
the objects are destroyed), and leave the library usable: the same sequence
then runs to the same, bit-identical results."""
from __future__ import annotations

import gc

import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAX_POINTS = 300   # upper bound on the checked calls of one sequence


def _rk4_and_adjoint():
    """Medium with blobs, on-shell k, FP64 and GF_F64X traces with
    checkpoints, the adjoint, new amplitudes."""
    wl = W.adjoint(n=96, n_steps=130, n_blobs=8)
    every = 64
    m = gf.gf_medium_create(**wl.medium)
    try:
        rays = gf.Rays.from_numpy(wl.x0, None)
        gf.gf_rays_onshell(m, rays, torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda(), 1.0)
        r64x = rays.clone()
        gf.gf_trace_rk4(m, r64x, 1.0, wl.dt, wl.n_steps, precision=gf.GF_F64X)
        ck = torch.empty((-(-wl.n_steps // every), 6, wl.n), dtype=torch.float64, device="cuda")
        gf.gf_trace_rk4(m, rays, 1.0, wl.dt, wl.n_steps, 0.0, every, ck)
        lam = torch.zeros_like(rays.y)
        lam[:3] = 2 * rays.y[:3]
        dtheta = torch.empty(wl.medium["blobs"].shape[0], dtype=torch.float64, device="cuda")
        gf.gf_trace_adjoint(m, wl.n, 1.0, wl.dt, wl.n_steps, every, ck, rays.steps, lam, dtheta)
        gf.gf_medium_set_amplitudes(m, 0.5 * torch.from_numpy(wl.extra["theta"]).cuda())
        r2 = gf.Rays.from_numpy(wl.x0, rays.state()[:, 3:])
        gf.gf_trace_rk4(m, r2, 1.0, wl.dt, 20)
        torch.cuda.synchronize()
        return [rays.state(), r64x.state(), dtheta.cpu().numpy(), r2.state()]
    finally:
        m.close()


def _spline_f32():
    """Spline medium (a small 8^3 grid) traced in FP64 and FP32."""
    wl = W.aniso(n=64, n_steps=40, g=8)
    m = gf.gf_medium_create(**wl.medium)
    try:
        out = []
        for dtype in (torch.float64, torch.float32):
            rays = gf.Rays.from_numpy(wl.x0, None, dtype=dtype)
            gf.gf_rays_onshell(m, rays, torch.from_numpy(np.ascontiguousarray(wl.d.T)).to("cuda", dtype), 1.0)
            gf.gf_trace_rk4(m, rays, 1.0, wl.dt, wl.n_steps)
            torch.cuda.synchronize()
            out.append(rays.state())
        return out
    finally:
        m.close()


def _batch():
    """Batch of media, persistent and per-medium DOPRI5 (graph capture and
    replay), then GF_F64X."""
    wl = W.batched(n_media=5, n_blobs=4, scale_counts=1.0 / 256)
    blobs, off = wl.extra["blobs"], wl.extra["offsets"]
    k0 = np.empty_like(wl.x0)
    for j in range(len(off) - 1):
        if off[j + 1] > off[j]:
            k0[off[j]:off[j + 1]], _ = O.onshell(O.medium(kind="luneburg", blobs=blobs[j]),
                                                 wl.x0[off[j]:off[j + 1]], wl.d[off[j]:off[j + 1]])
    media = []
    batch = None
    try:
        for j in range(len(off) - 1):
            media.append(gf.gf_medium_create("luneburg", blobs=blobs[j]))
        batch = gf.gf_batch_create(media, off)
        ctl = gf.step_ctl(t_max=3.0)
        out = []
        for sched in (gf.GF_SCHED_PERSISTENT, gf.GF_SCHED_PER_MEDIUM, gf.GF_SCHED_PERSISTENT):
            rays = gf.Rays.from_numpy(wl.x0, k0)
            rej = torch.zeros(rays.n, dtype=torch.int32, device="cuda")
            gf.gf_trace_dopri5(batch, rays, rej, 1.0, ctl, sched)
            torch.cuda.synchronize()
            out += [rays.state(), rej.cpu().numpy()]
        gf.gf_batch_set_precision(batch, gf.GF_F64X)
        rays = gf.Rays.from_numpy(wl.x0, k0)
        gf.gf_trace_dopri5(batch, rays, None, 1.0, ctl, gf.GF_SCHED_PERSISTENT)
        torch.cuda.synchronize()
        out.append(rays.state())
        return out
    finally:
        if batch is not None:
            batch.close()
        for m in media:
            m.close()


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("sequence", [_rk4_and_adjoint, _spline_f32, _batch],
                         ids=["rk4_adjoint", "spline_f32", "batch_dopri5"])
def test_injected_failures_release_everything_and_leave_the_library_usable(sequence):
    gf.gf_fault_inject(0)
    gc.collect()                     # objects of earlier tests are gone before the baseline
    base = gf.gf_bench_live_allocations()
    ref = sequence()
    assert gf.gf_bench_live_allocations() == base
    fired = 0
    for n in range(1, MAX_POINTS + 1):
        gf.gf_fault_inject(n)
        try:
            got = sequence()
        except gf.GfError as e:
            assert "injected fault" in str(e), str(e)
            fired += 1
        else:
            _same(got, ref)          # n lies beyond the sequence's checked calls
            break
        finally:
            gf.gf_fault_inject(0)
        torch.cuda.synchronize()
        gc.collect()
        assert gf.gf_bench_live_allocations() == base, (n, str(gf.gf_bench_live_allocations()))
        _same(sequence(), ref)       # the library (streams, caches) still works
    else:
        pytest.fail(f"sequence still failing after {MAX_POINTS} injection points")
    assert fired >= 5
    assert gf.gf_bench_live_allocations() == base
