"""GPU batched adaptive DOPRI5 (persistent work-stealing and one launch per
medium) against the FP64 oracle, through the C ABI.

An embedded error estimate is a ~tol-sized difference of O(1) stage values,
so its relative rounding is ~1e-16 / tol ~ 1e-7 at tol = 1e-9; any two
implementations choose step sizes that differ at ~1e-8, their step sequences
drift apart, and each solution carries its own global error (the oracle's at
tol = 1e-9 on these media: median 1e-7, max 1.4e-6 against tol = 1e-13).  A
1e-9 endpoint gate is therefore not attainable by any second implementation;
the gate is that the GPU solution is as accurate as the oracle's:
  per-ray error against the oracle at rtol = atol = 1e-13, at the same time,
  has median, 99th percentile and maximum within 2x those of the oracle's own
  tol = 1e-9 solution (+1e-9).
Exiting rays (no event location) are compared at each ray's own stopping time.
Both schedules and every launch shape return bit-identical buffers.
"""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import workloads as W
from tests._parity import rel_err

pytestmark = pytest.mark.gpu


def _setup(n_media=48, scale=1.0 / 64, nb=8):
    wl = W.batched(n_media=n_media, n_blobs=nb, scale_counts=scale)
    blobs, off = wl.extra["blobs"], wl.extra["offsets"]
    om = [O.medium(kind="luneburg", blobs=blobs[j]) for j in range(n_media)]
    k0 = np.empty_like(wl.x0)
    for j in range(n_media):
        lo, hi = off[j], off[j + 1]
        if hi > lo:
            k0[lo:hi], st = O.onshell(om[j], wl.x0[lo:hi], wl.d[lo:hi])
            assert (st == 0).all()
    media = [gf.gf_medium_create("luneburg", blobs=blobs[j]) for j in range(n_media)]
    batch = gf.gf_batch_create(media, off)
    return wl, om, media, batch, k0


def _ctl(wl, **kw):
    e = wl.extra
    args = dict(rtol=e["rtol"], atol=e["atol"], h0=e["h0"], t_max=e["t_max"], radius=wl.radius,
                max_steps=e["max_steps"])
    args.update(kw)
    return args


def _gpu(batch, x0, k0, ctl, sched=gf.GF_SCHED_PERSISTENT, tune=None, status=None):
    rays = gf.Rays.from_numpy(x0, k0)
    if status is not None:
        rays.status.copy_(torch.as_tensor(status, dtype=torch.int32))
    rej = torch.zeros(rays.n, dtype=torch.int32, device="cuda")
    gf.gf_trace_dopri5(batch, rays, rej, 1.0, gf.step_ctl(**ctl), sched, tune)
    torch.cuda.synchronize()
    return rays, rej


def _host(rays, rej):
    return dict(y=rays.state(), t=rays.t.cpu().numpy(), status=rays.status.cpu().numpy(),
                steps=rays.steps.cpu().numpy(), rej=rej.cpu().numpy(),
                dres=rays.d_res.cpu().numpy(), dmax=rays.d_max.cpu().numpy())


def _oracle(om, off, x0, k0, ctl, status=None):
    r = O.make_rays(x0, k0, status=status)
    O.trace_dopri5(om, off, r, 1.0, **ctl)
    return r


TIGHT = dict(rtol=1e-13, atol=1e-13)


def _as_accurate(e_g, e_o):
    for q in (0.5, 0.99, 1.0):
        a, b = np.quantile(e_g, q), np.quantile(e_o, q)
        assert a <= 2 * b + 1e-9, (q, a, b)


def _compare_fixed_time(g, o, om, off, x0, k0, ctl, t_end):
    assert (g["status"] == gf.GF_RAY_DONE).all() and (o.status == gf.GF_RAY_DONE).all()
    assert (g["t"] == t_end).all()
    ref = _oracle(om, off, x0, k0, dict(ctl, **TIGHT))
    _as_accurate(rel_err(g["y"], ref.y), rel_err(o.y, ref.y))
    # max |D| along an adaptive trace measures that trace's own integration
    # error: same magnitude on both sides, not the same value
    _as_accurate(g["dmax"], o.dmax)


def _err_at_own_time(y, t, rows, om, off, x0, k0, ctl):
    med = np.searchsorted(off, rows, side="right") - 1
    e = np.empty(len(rows))
    for i, (r, j) in enumerate(zip(rows, med)):
        one = O.make_rays(x0[r:r + 1], k0[r:r + 1])
        O.trace_dopri5([om[j]], [0, 1], one, 1.0, **dict(ctl, radius=0.0, t_max=float(t[i]), **TIGHT))
        e[i] = rel_err(y[i:i + 1], one.y)[0]
    return e


def _compare_exit(g, om, off, x0, k0, ctl, o=None, rows=None):
    """EXITED rays: GPU and oracle states each against a tight re-trace to their own stopping time."""
    rows = np.arange(len(g["t"])) if rows is None else rows
    assert (g["status"] == gf.GF_RAY_EXITED).all()
    assert (np.linalg.norm(g["y"][:, :3], axis=1) > ctl["radius"]).all()
    if o is None:
        o = O.make_rays(x0[rows], k0[rows])
        med = np.searchsorted(off, rows, side="right") - 1
        for i, j in enumerate(med):
            one = O.make_rays(x0[rows[i]:rows[i] + 1], k0[rows[i]:rows[i] + 1])
            O.trace_dopri5([om[j]], [0, 1], one, 1.0, **ctl)
            for name in ("y", "t", "status", "steps", "dres", "dmax", "rejects"):
                getattr(o, name)[i] = getattr(one, name)[0]
    assert (o.status == gf.GF_RAY_EXITED).all()
    assert np.abs(g["steps"] - o.steps).max() <= 15
    e_g = _err_at_own_time(g["y"], g["t"], rows, om, off, x0, k0, ctl)
    e_o = _err_at_own_time(o.y, o.t, rows, om, off, x0, k0, ctl)
    _as_accurate(e_g, e_o)
    return e_g


def test_persistent_matches_oracle():
    wl, om, media, batch, k0 = _setup()
    ctl = _ctl(wl)
    rays, rej = _gpu(batch, wl.x0, k0, ctl)
    g = _host(rays, rej)
    o = _oracle(om, wl.extra["offsets"], wl.x0, k0, ctl)
    _compare_exit(g, om, wl.extra["offsets"], wl.x0, k0, ctl, o)


def test_fixed_end_time_parity():
    """Every ray integrated to t = 2.5 (through the lens surface, before the
    exit), the tight equal-time gate."""
    wl, om, media, batch, k0 = _setup()
    ctl = _ctl(wl, t_max=2.5, radius=0.0)
    g = _host(*_gpu(batch, wl.x0, k0, ctl))
    o = _oracle(om, wl.extra["offsets"], wl.x0, k0, ctl)
    _compare_fixed_time(g, o, om, wl.extra["offsets"], wl.x0, k0, ctl, 2.5)


def test_schedules_and_launch_shapes_are_bitwise_identical():
    wl, om, media, batch, k0 = _setup(n_media=40, scale=1.0 / 32)
    ctl = _ctl(wl)
    ref = _host(*_gpu(batch, wl.x0, k0, ctl, gf.GF_SCHED_PER_MEDIUM))
    for tune in [None, (64, 1, 1, 1), (256, 2, 16, 7), (128, 2, 4, 256), (128, 1, 64, 32)]:
        g = _host(*_gpu(batch, wl.x0, k0, ctl, gf.GF_SCHED_PERSISTENT, tune))
        for k in ref:
            assert np.array_equal(g[k], ref[k]), (tune, k)


def test_graph_replay_and_inactive_rays():
    wl, om, media, batch, k0 = _setup(n_media=20)
    ctl = _ctl(wl)
    status = np.zeros(wl.n, np.int32)
    status[::7] = gf.GF_RAY_CUTOFF                    # pre-stopped rays stay untouched
    a = _host(*_gpu(batch, wl.x0, k0, ctl, status=status))
    b = _host(*_gpu(batch, wl.x0, k0, ctl, status=status))  # same shapes: graph replay path
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["y"][::7], np.concatenate([wl.x0, k0], 1)[::7])
    assert (a["steps"][::7] == 0).all() and (a["status"][::7] == gf.GF_RAY_CUTOFF).all()
    live = status == 0
    sub = {k: v[live] for k, v in a.items()}
    _compare_exit(sub, om, wl.extra["offsets"], wl.x0, k0, ctl, rows=np.where(live)[0])


def test_done_and_budget_statuses():
    wl, om, media, batch, k0 = _setup(n_media=12)
    ctl = _ctl(wl, t_max=0.75, radius=0.0)
    g = _host(*_gpu(batch, wl.x0, k0, ctl))
    o = _oracle(om, wl.extra["offsets"], wl.x0, k0, ctl)
    _compare_fixed_time(g, o, om, wl.extra["offsets"], wl.x0, k0, ctl, 0.75)
    ctl = _ctl(wl, max_steps=3)
    g = _host(*_gpu(batch, wl.x0, k0, ctl))
    o = _oracle(om, wl.extra["offsets"], wl.x0, k0, ctl)
    assert (g["status"] == gf.GF_RAY_MAX_STEPS).all() and (g["steps"] == 3).all()
    assert np.array_equal(o.status, g["status"]) and np.array_equal(o.rejects, g["rej"])
    assert rel_err(g["y"], o.y).max() <= 1e-9          # three steps from h0: sequences still agree
    # an unattainable tolerance drives the step below h_min
    ctl = _ctl(wl, rtol=1e-20, atol=1e-20)
    g = _host(*_gpu(batch, wl.x0, k0, ctl))
    o = _oracle(om, wl.extra["offsets"], wl.x0, k0, ctl)
    assert (g["status"] == gf.GF_RAY_STEP_UNDERFLOW).all()
    assert np.array_equal(g["status"], o.status)


def test_empty_media_and_zero_rays():
    blobs = W.batched(n_media=3).extra["blobs"]
    media = [gf.gf_medium_create("luneburg", blobs=blobs[j]) for j in range(3)]
    off = np.array([0, 0, 5, 5])
    batch = gf.gf_batch_create(media, off)
    x0, d = W.plane_disk_rays(np.random.default_rng(0), 5, 0.5)
    k0 = np.empty_like(x0)
    k0[:], _ = O.onshell(O.medium(kind="luneburg", blobs=blobs[1]), x0, d)
    rays, rej = _gpu(batch, x0, k0, dict(radius=1.5))
    assert (rays.status.cpu().numpy() == gf.GF_RAY_EXITED).all()
    with pytest.raises(gf.GfError, match="offsets"):
        gf.gf_trace_dopri5(batch, gf.Rays.empty(3), None, 1.0, gf.step_ctl())


def test_autotune_returns_a_valid_shape_and_caches_it(tmp_path):
    wl, om, media, batch, k0 = _setup(n_media=64, scale=1.0 / 16)
    rays = gf.Rays.from_numpy(wl.x0, k0)
    before = rays.state().copy()
    path = str(tmp_path / "tune.txt")
    t = gf.gf_dopri5_autotune(batch, rays, 1.0, gf.step_ctl(**_ctl(wl)), path)
    assert t.block in (64, 128, 256) and t.rays_per_thread in (1, 2) and t.compaction >= 1 and t.chunk >= 1
    assert np.array_equal(rays.state(), before)               # tuner works on scratch copies
    assert os.path.exists(path) and open(path).read().count("\t") == 1
    batch2 = gf.gf_batch_create(media, wl.extra["offsets"])
    t2 = gf.gf_dopri5_autotune(batch2, rays, 1.0, gf.step_ctl(**_ctl(wl)), path)
    assert t2.as_tuple() == t.as_tuple()
    g = _host(*_gpu(batch2, wl.x0, k0, _ctl(wl)))             # tuned shape used by default
    ref = _host(*_gpu(batch2, wl.x0, k0, _ctl(wl), gf.GF_SCHED_PER_MEDIUM))
    for k in ref:
        assert np.array_equal(g[k], ref[k])


def test_f64x_mode_parity_and_schedule_independence():
    """GF_F64X (double-float blob sums): as accurate as the oracle at a fixed
    end time and at the exits, bit-identical across both schedules and several
    launch shapes; switching back to GF_F64 gives a never-switched batch's
    results; GF_F32 is refused."""
    wl, om, media, batch, k0 = _setup()
    off = wl.extra["offsets"]
    gf.gf_batch_set_precision(batch, gf.GF_F64X)
    ctl = _ctl(wl, t_max=2.5, radius=0.0)
    g = _host(*_gpu(batch, wl.x0, k0, ctl))
    o = _oracle(om, off, wl.x0, k0, ctl)
    _compare_fixed_time(g, o, om, off, wl.x0, k0, ctl, 2.5)
    ctl = _ctl(wl)
    ref = _host(*_gpu(batch, wl.x0, k0, ctl, gf.GF_SCHED_PER_MEDIUM))
    for tune in [None, (64, 1, 1, 1), (256, 2, 16, 7)]:
        g = _host(*_gpu(batch, wl.x0, k0, ctl, gf.GF_SCHED_PERSISTENT, tune))
        for k in ref:
            assert np.array_equal(g[k], ref[k]), (tune, k)
    _compare_exit(ref, om, off, wl.x0, k0, ctl, _oracle(om, off, wl.x0, k0, ctl))
    gf.gf_batch_set_precision(batch, gf.GF_F64)
    fresh = gf.gf_batch_create(media, off)
    a, b = _host(*_gpu(batch, wl.x0, k0, ctl)), _host(*_gpu(fresh, wl.x0, k0, ctl))
    for k in a:
        assert np.array_equal(a[k], b[k])
    with pytest.raises(gf.GfError, match="GF_F64"):
        gf.gf_batch_set_precision(batch, gf.GF_F32)


def test_full_batched_workload_sampled():
    """All 4096 media (~12.2M rays, log-uniform counts) in one persistent graph
    launch; 48 seeded sampled rays re-traced by the oracle."""
    wl = W.batched()
    blobs, off = wl.extra["blobs"], wl.extra["offsets"]
    media = [gf.gf_medium_create("luneburg", blobs=blobs[j]) for j in range(len(off) - 1)]
    batch = gf.gf_batch_create(media, off)
    rays = gf.Rays.from_numpy(wl.x0, None)
    # on-shell k per medium: directions are +x; the library sets k on shell
    dirs = torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda()
    for j in range(len(media)):
        lo, hi = int(off[j]), int(off[j + 1])
        sub = gf.Rays(rays.y[:, lo:hi], rays.t[lo:hi], rays.status[lo:hi], rays.steps[lo:hi],
                      rays.d_res[lo:hi], rays.d_max[lo:hi])
        if hi > lo:
            s = sub.struct()
            s.ld = rays.y.stride(0)
            gf._check("gf_rays_onshell", gf.lib().gf_rays_onshell(
                media[j].handle, gf.GF_F64, gf.C.byref(s), dirs[:, lo:hi].data_ptr(), 1.0,
                torch.cuda.current_stream().cuda_stream))
    k_gpu = rays.state()[:, 3:].copy()
    rej = torch.zeros(rays.n, dtype=torch.int32, device="cuda")
    gf.gf_trace_dopri5(batch, rays, rej, 1.0, gf.step_ctl(**_ctl(wl)))
    torch.cuda.synchronize()
    g = _host(rays, rej)
    assert (g["status"] == gf.GF_RAY_EXITED).all()
    idx = np.sort(np.random.default_rng(5).choice(wl.n, 48, replace=False))
    om = {}
    med = np.searchsorted(off, idx, side="right") - 1
    for j in med:
        om[j] = O.medium(kind="luneburg", blobs=blobs[j])
    sub = {k: v[idx] for k, v in g.items()}
    _compare_exit(sub, om, off, wl.x0, k_gpu, _ctl(wl), rows=idx)
