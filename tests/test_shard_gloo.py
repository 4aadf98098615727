"""Multi-process (world_size 2, gloo, CPU) checks of the data-parallel path,
with the rank logic the benchmark uses (ray_share, media_share): shards cover
every ray once; the sum of per-shard adjoint gradients equals the
single-process gradient (oracle tangent-linear sensitivities on each shard),
for one ray set split across the ranks (strong scaling) and for every rank's
own ray set (weak scaling); a batch of media sharded by ray counts traces,
rank by rank, exactly what one process traces; the job time is the slowest
rank's."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2508_15967_gb300.shard import (allreduce_gradient, max_over_ranks, media_share, ray_share,
                                          shard_bounds, shard_media)


def test_shard_bounds_partition():
    for n in (0, 1, 7, 64, 1000, 12557776):
        for world in (1, 2, 3, 4, 8):
            spans = [shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_bounds(10, 2, 2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_ray_and_media_share():
    from paper_2508_15967_gb300 import workloads as W
    for world in (1, 2, 3, 8):
        weak = [ray_share("weak", 100, r, world) for r in range(world)]
        assert weak == [(r, 0, 100) for r in range(world)]          # own seeds, whole sets
        strong = [ray_share("strong", 100, r, world) for r in range(world)]
        assert all(sd == 0 for sd, _, _ in strong)                   # one shared set ...
        assert [(lo, hi) for _, lo, hi in strong] == [shard_bounds(100, r, world) for r in range(world)]
    off = W.batched(n_media=64).extra["offsets"]
    assert [media_share("weak", off, r, 4) for r in range(4)] == [(r, 0, 64) for r in range(4)]
    assert [media_share("strong", off, r, 4)[1:] for r in range(4)] == [shard_media(off, r, 4) for r in range(4)]
    with pytest.raises(ValueError):
        ray_share("diagonal", 10, 0, 1)
    # weak-scaling seeds give independent inputs of the same shape
    a, b = W.adjoint(n=16, shard=0), W.adjoint(n=16, shard=1)
    assert a.x0.shape == b.x0.shape and not np.allclose(a.x0, b.x0)
    assert np.array_equal(a.medium["blobs"], b.medium["blobs"])   # the parameters are shared
    c, d = W.batched(n_media=8, shard=0), W.batched(n_media=8, shard=1)
    assert not np.array_equal(c.extra["blobs"], d.extra["blobs"])


def _grad_of_rays(idx, shard=0):
    import oracle as O
    from paper_2508_15967_gb300 import workloads as W
    wl = W.adjoint(n=24, n_steps=150, n_blobs=6, shard=shard)
    m = O.medium(**wl.medium)
    k0, _ = O.onshell(m, wl.x0, wl.d)
    xstar = wl.x0 + 0.05
    r = O.make_rays(wl.x0[idx], k0[idx])
    S = O.tangent_rk4(m, r, 1.0, wl.dt, wl.n_steps)
    return O.loss_grad(r.y, xstar[idx], S)


def _worker(rank, world, port, out, scaling="strong"):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    seed_shard, lo, hi = ray_share(scaling, 24, rank, world)
    g = torch.tensor(_grad_of_rays(np.arange(lo, hi), seed_shard))
    allreduce_gradient(g)
    t = max_over_ranks(0.5 + rank)
    out[rank] = (g.numpy(), t)
    torch.distributed.destroy_process_group()


def test_data_parallel_adjoint_gradient_gloo_world2():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    full = _grad_of_rays(np.arange(24))
    for rank in range(world):
        g, t = res[rank]
        np.testing.assert_allclose(g, full, rtol=1e-12, atol=1e-15)
        assert t == 1.5


def test_weak_scaling_adjoint_gradient_gloo_world2():
    """Every rank its own rays (seed shard = rank): the all-reduced gradient is
    the gradient of the sum of both ranks' losses."""
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out, "weak"), nprocs=world, join=True)
        res = dict(out)
    total = _grad_of_rays(np.arange(24), 0) + _grad_of_rays(np.arange(24), 1)
    for rank in range(world):
        np.testing.assert_allclose(res[rank][0], total, rtol=1e-12, atol=1e-15)


def test_shard_media_partition_and_balance():
    from paper_2508_15967_gb300 import workloads as W
    off = W.batched(n_media=4096).extra["offsets"]
    counts = np.diff(off)
    for world in (1, 2, 3, 4, 8):
        spans = [shard_media(off, r, world) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == len(counts)
        assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
        rays = np.array([off[hi] - off[lo] for lo, hi in spans])
        assert rays.sum() == off[-1]
        assert np.abs(rays - off[-1] / world).max() <= counts.max()
    assert [shard_media([0, 0, 0], r, 2) for r in range(2)] == [(0, 0), (0, 2)]   # no rays: still a partition
    with pytest.raises(ValueError):
        shard_media([0, 5, 3], 0, 2)


def _batch_case():
    from paper_2508_15967_gb300 import workloads as W
    import oracle as O
    wl = W.batched(n_media=10, scale_counts=1.0 / 512)
    blobs, off = wl.extra["blobs"], wl.extra["offsets"]
    om = [O.medium(kind="luneburg", blobs=blobs[j]) for j in range(len(off) - 1)]
    k0 = np.empty_like(wl.x0)
    for j in range(len(om)):
        if off[j + 1] > off[j]:
            k0[off[j]:off[j + 1]], _ = O.onshell(om[j], wl.x0[off[j]:off[j + 1]], wl.d[off[j]:off[j + 1]])
    ctl = dict(rtol=1e-9, atol=1e-9, h0=1e-3, t_max=10.0, radius=1.5, max_steps=100000)
    return wl, om, off, k0, ctl


def _media_worker(rank, world, port, out):
    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    wl, om, off, k0, ctl = _batch_case()
    _, m_lo, m_hi = media_share("strong", off, rank, world)
    lo, hi = int(off[m_lo]), int(off[m_hi])
    r = O.make_rays(wl.x0[lo:hi], k0[lo:hi])
    O.trace_dopri5(om[m_lo:m_hi], np.asarray(off[m_lo:m_hi + 1]) - lo, r, 1.0, **ctl)
    out[rank] = (lo, hi, r.y.copy(), r.steps.copy(), r.status.copy())
    torch.distributed.destroy_process_group()


def test_batched_media_shards_gloo_world2():
    import oracle as O
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_media_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    wl, om, off, k0, ctl = _batch_case()
    r = O.make_rays(wl.x0, k0)
    O.trace_dopri5(om, off, r, 1.0, **ctl)
    spans = sorted(res[k][:2] for k in range(world))
    assert spans[0][0] == 0 and spans[-1][1] == wl.n and spans[0][1] == spans[1][0]
    for k in range(world):
        lo, hi, y, steps, status = res[k]
        assert np.array_equal(y, r.y[lo:hi]) and np.array_equal(steps, r.steps[lo:hi])
        assert np.array_equal(status, r.status[lo:hi])
