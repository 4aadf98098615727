"""Multi-process (world_size 2, gloo, CPU) checks of the data-parallel path:
shards cover every ray once; the sum of per-shard adjoint gradients equals the
single-process gradient (oracle tangent-linear sensitivities on each shard);
the job time is the slowest rank's."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2508_15967_gb300.shard import allreduce_gradient, max_over_ranks, shard_bounds


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


def _grad_of_rays(idx):
    import oracle as O
    from paper_2508_15967_gb300 import workloads as W
    wl = W.adjoint(n=24, n_steps=150, n_blobs=6)
    m = O.medium(**wl.medium)
    k0, _ = O.onshell(m, wl.x0, wl.d)
    xstar = wl.x0 + 0.05
    r = O.make_rays(wl.x0[idx], k0[idx])
    S = O.tangent_rk4(m, r, 1.0, wl.dt, wl.n_steps)
    return O.loss_grad(r.y, xstar[idx], S)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard_bounds(24, rank, world)
    g = torch.tensor(_grad_of_rays(np.arange(lo, hi)))
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
