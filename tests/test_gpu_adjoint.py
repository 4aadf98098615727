"""GPU discrete adjoint of the RK4 trace (dL/dtheta for the blob amplitudes)
against the oracle's forward tangent-linear sensitivities (<= 1e-9, a
different derivation of the same derivative) and against central finite
differences of the GPU forward loss (h = 1e-6, <= 1e-5, every parameter) on
rays that keep clear of the Luneburg kink (min over stage points of
||x|^2 - 1| > 1e-5, computed by the oracle).  Loss: L = sum_rays |x_N - x*_N|^2.

Errors are measured per component: |g_j - ref_j| / max(|ref_j|, 1e-3 max_i |ref_i|),
so that a small component is held to the tolerance relative to its own size
(down to a floor of 1e-3 of the largest component, below which a component
is numerically zero against the others)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(n, n_steps, n_blobs=64):
    wl = W.adjoint(n=n, n_steps=n_steps, n_blobs=n_blobs)
    om = O.medium(**wl.medium)
    k0, st = O.onshell(om, wl.x0, wl.d)
    assert (st == 0).all()
    blobs_star = wl.medium["blobs"].copy()
    blobs_star[:, 0] = wl.extra["theta_star"]
    rs = O.make_rays(wl.x0, k0)
    O.trace_rk4(O.medium(kind="luneburg", blobs=blobs_star), rs, 1.0, wl.dt, n_steps)
    xstar = rs.y[:, :3].copy()
    y0 = np.concatenate([wl.x0, k0], 1)
    return wl, om, y0, xstar


def _gpu_grad(wl, y0, xstar, every=64, theta=None):
    m = gf.gf_medium_create(**wl.medium)
    th = torch.tensor(wl.extra["theta"] if theta is None else theta, device="cuda", requires_grad=True)
    y0_t = torch.from_numpy(np.ascontiguousarray(y0.T)).cuda()
    yN = gf.trace_rk4_autograd(m, th, y0_t, 1.0, wl.dt, wl.n_steps, every)
    xs = torch.from_numpy(np.ascontiguousarray(xstar.T)).cuda()
    loss = ((yN[:3] - xs) ** 2).sum()
    loss.backward()
    return th.grad.cpu().numpy(), loss.item(), yN.detach()


def _oracle_grad(om, y0, xstar, wl):
    r = O.make_rays(y0[:, :3], y0[:, 3:])
    S = O.tangent_rk4(om, r, 1.0, wl.dt, wl.n_steps)
    return O.loss_grad(r.y, xstar, S)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _rel_per_component(a, ref, floor=1e-3):
    """max_j |a_j - ref_j| / max(|ref_j|, floor * max_i |ref_i|)."""
    ref = np.asarray(ref)
    return (np.abs(np.asarray(a) - ref) / np.maximum(np.abs(ref), floor * np.abs(ref).max())).max()


def test_adjoint_matches_oracle_tangent_linear():
    """256 rays (4 blocks), 1000 steps, 64 blobs: adjoint vs tangent-linear."""
    wl, om, y0, xstar = _case(256, 1000)
    g_gpu, _, _ = _gpu_grad(wl, y0, xstar)
    g_or = _oracle_grad(om, y0, xstar, wl)
    assert _rel_per_component(g_gpu, g_or) <= 1e-9, _rel_per_component(g_gpu, g_or)


def test_adjoint_full_length_trace():
    """The adjoint workload's full 4000 steps (63 checkpoint segments, the last
    one partial) on a ragged 100-ray subset."""
    wl, om, y0, xstar = _case(100, 4000)
    g_gpu, _, _ = _gpu_grad(wl, y0, xstar)
    g_or = _oracle_grad(om, y0, xstar, wl)
    assert _rel_per_component(g_gpu, g_or) <= 1e-9, _rel_per_component(g_gpu, g_or)


def test_adjoint_matches_central_differences():
    """Central differences (h = 1e-6) of the GPU forward loss for all 64
    amplitudes, 128 traces run concurrently on 16 streams, per component."""
    wl, om, y0, xstar = _case(192, 4000)
    r = O.make_rays(y0[:, :3], y0[:, 3:])
    kink = O.trace_rk4_kink(om, r, 1.0, wl.dt, wl.n_steps)
    keep = kink > 1e-5
    assert keep.mean() > 0.9
    y0k, xk = y0[keep], xstar[keep]
    g_gpu, _, _ = _gpu_grad(wl, y0k, xk)
    y0_t = torch.from_numpy(np.ascontiguousarray(y0k.T)).cuda()
    xs = torch.from_numpy(np.ascontiguousarray(xk.T)).cuda()
    th = wl.extra["theta"]
    h = 1e-6
    streams = [torch.cuda.Stream() for _ in range(16)]
    traces = []
    torch.cuda.synchronize()
    for j in range(len(th)):
        for sign in (1.0, -1.0):
            blobs = wl.medium["blobs"].copy()
            blobs[j, 0] = th[j] + sign * h
            m = gf.gf_medium_create("luneburg", blobs=blobs)
            rays = gf.Rays.empty(y0k.shape[0], diagnostics=False)
            rays.y.copy_(y0_t)
            st = streams[len(traces) % len(streams)]
            st.wait_stream(torch.cuda.current_stream())
            gf.gf_trace_rk4(m, rays, 1.0, wl.dt, wl.n_steps, stream=st)
            traces.append((m, rays))
    torch.cuda.synchronize()
    loss = [((rays.y[:3] - xs) ** 2).sum().item() for _, rays in traces]
    fd = np.array([(loss[2 * j] - loss[2 * j + 1]) / (2 * h) for j in range(len(th))])
    assert _rel_per_component(g_gpu, fd) <= 1e-5, _rel_per_component(g_gpu, fd)


def test_autograd_dy0_and_direct_call_agree():
    """theta.grad from the autograd Function equals a direct gf_trace_adjoint
    call bit for bit; dL/dy0 matches differences of the launch state."""
    wl, om, y0, xstar = _case(70, 600)
    m = gf.gf_medium_create(**wl.medium)
    th = torch.tensor(wl.extra["theta"], device="cuda", requires_grad=True)
    y0_t = torch.from_numpy(np.ascontiguousarray(y0.T)).cuda().requires_grad_(True)
    xs = torch.from_numpy(np.ascontiguousarray(xstar.T)).cuda()
    yN = gf.trace_rk4_autograd(m, th, y0_t, 1.0, wl.dt, wl.n_steps, 64)
    ((yN[:3] - xs) ** 2).sum().backward()
    # direct call
    rays = gf.Rays.empty(70)
    rays.y.copy_(y0_t.detach())
    ck = torch.empty((10, 6, 70), dtype=torch.float64, device="cuda")
    gf.gf_medium_set_amplitudes(m, th.detach())
    gf.gf_trace_rk4(m, rays, 1.0, wl.dt, 600, 0.0, 64, ck)
    lam = torch.zeros_like(rays.y)
    lam[:3] = 2 * (rays.y[:3] - xs)
    dth = torch.empty(64, dtype=torch.float64, device="cuda")
    gf.gf_trace_adjoint(m, 70, 1.0, wl.dt, 600, 64, ck, rays.steps, lam, dth)
    assert torch.equal(dth, th.grad)
    g0 = y0_t.grad.cpu().numpy()

    def loss_y(yy):
        r = gf.Rays.empty(70)
        r.y.copy_(torch.from_numpy(np.ascontiguousarray(yy.T)).cuda())
        gf.gf_trace_rk4(m, r, 1.0, wl.dt, 600)
        return ((r.y[:3] - xs) ** 2).sum().item()

    for ray, c in [(0, 1), (5, 3), (33, 2), (69, 4)]:
        h = 1e-7
        yp, ym = y0.copy(), y0.copy()
        yp[ray, c] += h
        ym[ray, c] -= h
        fd = (loss_y(yp) - loss_y(ym)) / (2 * h)
        assert abs(fd - g0[c, ray]) <= 1e-6 * max(1.0, abs(fd)), (ray, c, fd, g0[c, ray])


def test_checkpoint_interval_does_not_change_the_gradient():
    """The recomputation reproduces the forward trace's bits and the sweep
    runs in the same order whatever the segment length: the gradient is the
    same bit for bit for every checkpoint interval."""
    wl, om, y0, xstar = _case(64, 300)
    ref, _, _ = _gpu_grad(wl, y0, xstar, every=64)
    for every in (1, 7, 300, 1000):
        g, _, _ = _gpu_grad(wl, y0, xstar, every=every)
        assert np.array_equal(g, ref), (every, _rel_per_component(g, ref))


def test_recomputation_reproduces_the_forward_checkpoints():
    """Work counters of the backward: every recomputed segment ends on the next
    checkpoint of the forward trace in every bit (counters[3] = 0), including
    rays that stop early; the sweep evaluates blob terms (counters[2] > 0)."""
    wl, om, y0, xstar = _case(300, 700)
    m = gf.gf_medium_create(**wl.medium)
    rays = gf.Rays.from_numpy(y0[:, :3], y0[:, 3:])
    st = np.zeros(300, np.int32)
    st[::17] = gf.GF_RAY_CUTOFF                        # some rays never move
    rays.status.copy_(torch.from_numpy(st))
    every = 64
    ck = torch.full((-(-700 // every), 6, 300), float("nan"), dtype=torch.float64, device="cuda")
    gf.gf_trace_rk4(m, rays, 1.0, wl.dt, 700, 1.2, every, ck)   # radius 1.2: rays stop on leaving
    steps = rays.steps.cpu().numpy()
    assert (steps[::17] == 0).all() and 0 < steps.min(initial=700, where=st == 0) < 700
    lam = torch.zeros_like(rays.y)
    lam[:3] = 2 * (rays.y[:3] - torch.from_numpy(np.ascontiguousarray(xstar.T)).cuda())
    counters = torch.zeros(4, dtype=torch.int64, device="cuda")
    dth = torch.empty(64, dtype=torch.float64, device="cuda")
    gf.gf_bench_set_counters(counters)
    try:
        gf.gf_trace_adjoint(m, 300, 1.0, wl.dt, 700, every, ck, rays.steps, lam, dth)
        torch.cuda.synchronize()
    finally:
        gf.gf_bench_set_counters(None)
    c = counters.cpu().numpy()
    assert c[0] == 4 * steps.sum() and c[1] > 0 and c[2] > 0
    assert c[3] == 0, f"{c[3]} recomputed segment-end components differ from the checkpoints"


def test_adjoint_edge_cases():
    wl, om, y0, xstar = _case(10, 50)
    m = gf.gf_medium_create(**wl.medium)
    dth = torch.full((64,), 7.0, dtype=torch.float64, device="cuda")
    empty = torch.empty((6, 0), dtype=torch.float64, device="cuda")
    ck = torch.empty((1, 6, 1), dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    gf.gf_trace_adjoint(m, 0, 1.0, wl.dt, 50, 64, ck, st, empty, dth)        # no rays: zero gradient
    torch.cuda.synchronize()
    assert (dth == 0).all()
    # rays that did not move (steps_done = 0) pass lambda through, add nothing
    lam = torch.randn((6, 10), dtype=torch.float64, device="cuda")
    dy0 = torch.empty_like(lam)
    ck = torch.zeros((1, 6, 10), dtype=torch.float64, device="cuda")
    zeros = torch.zeros(10, dtype=torch.int32, device="cuda")
    gf.gf_trace_adjoint(m, 10, 1.0, wl.dt, 50, 64, ck, zeros, lam, dth, dy0)
    torch.cuda.synchronize()
    assert (dth == 0).all() and torch.equal(dy0, lam)
    with pytest.raises(gf.GfError, match="scratch"):
        gf.gf_trace_adjoint(m, 10, 1.0, wl.dt, 50, 64, ck, zeros, lam, dth, dy0,
                            scratch=torch.empty(16, dtype=torch.uint8, device="cuda"))
    with pytest.raises(gf.GfError, match="blob"):
        gf.gf_trace_adjoint(gf.gf_medium_create("luneburg"), 10, 1.0, wl.dt, 50, 64, ck, zeros, lam, dth)


def test_full_size_adjoint_sampled_rays():
    """The adjoint workload at full size (65,536 rays, 4000 steps, 64 blobs,
    checkpoints every 64) in the benchmark's launch shape, with lambda masked to
    48 sampled rays so the oracle's tangent-linear gradient of the same loss
    can be computed; plus additivity of the full gradient over ray halves."""
    wl = W.adjoint()
    m = gf.gf_medium_create(**wl.medium)
    rays = gf.Rays.empty(wl.n)
    rays.y[:3].copy_(torch.from_numpy(np.ascontiguousarray(wl.x0.T)).cuda())
    gf.gf_rays_onshell(m, rays, torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda(), 1.0)
    y0 = rays.y.clone()
    ck = torch.empty((63, 6, wl.n), dtype=torch.float64, device="cuda")
    gf.gf_trace_rk4(m, rays, 1.0, wl.dt, wl.n_steps, 0.0, 64, ck)
    rng = np.random.default_rng(3)
    xstar = torch.from_numpy(np.ascontiguousarray((wl.x0 + rng.normal(0, 0.01, wl.x0.shape)).T)).cuda()
    idx = np.sort(rng.choice(wl.n, 48, replace=False))
    lam = torch.zeros_like(rays.y)
    lam[:3, idx] = 2 * (rays.y[:3, idx] - xstar[:, idx])
    dth = torch.empty(64, dtype=torch.float64, device="cuda")
    gf.gf_trace_adjoint(m, wl.n, 1.0, wl.dt, wl.n_steps, 64, ck, rays.steps, lam, dth)
    y0s = y0[:, idx].T.cpu().numpy()
    r = O.make_rays(y0s[:, :3], y0s[:, 3:])
    S = O.tangent_rk4(O.medium(**wl.medium), r, 1.0, wl.dt, wl.n_steps)
    g_or = O.loss_grad(r.y, xstar[:, idx].T.cpu().numpy(), S)
    assert _rel_per_component(dth.cpu().numpy(), g_or) <= 1e-9
    # additivity over disjoint ray sets
    lam = torch.zeros_like(rays.y)
    lam[:3] = 2 * (rays.y[:3] - xstar)
    full = torch.empty_like(dth)
    gf.gf_trace_adjoint(m, wl.n, 1.0, wl.dt, wl.n_steps, 64, ck, rays.steps, lam, full)
    parts = torch.zeros_like(dth)
    for half in (slice(0, wl.n // 2), slice(wl.n // 2, wl.n)):
        l2 = torch.zeros_like(lam)
        l2[:, half] = lam[:, half]
        gf.gf_trace_adjoint(m, wl.n, 1.0, wl.dt, wl.n_steps, 64, ck, rays.steps, l2, dth)
        parts += dth
    assert _rel(parts.cpu().numpy(), full.cpu().numpy()) <= 1e-12
