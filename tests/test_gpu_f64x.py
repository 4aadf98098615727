"""The GF_F64X mode (FP64 state and integrator, Gaussian-blob sums in
double-float on the FP32 pipes) against the FP64 oracle at the FP64 gates:
endpoints <= 1e-9 relative, |D| drift <= 1e-8, bit-exact statuses."""
from __future__ import annotations

from decimal import Decimal, getcontext

import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import workloads as W
from tests._parity import GpuResult, assert_parity, oracle_rk4, rel_err

pytestmark = pytest.mark.gpu


def test_double_float_exp_accuracy():
    """The double-float 2^a against exact decimal values of 2^(hi + lo) of
    the float pair the input is split into."""
    getcontext().prec = 50
    ln2 = Decimal(2).ln()
    rng = np.random.default_rng(4)
    a = np.concatenate([-rng.uniform(0, 1, 2000), -rng.uniform(0, 4, 1000), -rng.uniform(0, 58.5, 3000),
                        -(2 * np.arange(1, 300) + 1) / 4096.0, [0.0, -1e-30, -2.0 ** -12, -58.5, -62.9]])
    got = gf.gf_bench_exp_df(torch.tensor(a, device="cuda")).cpu().numpy()
    hi = a.astype(np.float32).astype(np.float64)
    lo = (a - hi).astype(np.float32).astype(np.float64)
    ref = np.array([float(((Decimal(h) + Decimal(l)) * ln2).exp()) for h, l in zip(hi, lo)])
    # a.lo enters through one float product, so the relative error scales with
    # max(1, |a|); about 2^-47 at worst, ~2^-50 typically
    rel = np.abs(got - ref) / ref / np.maximum(1.0, np.abs(a))
    assert rel.max() <= 1.2e-14, (rel.max(), a[np.argmax(rel)])
    assert np.median(rel) <= 1e-15


def _gpu_x(spec, x0, k0, dt, n_steps):
    m = gf.gf_medium_create(**spec)
    rays = gf.Rays.from_numpy(x0, k0)
    gf.gf_trace_rk4(m, rays, 1.0, dt, n_steps, precision=gf.GF_F64X)
    return GpuResult(rays)


def test_f64x_grin_parity():
    wl = W.grin(n=1000)
    k0, _ = O.onshell(O.medium(**wl.medium), wl.x0, wl.d)
    g = _gpu_x(wl.medium, wl.x0, k0, wl.dt, wl.n_steps)
    o, _ = oracle_rk4(wl.medium, wl.x0, k0, 1.0, wl.dt, wl.n_steps)
    worst = assert_parity(g, o, 1e-9)
    assert g.dmax.max() <= 1e-8
    print("f64x grin worst rel err", worst)


def test_f64x_luneburg_64_blobs_parity():
    wl = W.adjoint(n=300, n_steps=4000)
    k0, _ = O.onshell(O.medium(**wl.medium), wl.x0, wl.d)
    g = _gpu_x(wl.medium, wl.x0, k0, wl.dt, wl.n_steps)
    o, _ = oracle_rk4(wl.medium, wl.x0, k0, 1.0, wl.dt, wl.n_steps)
    assert_parity(g, o, 1e-9, diag_atol=1e-11)


def test_f64x_full_size_sampled():
    wl = W.grin()
    m = gf.gf_medium_create(**wl.medium)
    rays = gf.Rays.from_numpy(wl.x0, None)
    gf.gf_rays_onshell(m, rays, torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda(), 1.0)
    k_gpu = rays.state()[:, 3:].copy()
    gf.gf_trace_rk4(m, rays, 1.0, wl.dt, wl.n_steps, precision=gf.GF_F64X)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(77).choice(wl.n, 128, replace=False))
    o, _ = oracle_rk4(wl.medium, wl.x0[idx], k_gpu[idx], 1.0, wl.dt, wl.n_steps)
    assert rel_err(rays.state()[idx], o.y).max() <= 1e-9
    assert rays.d_max.max().item() <= 1e-8 and (rays.status == 0).all()
