"""Generated media: dispersion relations written as expression graphs,
differentiated and simplified symbolically, emitted as CUDA and compiled at
run time (gf_jit_medium_create) -- traced on the GPU and compared with the
FP64 oracle (<= 1e-9) and with the hand-written kernels."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import symbolic as S
from paper_2508_15967_gb300 import workloads as W
from tests._parity import GpuResult, assert_parity, oracle_rk4, rel_err

pytestmark = pytest.mark.gpu


def _trace(m, x0, k0, dt, n_steps):
    rays = gf.Rays.from_numpy(x0, k0)
    gf.gf_trace_rk4(m, rays, 1.0, dt, n_steps)
    return GpuResult(rays)


def test_generated_grin_medium_matches_oracle_and_builtin():
    wl = W.grin(n=513, n_steps=4000)
    D = S.isotropic(S.grin_n2(1.5, 2.0) + S.gaussian_blobs(wl.medium["blobs"]))
    m = gf.gf_jit_medium_create(S.medium_source(D))
    k0, _ = O.onshell(O.medium(**wl.medium), wl.x0, wl.d)
    g = _trace(m, wl.x0, k0, wl.dt, wl.n_steps)
    o, _ = oracle_rk4(wl.medium, wl.x0, k0, 1.0, wl.dt, wl.n_steps)
    assert_parity(g, o, 1e-9)
    b = _trace(gf.gf_medium_create(**wl.medium), wl.x0, k0, wl.dt, wl.n_steps)
    assert rel_err(g.y, b.y).max() <= 1e-11


def test_generated_luneburg_with_blobs():
    wl = W.adjoint(n=300, n_steps=2500)
    D = S.isotropic(S.luneburg_n2() + S.gaussian_blobs(wl.medium["blobs"]))
    m = gf.gf_jit_medium_create(S.medium_source(D))
    k0, _ = O.onshell(O.medium(**wl.medium), wl.x0, wl.d)
    g = _trace(m, wl.x0, k0, wl.dt, wl.n_steps)
    o, _ = oracle_rk4(wl.medium, wl.x0, k0, 1.0, wl.dt, wl.n_steps)
    assert_parity(g, o, 1e-9, diag_atol=1e-11)


def test_generated_cold_plasma_matches_handwritten():
    """The cold plasma written only as D (no hand-derived gradient) traces like
    the hand-written cold-plasma kernel and the oracle."""
    spec = dict(kind="cold", species=((0.3, -0.5), (0.02, 0.05)), profile=(1.0, 0.1, 1.0, 0.05))
    D = S.cold_plasma(spec["species"], spec["profile"])
    m = gf.gf_jit_medium_create(S.medium_source(D))
    rng = np.random.default_rng(5)
    n = 400
    x0 = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), np.zeros(n)])
    kyz = np.column_stack([rng.uniform(-0.25, 0.25, n), rng.uniform(-0.2, 0.2, n)])
    k0, st, _ = O.newton_kx(O.medium(**spec), x0, np.column_stack([np.full(n, 1.2), kyz]))
    assert (st == 0).all()
    g = _trace(m, x0, k0, 0.01, 2000)
    o, _ = oracle_rk4(spec, x0, k0, 1.0, 0.01, 2000)
    assert_parity(g, o, 1e-9, diag_atol=1e-11)
    h = _trace(gf.gf_medium_create(**spec), x0, k0, 0.01, 2000)
    assert rel_err(g.y, h.y).max() <= 1e-11


def test_generated_medium_restrictions_and_errors():
    D = S.isotropic(S.luneburg_n2())
    m = gf.gf_jit_medium_create(S.medium_source(D))
    rays = gf.Rays.from_numpy(np.zeros((4, 3)), np.ones((4, 3)), torch.float32)
    with pytest.raises(gf.GfError, match="GF_F64"):
        gf.gf_trace_rk4(m, rays, 1.0, 0.01, 10)
    with pytest.raises(gf.GfError, match="compile"):
        gf.gf_jit_medium_create("this is not CUDA")
