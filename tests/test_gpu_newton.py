"""GPU Newton initialisation of k_x (the paper's Sec. 4 procedure) against the
oracle's Newton solver and the closed-form roots."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["grin", "luneburg", "aniso"])
def test_newton_kx_matches_oracle(name):
    rng = np.random.default_rng(2)
    n = 1000
    if name == "grin":
        spec = W.grin(n=1).medium
        x = rng.uniform(-0.3, 0.3, (n, 3))
    elif name == "luneburg":
        spec = W.adjoint(n=1).medium
        x = rng.uniform(-1.2, 1.2, (n, 3))
    else:
        spec = W.aniso(n=1, g=32).medium
        x = rng.uniform(-1, 1, (n, 3))
    k = np.column_stack([np.where(rng.random(n) < 0.5, -2.0, 2.0), rng.uniform(-0.8, 0.8, (n, 2))])
    k_o, st_o, _ = O.newton_kx(O.medium(**spec), x, k, 1.0)
    m = gf.gf_medium_create(**spec)
    rays = gf.Rays.from_numpy(x, k)
    gf.gf_rays_newton_kx(m, rays, 1.0)
    torch.cuda.synchronize()
    k_g = rays.state()[:, 3:]
    st_g = rays.status.cpu().numpy()
    assert np.array_equal(st_g, st_o)
    ok = st_o == 0
    assert ok.mean() > 0.5 and (~ok).any()       # both branches of the outcome occur
    np.testing.assert_allclose(k_g[ok, 0], k_o[ok, 0], rtol=2e-15, atol=1e-14)   # |k| ~ 1 scale
    np.testing.assert_array_equal(k_g[:, 1:], k[:, 1:])
    D = O.eval_dispersion(O.medium(**spec), x[ok], k_g[ok])[:, 0]
    assert np.abs(D).max() <= 8e-15
