"""The library's table-driven exponential (all Gaussian-blob terms use it)
against correctly rounded references (mpmath, 50 digits) and CUDA's exp."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import paper_2508_15967_gb300 as gf

pytestmark = pytest.mark.gpu


def _ulp_err(x: np.ndarray, ref: np.ndarray) -> np.ndarray:
    return np.abs(x - ref) / np.spacing(np.abs(ref))


def test_exp_error_bound_against_correct_rounding():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(0)
    a = np.concatenate([-rng.uniform(0, 1, 3000), -rng.uniform(0, 60, 3000),
                        -rng.uniform(0, 707.9, 2000), -np.log(2) / 64 * np.arange(0, 400),
                        -np.log(2) / 128 * (2 * np.arange(1, 200) + 1), [0.0, -0.0, -1e-300, -5e-324]])
    lib, cuda = (t.cpu().numpy() for t in gf.gf_bench_exp(torch.tensor(a, device="cuda")))
    ref = np.array([float(mpmath.exp(mpmath.mpf(v))) for v in a])
    # error against the exact value is < 1.16 ulp (table rounding 0.5, final
    # fma 0.5, polynomial truncation < 0.16), i.e. at most 2 ulp from the rounded value
    e_lib = _ulp_err(lib, ref)
    assert e_lib.max() <= 2.0, (e_lib.max(), a[np.argmax(e_lib)])
    assert e_lib.mean() < 0.4
    assert _ulp_err(lib, cuda).max() <= 3.0


def test_exp_flush_and_special_values():
    a = torch.tensor([-708.0, -708.3, -745.0, -1e4, -float("inf"), 0.0], device="cuda", dtype=torch.float64)
    lib, cuda = gf.gf_bench_exp(a)
    lib = lib.cpu().numpy()
    assert (lib[:5] == 0).all()                  # documented flush below 2^-1021
    assert lib[5] == 1.0
    # above the flush threshold the scaling stays exact down to the smallest normals
    a = torch.tensor([-707.9, -700.0, -690.0], device="cuda", dtype=torch.float64)
    lib, cuda = gf.gf_bench_exp(a)
    np.testing.assert_allclose(lib.cpu().numpy(), cuda.cpu().numpy(), rtol=4e-16)


def test_reciprocal_and_truncation_helpers():
    """The FP64 evaluator's 1/n^2 (FP32 seed + one cubic Newton step) is within
    one ulp of the exact reciprocal (mpmath), and its double -> float
    truncation of positions keeps the sign and errs by less than 2^-23."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.uniform(1e-3, 10, 4000), 10.0 ** rng.uniform(-40, 40, 4000),
                        [2.0 ** -120, 2.0 ** 120 * (1 - 2 ** -52), 2.0 ** 120, 2.0 ** -121, 1.0, 2.25, 1e-300]])
    r, _ = (t.cpu().numpy() for t in gf.gf_bench_recip(torch.tensor(v, device="cuda")))
    exact = np.array([float(1 / mpmath.mpf(x)) for x in v])
    err = np.array([abs(mpmath.mpf(a) - 1 / mpmath.mpf(x)) for a, x in zip(r, v)], dtype=float)
    assert (err / np.spacing(np.abs(exact))).max() <= 1.0
    x = np.concatenate([rng.choice([-1.0, 1.0], 4000) * 10.0 ** rng.uniform(-30, 30, 4000),
                        [0.0, -0.0, 1.5, -2.75, 3.5e38, -1e300]])
    _, f = (t.cpu().numpy() for t in gf.gf_bench_recip(torch.tensor(x, device="cuda")))
    f = f.astype(np.float64)
    body = np.abs(x) >= 2.0 ** -126
    body &= np.abs(x) < 2.0 ** 128
    assert (np.abs(f[body]) <= np.abs(x[body])).all() and (np.sign(f[body]) == np.sign(x[body])).all()
    assert (np.abs(f[body] - x[body]) / np.abs(x[body])).max() < 2.0 ** -23
    assert np.isinf(f[-2]) and np.isinf(f[-1]) and f[-1] < 0 and f[-6] == 0.0
