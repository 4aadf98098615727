"""The library's table-driven base-2 exponential (every Gaussian-blob term of
the FP64 evaluator uses it) against exact references (Python's decimal and
fractions modules, so the tests need no third-party package) and CUDA's exp2."""
from __future__ import annotations

import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest
import torch

import paper_2508_15967_gb300 as gf

pytestmark = pytest.mark.gpu


def _exp2_exact(a: float) -> Decimal:
    getcontext().prec = 50
    return (Decimal(a) * Decimal(2).ln()).exp()


def _ulp_err(x: np.ndarray, a: np.ndarray) -> np.ndarray:
    """|x - 2^a| in ulps of the exact value."""
    out = np.empty(len(a))
    for i, (v, ai) in enumerate(zip(x, a)):
        ex = _exp2_exact(float(ai))
        out[i] = float(abs(Decimal(float(v)) - ex) / Decimal(math.ulp(float(ex))))
    return out


def test_exp_error_bound_against_correct_rounding():
    rng = np.random.default_rng(0)
    blob = np.concatenate([-rng.uniform(0, 1, 3000), -rng.uniform(0, 64, 3000),
                           -np.arange(0, 400) / 64.0, -(2 * np.arange(1, 300) + 1) / 4096.0,
                           [0.0, -0.0, -1e-300, -5e-324, -2.0 ** -12, -58.5]])
    wide = -rng.uniform(64, 1020.99, 2000)
    a = np.concatenate([blob, wide])
    lib, cuda = (t.cpu().numpy() for t in gf.gf_bench_exp(torch.tensor(a, device="cuda")))
    e_lib = _ulp_err(lib, a)
    nb = len(blob)
    # documented bound: table and final rounding 0.5 ulp each plus ~0.03 ulp
    # from the float-pair reduction and polynomial: < 1.05 ulp over the range
    assert e_lib[:nb].max() < 1.05, (e_lib[:nb].max(), a[np.argmax(e_lib[:nb])])
    assert e_lib[nb:].max() < 1.05, (e_lib[nb:].max(), a[nb + np.argmax(e_lib[nb:])])
    assert e_lib.mean() < 0.4
    assert (np.abs(lib - cuda) <= 3.0 * np.spacing(np.abs(cuda))).all()


def test_exp_integer_and_fma_forms_return_the_same_bits():
    """The form without FP64 operations (FP64-bound kernels) and the form with
    the table product as an FP64 FMA (the adjoint's recomputation) must round
    T (1 + P) identically: dense sweeps of the blob range, table-index and
    binade boundaries, values near multiples of 2^-11, and the wide range."""
    rng = np.random.default_rng(11)
    j = np.arange(-2048 * 64, 1)
    a = np.concatenate([-rng.uniform(0, 64, 400_000), -rng.uniform(64, 1020.99, 100_000),
                        j / 2048.0, j / 2048.0 + 2.0 ** -40, j / 2048.0 - 2.0 ** -40,
                        (j[:-1] + 0.5) / 2048.0, -np.abs(rng.normal(0, 1e-6, 20_000)),
                        [0.0, -0.0, -1e-300, -5e-324, -2.0 ** -12, -58.5, -1021.0 + 1e-9]])
    a = a[a <= 0]
    t = torch.tensor(a, device="cuda")
    lib, _ = gf.gf_bench_exp(t)
    fp = gf.gf_bench_exp_fp(t)
    same = torch.eq(lib.view(torch.int64), fp.view(torch.int64))
    assert bool(same.all()), a[~same.cpu().numpy()][:8]


def test_exp_flush_and_special_values():
    a = torch.tensor([-1021.0, -1021.5, -1075.0, -1e4, -float("inf"), 0.0, -0.0], device="cuda",
                     dtype=torch.float64)
    lib, _ = gf.gf_bench_exp(a)
    lib = lib.cpu().numpy()
    assert (lib[:5] == 0).all()                  # documented flush: a <= -1021
    assert lib[5] == 1.0 and lib[6] == 1.0
    # above the flush threshold the power-of-two scaling stays exact down to the smallest normals
    a = torch.tensor([-1020.999, -1020.5, -1000.0, -995.25], device="cuda", dtype=torch.float64)
    lib, cuda = gf.gf_bench_exp(a)
    lib = lib.cpu().numpy()
    assert (lib >= 2.0 ** -1022).all()
    assert (_ulp_err(lib, a.cpu().numpy()) < 1.05).all()


def test_reciprocal_and_truncation_helpers():
    """The FP64 evaluator's 1/n^2 (FP32 seed + one cubic Newton step) is within
    one ulp of the exact reciprocal (exact rationals), and its double -> float
    truncation of positions keeps the sign and errs by less than 2^-23."""
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.uniform(1e-3, 10, 4000), 10.0 ** rng.uniform(-40, 40, 4000),
                        [2.0 ** -120, 2.0 ** 120 * (1 - 2 ** -52), 2.0 ** 120, 2.0 ** -121, 1.0, 2.25, 1e-300]])
    r, _ = (t.cpu().numpy() for t in gf.gf_bench_recip(torch.tensor(v, device="cuda")))
    for ri, xi in zip(r, v):
        exact = 1 / Fraction(float(xi))
        assert abs(Fraction(float(ri)) - exact) <= Fraction(math.ulp(float(exact))), (xi, ri)
    x = np.concatenate([rng.choice([-1.0, 1.0], 4000) * 10.0 ** rng.uniform(-30, 30, 4000),
                        [0.0, -0.0, 1.5, -2.75, 3.5e38, -1e300]])
    _, f = (t.cpu().numpy() for t in gf.gf_bench_recip(torch.tensor(x, device="cuda")))
    f = f.astype(np.float64)
    body = np.abs(x) >= 2.0 ** -126
    body &= np.abs(x) < 2.0 ** 128
    assert (np.abs(f[body]) <= np.abs(x[body])).all() and (np.sign(f[body]) == np.sign(x[body])).all()
    assert (np.abs(f[body] - x[body]) / np.abs(x[body])).max() < 2.0 ** -23
    assert np.isinf(f[-2]) and np.isinf(f[-1]) and f[-1] < 0 and f[-6] == 0.0
