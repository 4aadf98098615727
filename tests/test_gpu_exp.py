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


def _gauss_exact(u) -> Decimal:
    """2^-(u0^2 + u1^2 + u2^2) of the given doubles, the exponent exact."""
    getcontext().prec = 50
    q = sum(Fraction(float(c)) ** 2 for c in u)
    return (-(Decimal(q.numerator) / Decimal(q.denominator)) * Decimal(2).ln()).exp()


def _blob_points(rng, n):
    d = rng.normal(0, 1, (n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = [rng.uniform(-7.6, 7.6, (n, 3)),                                 # culled and live
           d * np.sqrt(rng.uniform(0, 58.5, (n, 1))),                      # live, any exponent
           d * np.sqrt(rng.integers(0, 58 * 2048, (n, 1)) / 2048.0),       # exponent on the k/2048 grid
           rng.normal(0, 1, (n, 3)) * 10.0 ** rng.uniform(-12, 0.5, (n, 3)),   # mixed magnitudes
           rng.uniform(-1e-3, 1e-3, (n, 3))]                               # near the centre
    return np.concatenate(pts)


def test_blob_gaussian_against_the_exact_gaussian():
    """The FP64 evaluator's blob Gaussian sums |u|^2 exactly in integer fixed
    point: within 1.05 ulp of 2^-|u|^2 for the given u (no rounding of the
    exponent), +0 exactly for the negligible terms (|u|^2 >= 58.5), and the
    same bits in its integer and FMA forms."""
    rng = np.random.default_rng(21)
    u = _blob_points(rng, 1200)
    u = np.concatenate([u, [[0.0, 0.0, 0.0], [-0.0, 5e-324, 0.0], [2.0 ** -30, 2.0 ** -40, 0.0],
                            [7.6, 0.0, 0.0], [1.0, 1.0, 1.0], [np.sqrt(58.5) * (1 - 1e-15), 0.0, 0.0]]])
    gi, gfp = (t.cpu().numpy() for t in gf.gf_bench_blob_gauss(torch.tensor(u.T.copy(), device="cuda")))
    assert (gi.view(np.int64) == gfp.view(np.int64)).all()
    q = np.array([float(sum(Fraction(float(c)) ** 2 for c in p)) for p in u])
    live = q < 58.5 - 1e-9
    dead = q >= 58.5 + 1e-9
    assert (gi[dead] == 0).all() and not np.signbit(gi[dead]).any()
    err = np.array([float(abs(Decimal(float(g)) - ex) / Decimal(math.ulp(float(ex))))
                    for g, ex in ((g, _gauss_exact(p)) for g, p in zip(gi[live], u[live]))])
    assert err.max() < 1.05, (err.max(), u[live][np.argmax(err)])
    assert err.mean() < 0.4
    assert gi[len(u) - 6] == 1.0 and gi[len(u) - 5] == 1.0


def test_blob_gaussian_forms_agree_and_special_values():
    rng = np.random.default_rng(22)
    u = _blob_points(rng, 200_000)
    t = torch.tensor(u.T.copy(), device="cuda")
    gi, gfp = gf.gf_bench_blob_gauss(t)
    assert torch.equal(gi.view(torch.int64), gfp.view(torch.int64))
    # against CUDA's exp2 of the FP64-rounded exponent: the only gap is that rounding
    q = (t * t).sum(0)
    ref = torch.exp2(-q)
    live = q < 58.0
    rel = ((gi - ref).abs() / ref)[live]
    assert float(rel.max()) < 64 * 2.0 ** -52
    # |u_i| >= 8 is negligible whatever the others; inf and NaN give NaN
    s = torch.tensor([[8.0, 0.0, 0.0], [-9.5, 0.0, 0.0], [1e300, 0.0, 0.0], [float("inf"), 0.0, 0.0],
                      [float("nan"), 0.0, 0.0], [0.0, -float("inf"), 1.0]], device="cuda", dtype=torch.float64)
    gs, _ = gf.gf_bench_blob_gauss(s.T.contiguous())
    gs = gs.cpu().numpy()
    assert (gs[:3] == 0).all() and np.isnan(gs[3:]).all()
