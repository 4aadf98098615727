"""Pins of the FP64 CPU oracle against what the mathematics fixes (CPU only).

None of these compares the oracle with itself or retypes its formulas: the
checks are closed-form rays, central differences, conservation laws,
polynomial reproduction, convergence order, published tables, and brute-force
finite differences of whole traces.  The comment on each test names the
mistakes in the oracle that it would catch.
"""
from __future__ import annotations

import math
from fractions import Fraction
import os

import numpy as np
import pytest

import oracle as O
from paper_2508_15967_gb300 import workloads as W
from tests import _closed_forms as CF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _media():
    rng = np.random.default_rng(11)
    blobs = W.blob_table(rng, 5, 0.05)
    grid = W.aniso_grid(np.random.default_rng(12), g=16, n_modes=6)
    return {
        "homog": O.medium(kind="homog", n_h=1.37),
        "luneburg_in": O.medium(kind="luneburg"),
        "luneburg_out": O.medium(kind="luneburg"),
        "quadratic": O.medium(kind="quadratic", blobs=blobs),
        "grin_blobs": O.medium(kind="grin", n0=1.5, a=2.0, blobs=blobs),
        "spline": O.medium(kind="spline", grid=grid),
    }


def _points(name, n=12):
    rng = np.random.default_rng(hash(name) % 1000)
    if name == "luneburg_in":
        x = rng.uniform(-0.5, 0.5, (n, 3))
    elif name == "luneburg_out":
        x = rng.uniform(0.8, 1.5, (n, 3))
    elif name == "grin_blobs":
        x = rng.uniform(-0.3, 0.3, (n, 3))
    elif name == "quadratic":
        x = rng.uniform(-0.7, 0.7, (n, 3))
    else:
        x = rng.uniform(-0.9, 0.9, (n, 3))
    k = rng.uniform(-1.2, 1.2, (n, 3))
    return x, k


def _fd5(f, v, h):
    """4th-order central difference of f along each coordinate of v (rows)."""
    out = []
    for c in range(v.shape[1]):
        e = np.zeros_like(v)
        e[:, c] = h
        out.append((-f(v + 2 * e) + 8 * f(v + e) - 8 * f(v - e) + f(v - 2 * e)) / (12 * h))
    return np.stack(out, axis=1)


# ---------------------------------------------------------------- dispersion

@pytest.mark.parametrize("name", ["homog", "luneburg_in", "luneburg_out", "quadratic",
                                  "grin_blobs", "spline"])
def test_partials_match_central_differences(name):
    """D_x, D_k, D_w vs 5-point differences of D (catches a dropped term, wrong
    sign, wrong blob width power, transposed M index or wrong spline derivative
    weight)."""
    m = _media()[name]
    x, k = _points(name)
    w = 1.0
    ev = O.eval_dispersion(m, x, k, w)
    h = 1e-4
    Dx_fd = _fd5(lambda xx: O.eval_dispersion(m, xx, k, w)[:, 0], x, h)
    Dk_fd = _fd5(lambda kk: O.eval_dispersion(m, x, kk, w)[:, 0], k, h)
    Dw_fd = (-O.eval_dispersion(m, x, k, w + 2 * h)[:, 0] + 8 * O.eval_dispersion(m, x, k, w + h)[:, 0]
             - 8 * O.eval_dispersion(m, x, k, w - h)[:, 0] + O.eval_dispersion(m, x, k, w - 2 * h)[:, 0]) / (12 * h)
    scale = 1 + np.abs(ev[:, 1:8]).max()
    np.testing.assert_allclose(ev[:, 1:4], Dx_fd, atol=2e-8 * scale)
    np.testing.assert_allclose(ev[:, 4:7], Dk_fd, atol=2e-8 * scale)
    np.testing.assert_allclose(ev[:, 7], Dw_fd, atol=2e-8 * scale)


def test_dispersion_values_closed_form():
    """D itself at hand-picked points (catches the Luneburg branch, the GRIN
    axis choice and a wrong blob normalisation)."""
    w = 1.3
    x = np.array([[0.3, -0.2, 0.1], [1.2, 0.0, 0.0], [0.0, 0.1, -0.2]])
    k = np.array([[0.5, 0.25, -1.0], [1.0, 1.0, 0.0], [0.3, 0.0, 0.0]])
    kk = (k * k).sum(1)
    lun = O.eval_dispersion(O.medium(kind="luneburg"), x, k, w)[:, 0]
    n2 = np.where((x * x).sum(1) <= 1, 2 - (x * x).sum(1), 1.0)
    np.testing.assert_allclose(lun, kk - w * w * n2, rtol=0, atol=1e-15)
    grin = O.eval_dispersion(O.medium(kind="grin", n0=1.5, a=2.0), x, k, w)[:, 0]
    n2 = 2.25 * (1 - 4 * (x[:, 1] ** 2 + x[:, 2] ** 2))
    np.testing.assert_allclose(grin, kk - w * w * n2, rtol=0, atol=1e-14)
    blob = np.array([[0.7, 0.1, -0.1, 0.2, 0.15]])
    hb = O.eval_dispersion(O.medium(kind="homog", n_h=1.0, blobs=blob), x, k, w)[:, 0]
    r2 = ((x - blob[0, 1:4]) ** 2).sum(1)
    n2 = 1 + 0.7 * np.exp(-r2 / (2 * 0.15 ** 2))
    np.testing.assert_allclose(hb, kk - w * w * n2, rtol=0, atol=1e-14)


@pytest.mark.parametrize("kind", ["quadratic", "grin", "luneburg"])
def test_index_hessian_matches_differences(kind):
    """Hessian of n^2 used by the sensitivities vs differences of grad n^2."""
    blobs = W.blob_table(np.random.default_rng(3), 4, 0.05)
    m = O.medium(kind=kind, blobs=blobs)
    x = np.random.default_rng(4).uniform(-0.5, 0.5, (10, 3))
    out = O.index_hess(m, x)
    H_fd = _fd5(lambda xx: O.index_hess(m, xx)[:, 1:4], x, 1e-4)  # (n, 3[c], 3[i])
    H = out[:, 4:].reshape(-1, 3, 3)
    np.testing.assert_allclose(H, np.transpose(H_fd, (0, 2, 1)), atol=1e-7)
    np.testing.assert_allclose(H, np.transpose(H, (0, 2, 1)), atol=1e-14)


# ---------------------------------------------------------------- on-shell

@pytest.mark.parametrize("name", ["homog", "luneburg_in", "quadratic", "grin_blobs", "spline"])
def test_onshell_residual_below_paper_tolerance(name):
    """|D(x0, k0)| < 1e-15-ish: the paper initialises rays to |D| < 1e-15
    (Sec. 4); k0 must also be parallel to the given direction."""
    m = _media()[name]
    x, _ = _points(name, 50)
    d = W.sphere_directions(np.random.default_rng(5), 50)
    k0, st = O.onshell(m, x, d, 1.0)
    assert (st == O.ACTIVE).all()
    D = O.eval_dispersion(m, x, k0, 1.0)[:, 0]
    assert np.abs(D).max() < 4e-15
    cos = (k0 * d).sum(1) / np.linalg.norm(k0, axis=1)
    np.testing.assert_allclose(cos, 1.0, atol=1e-15)


def test_onshell_cutoff_where_no_real_root():
    """Outside r = 1/a the GRIN index is imaginary: cut-off status, k0 = 0."""
    m = O.medium(kind="grin", n0=1.5, a=2.0)
    x = np.array([[0.0, 0.6, 0.0], [0.0, 0.1, 0.0]])
    k0, st = O.onshell(m, x, np.array([[1.0, 0, 0], [1.0, 0, 0]]))
    assert st.tolist() == [O.CUTOFF, O.ACTIVE]
    assert (k0[0] == 0).all()


# ---------------------------------------------------------------- RK4 rays

def test_homogeneous_rays_are_exact_straight_lines():
    """RK4 is exact on a constant right-hand side: x = x0 + k t/(w n^2) to
    rounding, k unchanged bit for bit (catches wrong RK4 weights, a sign flip
    of -D_k/D_w, a t bookkeeping error)."""
    m = O.medium(kind="homog", n_h=1.7)
    rng = np.random.default_rng(1)
    x0 = rng.uniform(-1, 1, (20, 3))
    d = W.sphere_directions(rng, 20)
    k0, _ = O.onshell(m, x0, d, 1.3)
    r = O.make_rays(x0, k0)
    O.trace_rk4(m, r, 1.3, 1e-2, 500)
    x_ex, k_ex = CF.straight(x0, k0, 1.7, 5.0, 1.3)
    np.testing.assert_allclose(r.y[:, :3], x_ex, atol=1e-13)
    assert np.array_equal(r.y[:, 3:], k0)
    np.testing.assert_allclose(r.t, 5.0, rtol=0, atol=1e-14)
    assert (r.steps == 500).all() and (r.status == O.ACTIVE).all()
    # group speed 1/n on shell
    v = np.linalg.norm(r.y[:, :3] - x0, axis=1) / 5.0
    np.testing.assert_allclose(v, 1 / 1.7, rtol=1e-13)


def _grin_case():
    m = O.medium(kind="grin", n0=1.5, a=2.0)
    wl = W.grin(n=6, n_steps=0)
    k0, _ = O.onshell(m, wl.x0, wl.d)
    return m, wl.x0, k0


@pytest.mark.parametrize("T", [1.0, 3.0])
def test_grin_sinusoidal_closed_form_fourth_order(T):
    """Parabolic fibre without blobs: oracle vs the closed-form sinusoidal ray,
    error O(dt^4) with halving ratio ~16 (catches any RK4 stage coefficient
    error, which drops the order, and a wrong a^2 / n0^2 factor)."""
    m, x0, k0 = _grin_case()
    errs = []
    for n in (50, 100, 200):
        r = O.make_rays(x0, k0)
        O.trace_rk4(m, r, 1.0, T / n, n)
        e = 0.0
        for i in range(len(x0)):
            x_ex, k_ex = CF.grin(x0[i], k0[i], 1.5, 2.0, T)
            e = max(e, np.abs(r.y[i, :3] - x_ex).max(), np.abs(r.y[i, 3:] - k_ex).max())
        errs.append(e)
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(12 < q < 20 for q in ratios), (errs, ratios)
    assert errs[-1] < 1e-7


def test_grin_invariants():
    """k_x is exactly conserved (dn^2/dx = 0), L_x = y kz - z ky and D to O(dt^4)."""
    m, x0, k0 = _grin_case()
    r = O.make_rays(x0, k0)
    O.trace_rk4(m, r, 1.0, 5e-4, 4000)
    assert np.array_equal(r.y[:, 3], k0[:, 0])
    L0 = x0[:, 1] * k0[:, 2] - x0[:, 2] * k0[:, 1]
    L1 = r.y[:, 1] * r.y[:, 5] - r.y[:, 2] * r.y[:, 4]
    np.testing.assert_allclose(L1, L0, atol=1e-12)
    assert r.dmax.max() < 1e-12


def test_grin_blobs_conserve_dispersion():
    """The GRIN + 16 blob workload (dt = 5e-4, 10,000 steps): |D| drift <= 1e-8,
    the benchmark spec's bound, on a seeded subset of rays (catches a gradient that is
    not the gradient of the n^2 used in D)."""
    wl = W.grin(n=48)
    m = O.medium(**wl.medium)
    k0, _ = O.onshell(m, wl.x0, wl.d)
    r = O.make_rays(wl.x0, k0)
    O.trace_rk4(m, r, 1.0, wl.dt, wl.n_steps)
    assert (r.status == O.ACTIVE).all()
    assert r.dmax.max() < 1e-8
    assert np.abs(r.dres).max() < 1e-8


def test_quadratic_law_ellipse_fourth_order():
    """n^2 = 2 - |x|^2 everywhere: rays are centred ellipses (closed form),
    convergence order 4; angular momentum x cross k conserved to O(dt^4)."""
    rng = np.random.default_rng(9)
    m = O.medium(kind="quadratic")
    p = rng.uniform(-0.6, 0.6, (5, 3))
    u = W.sphere_directions(rng, 5)
    k0, _ = O.onshell(m, p, u)
    T = 2.0
    errs = []
    for n in (200, 400, 800):
        r = O.make_rays(p, k0)
        O.trace_rk4(m, r, 1.0, T / n, n)
        e = 0.0
        for i in range(5):
            x_ex, k_ex = CF.quadratic(p[i], k0[i], T)
            e = max(e, np.abs(r.y[i, :3] - x_ex).max(), np.abs(r.y[i, 3:] - k_ex).max())
        errs.append(e)
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(12 < q < 20 for q in ratios), (errs, ratios)
    r = O.make_rays(p, k0)
    O.trace_rk4(m, r, 1.0, 1e-3, 2000)
    L0 = np.cross(p, k0)
    L1 = np.cross(r.y[:, :3], r.y[:, 3:])
    np.testing.assert_allclose(L1, L0, atol=1e-12)


def test_luneburg_workload_matches_closed_form_and_focuses():
    """The Luneburg workload: at t = 2 (2000 steps of 1e-3) the rays agree with
    the closed form to the O(dt) error of crossing the |x| = 1 kink; traced to
    t = 1 + pi/2 every ray reaches the focus (1, 0, 0)."""
    wl = W.luneburg(n=64)
    m = O.medium(**wl.medium)
    k0, _ = O.onshell(m, wl.x0, wl.d)
    assert np.array_equal(k0, wl.d)
    r = O.make_rays(wl.x0, k0)
    O.trace_rk4(m, r, 1.0, wl.dt, wl.n_steps)
    for i in range(64):
        x_ex, k_ex = CF.luneburg_from_plane(wl.x0[i, 1], wl.x0[i, 2], 2.0)
        assert np.abs(r.y[i, :3] - x_ex).max() < 1e-3
        assert np.abs(r.y[i, 3:] - k_ex).max() < 1e-3
    n = 2571
    r = O.make_rays(wl.x0, k0)
    O.trace_rk4(m, r, 1.0, (1 + math.pi / 2) / n, n)
    dist = np.linalg.norm(r.y[:, :3] - np.array([1.0, 0, 0]), axis=1)
    assert dist.max() < 1e-3
    assert r.dmax.max() < 5e-3          # O(dt) jump of grad n^2 at the lens surface


def test_rk4_order_on_blobby_medium():
    """No closed form with blobs: Richardson ratio |y(h)-y(h/2)| / |y(h/2)-y(h/4)| ~ 16."""
    wl = W.grin(n=4)
    m = O.medium(**wl.medium)
    k0, _ = O.onshell(m, wl.x0, wl.d)
    ys = []
    for n in (400, 800, 1600):
        r = O.make_rays(wl.x0, k0)
        O.trace_rk4(m, r, 1.0, 4.0 / n, n)
        ys.append(r.y.copy())
    q = np.abs(ys[0] - ys[1]).max() / np.abs(ys[1] - ys[2]).max()
    assert 12 < q < 20, q


def test_exit_status_and_step_count():
    """Homogeneous rays with a termination sphere stop on the first step whose
    end point is outside it (closed form step index)."""
    m = O.medium(kind="homog", n_h=1.0)
    x0 = np.zeros((3, 3))
    d = np.array([[1.0, 0, 0], [0, 1.0, 0], [0.6, 0.8, 0]])
    k0, _ = O.onshell(m, x0, d)
    r = O.make_rays(x0, k0)
    O.trace_rk4(m, r, 1.0, 0.01, 1000, radius=0.505)
    assert (r.status == O.EXITED).all()
    assert (r.steps == 51).all(), r.steps          # first n with 0.01 n > 0.505
    np.testing.assert_allclose(np.linalg.norm(r.y[:, :3], axis=1), 0.51, atol=1e-14)


def test_cutoff_freezes_ray():
    """A GRIN ray launched steeply reaches n^2 <= 0 at r = 1/a: cut-off status,
    the state is the one before the failing step (still propagating there)."""
    m = O.medium(kind="grin", n0=1.5, a=2.0)
    x0 = np.array([[0.0, 0.45, 0.0]])
    d = np.array([[0.2, 1.0, 0.0]])
    k0, _ = O.onshell(m, x0, d)
    r = O.make_rays(x0, k0)
    O.trace_rk4(m, r, 1.0, 1e-2, 1000)
    assert r.status[0] == O.CUTOFF
    assert 0 < r.steps[0] < 1000
    ev = O.eval_dispersion(m, r.y[:, :3], r.y[:, 3:])
    assert ev[0, 8] > 0


def test_checkpoints_and_resume():
    """Checkpoint j holds the state before step j*every, and a trace split in
    two calls equals one call bit for bit in x and k."""
    wl = W.grin(n=5)
    m = O.medium(**wl.medium)
    k0, _ = O.onshell(m, wl.x0, wl.d)
    r = O.make_rays(wl.x0, k0)
    ck = O.trace_rk4(m, r, 1.0, 1e-3, 130, checkpoint_every=64)
    assert ck.shape == (5, 3, 6)
    assert np.array_equal(ck[:, 0], r.y * 0 + np.concatenate([wl.x0, k0], 1))
    r2 = O.make_rays(wl.x0, k0)
    O.trace_rk4(m, r2, 1.0, 1e-3, 64)
    assert np.array_equal(ck[:, 1], r2.y)
    O.trace_rk4(m, r2, 1.0, 1e-3, 66)
    assert np.array_equal(r2.y, r.y)
    assert (r2.steps == 130).all()


# ---------------------------------------------------------------- spline

def _fracs(s):
    return [float(Fraction(v.strip())) for v in s.split(",")]


def _bspline_golden():
    rows = {}
    for line in open(os.path.join(GOLDEN, "bspline_weights.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f, rest = line.split(":", 1)
        wv, dv = rest.split("|")
        rows[float(Fraction(f.strip()))] = (_fracs(wv), _fracs(dv))
    return rows


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_spline_weights_match_de_boor(axis):
    """A grid whose eps is a unit spike on one node plane along `axis`: the
    value and derivative at f = 0 and f = 1/2 are de Boor's B-spline weights
    (catches a wrong weight polynomial, a shifted stencil or a swapped axis)."""
    g = 16
    h = 2.0 / g
    grid = W.constant_grid(g)
    j = 7
    sl = [slice(None)] * 3
    sl[2 - axis] = j                      # grid index order is [iz, iy, ix]
    grid[tuple(sl) + (6,)] = 2.0          # eps = 1 + spike
    m = O.medium(kind="spline", grid=grid)
    gold = _bspline_golden()
    for f, (wv, dv) in gold.items():
        for a in range(4):                # spike weight when the stencil base is i = j + 1 - a
            i = j + 1 - a
            x = np.zeros((1, 3)) + 0.013
            x[0, axis] = -1 + (i + f) * h
            k = np.zeros((1, 3))
            ev = O.eval_dispersion(m, x, k, 1.0)
            eps = ev[0, 8]
            dEps = -ev[0, 1 + axis]       # D_x = -w^2 d eps / dx with k = 0
            assert abs(eps - (1 + wv[a])) < 1e-13
            assert abs(dEps - dv[a] / h) < 1e-11


def test_spline_reproduces_affine_fields():
    """Cubic B-splines reproduce affine functions exactly (away from the
    periodic seam): eps = 2 + x/2, M11 = 1 + y/4, M23 = z/8."""
    g = 16
    ax = -1 + (2.0 / g) * np.arange(g)
    grid = W.constant_grid(g)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    grid[..., 6] = 2 + X / 2
    grid[..., 0] = 1 + Y / 4
    grid[..., 4] = Z / 8
    m = O.medium(kind="spline", grid=grid)
    rng = np.random.default_rng(2)
    x = rng.uniform(-1 + 2 * 2.0 / g, 1 - 3 * 2.0 / g, (30, 3))
    k = rng.uniform(-1, 1, (30, 3))
    w = 0.7
    ev = O.eval_dispersion(m, x, k, w)
    eps = 2 + x[:, 0] / 2
    M11 = 1 + x[:, 1] / 4
    M23 = x[:, 2] / 8
    D = M11 * k[:, 0] ** 2 + k[:, 1] ** 2 + k[:, 2] ** 2 + 2 * M23 * k[:, 1] * k[:, 2] - w * w * eps
    np.testing.assert_allclose(ev[:, 0], D, atol=1e-14)
    np.testing.assert_allclose(ev[:, 8], eps, atol=1e-14)
    np.testing.assert_allclose(ev[:, 1], -w * w * 0.5, atol=1e-13)
    np.testing.assert_allclose(ev[:, 2], k[:, 0] ** 2 / 4, atol=1e-13)
    np.testing.assert_allclose(ev[:, 3], 2 * k[:, 1] * k[:, 2] / 8, atol=1e-13)
    np.testing.assert_allclose(ev[:, 4], 2 * M11 * k[:, 0], atol=1e-14)
    np.testing.assert_allclose(ev[:, 5], 2 * (k[:, 1] + M23 * k[:, 2]), atol=1e-14)
    np.testing.assert_allclose(ev[:, 7], -2 * w * eps, atol=1e-14)


def test_spline_periodicity_and_constant_medium_rays():
    """Lookups are periodic with period 2; a constant grid (M = I, eps = 1) is
    the homogeneous medium n = 1, so rays are straight lines at unit speed."""
    grid = W.aniso_grid(np.random.default_rng(4), g=16, n_modes=6)
    m = O.medium(kind="spline", grid=grid)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (10, 3))
    k = rng.uniform(-1, 1, (10, 3))
    a = O.eval_dispersion(m, x, k)
    b = O.eval_dispersion(m, x + np.array([2.0, -4.0, 6.0]), k)
    np.testing.assert_allclose(a, b, atol=1e-12)
    mc = O.medium(kind="spline", grid=W.constant_grid(16))
    x0 = rng.uniform(-1, 1, (8, 3))
    d = W.sphere_directions(rng, 8)
    k0, _ = O.onshell(mc, x0, d)
    r = O.make_rays(x0, k0)
    O.trace_rk4(mc, r, 1.0, 1e-2, 300)
    x_ex, _ = CF.straight(x0, k0, 1.0, 3.0)
    np.testing.assert_allclose(r.y[:, :3], x_ex, atol=1e-12)


def test_spline_workload_conserves_dispersion():
    """Anisotropic 128^3 workload on a seeded subset: D conserved along rays."""
    wl = W.aniso(n=16, g=32, n_modes=32)
    m = O.medium(**wl.medium)
    k0, _ = O.onshell(m, wl.x0, wl.d)
    r = O.make_rays(wl.x0, k0)
    O.trace_rk4(m, r, 1.0, wl.dt, 1000)
    assert (r.status == O.ACTIVE).all()
    assert r.dmax.max() < 1e-8


# ---------------------------------------------------------------- DOPRI5

def _tableau_golden():
    rows = {}
    for line in open(os.path.join(GOLDEN, "dopri5_tableau.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split(":", 1)
        rows[k.strip()] = [Fraction(s.strip()) for s in v.split(",")]
    return rows


def test_dopri5_golden_tableau_satisfies_order_conditions():
    """Pins the transcript of the published tableau: row sums equal c, the
    5th-order weights satisfy the quadrature conditions sum b c^q = 1/(q+1)
    (q < 5) and b*, of order 4, those up to q = 3."""
    g = _tableau_golden()
    c = g["c"]
    for i in range(2, 8):
        assert sum(g[f"a{i}"]) == c[i - 1]
    for q in range(5):
        assert sum(b * ci ** q for b, ci in zip(g["b"], c)) == Fraction(1, q + 1)
    for q in range(4):
        assert sum(b * ci ** q for b, ci in zip(g["bstar"], c)) == Fraction(1, q + 1)
    assert g["b"][:6] == g["a7"]
    # one non-quadrature order condition: sum b_i a_ij c_j = 1/6
    A = [[Fraction(0)] * 7 for _ in range(7)]
    for i in range(2, 8):
        for j, v in enumerate(g[f"a{i}"]):
            A[i - 1][j] = v
    assert sum(g["b"][i] * A[i][j] * c[j] for i in range(7) for j in range(7)) == Fraction(1, 6)


def test_oracle_dopri5_tableau_equals_published_values():
    g = _tableau_golden()
    t = O.dopri5_tableau()
    np.testing.assert_array_equal(t[0:7], [float(v) for v in g["c"]])
    A = t[7:49].reshape(7, 6)
    for i in range(2, 8):
        row = [float(v) for v in g[f"a{i}"]]
        np.testing.assert_array_equal(A[i - 1, :len(row)], row)
        assert (A[i - 1, len(row):] == 0).all()
    np.testing.assert_array_equal(t[49:56], [float(v) for v in g["b"]])
    np.testing.assert_array_equal(t[56:63], [float(v) for v in g["bstar"]])


def test_dopri5_error_follows_tolerance_on_ellipse():
    """Quadratic-law ellipse (closed form): the endpoint error at rtol = atol =
    1e-9 is ~1e-8 or better and shrinks with the tolerance; accepted steps grow
    roughly like tol^(-1/5) (catches a wrong error estimate or controller)."""
    rng = np.random.default_rng(21)
    m = O.medium(kind="quadratic")
    p = W.sphere_directions(rng, 6)
    u = W.sphere_directions(rng, 6)
    k0, _ = O.onshell(m, p, u)
    T = 2.0
    out = {}
    for tol in (1e-6, 1e-9):
        r = O.make_rays(p, k0)
        O.trace_dopri5([m], [0, 6], r, 1.0, rtol=tol, atol=tol, t_max=T, radius=0.0)
        assert (r.status == O.DONE).all()
        assert (r.t == T).all()
        e = max(np.abs(r.y[i, :3] - CF.quadratic(p[i], k0[i], T)[0]).max() for i in range(6))
        out[tol] = (e, r.steps.mean(), r.rejects.sum())
    assert out[1e-9][0] < 2e-8
    assert out[1e-6][0] > 10 * out[1e-9][0]
    q = out[1e-9][1] / out[1e-6][1]
    assert 2.5 < q < 6.5, out


def test_dopri5_luneburg_exits_and_statuses():
    """Luneburg rays from x = -1 pass the focus (1, 0, 0) and leave along -p,
    p the entry point on the lens (closed form); the first accepted step that
    ends outside r = 1.5 stops them (no event location, so the stopping point
    is anywhere on that straight line).  Budget and underflow statuses fire
    when provoked."""
    wl = W.luneburg(n=16)
    m = O.medium(kind="luneburg")
    r = O.make_rays(wl.x0, wl.d)
    O.trace_dopri5([m], [0, 16], r, 1.0, rtol=1e-9, atol=1e-9, radius=1.5)
    assert (r.status == O.EXITED).all()
    assert (np.linalg.norm(r.y[:, :3], axis=1) > 1.5).all()
    p = np.column_stack([-np.sqrt(1 - wl.x0[:, 1] ** 2 - wl.x0[:, 2] ** 2), wl.x0[:, 1:]])
    np.testing.assert_allclose(r.y[:, 3:], -p, atol=1e-5)
    off = np.cross(r.y[:, :3] - np.array([1.0, 0, 0]), -p)
    assert np.abs(off).max() < 1e-5
    # time on the line: focus at 1 + pi/2, unit speed outside the lens
    np.testing.assert_allclose(r.t, 1 + math.pi / 2 + np.linalg.norm(r.y[:, :3] - [1, 0, 0], axis=1),
                               atol=1e-5)
    r = O.make_rays(wl.x0, wl.d)
    O.trace_dopri5([m], [0, 16], r, 1.0, max_steps=5)
    assert (r.status == O.MAX_STEPS).all() and (r.steps == 5).all()
    r = O.make_rays(wl.x0[:2], wl.d[:2])
    O.trace_dopri5([m], [0, 2], r, 1.0, rtol=1e-20, atol=1e-20)
    assert (r.status == O.STEP_UNDERFLOW).all()


def test_dopri5_agrees_with_fine_rk4():
    """On a blobby medium, DOPRI5 at 1e-10 and RK4 with a fine fixed step land
    on the same point at the same time."""
    wl = W.batched(n_media=1, scale_counts=1.0 / 1024)
    blobs = wl.extra["blobs"][0]
    m = O.medium(kind="quadratic", blobs=blobs)
    rng = np.random.default_rng(8)
    p = 0.5 * W.sphere_directions(rng, 4)
    k0, _ = O.onshell(m, p, W.sphere_directions(rng, 4))
    r1 = O.make_rays(p, k0)
    O.trace_dopri5([m], [0, 4], r1, 1.0, rtol=1e-11, atol=1e-11, t_max=1.5, radius=0.0)
    r2 = O.make_rays(p, k0)
    O.trace_rk4(m, r2, 1.0, 1.5 / 6000, 6000)
    np.testing.assert_allclose(r1.y, r2.y, atol=1e-9)


def test_dopri5_kink_makes_step_placement_ill_conditioned():
    """The Luneburg surface |x| = 1 (grad n^2 jumps) makes the adaptive trace
    sensitive to the rounding of its step sizes: a relative change of 1e-6 in
    rtol (every step 2e-7 shorter) moves at least 5% of the endpoints at t = 2.5
    by more than 1e-9, while the same change in the kink-free quadratic law
    with the same blobs moves none by more than 1e-12.  This is the oracle's
    own conditioning, which bounds how closely any second implementation can
    follow it through the kink."""
    wl = W.batched(n_media=12, scale_counts=1.0 / 64)
    blobs, off = wl.extra["blobs"], wl.extra["offsets"]
    moved = {}
    for kind in ("luneburg", "quadratic"):
        media = [O.medium(kind=kind, blobs=blobs[j]) for j in range(12)]
        k0 = np.empty_like(wl.x0)
        for j in range(12):
            if off[j + 1] > off[j]:
                k0[off[j]:off[j + 1]], _ = O.onshell(media[j], wl.x0[off[j]:off[j + 1]], wl.d[off[j]:off[j + 1]])
        ys = []
        for rtol in (1e-9, 1e-9 * (1 + 1e-6)):
            r = O.make_rays(wl.x0, k0)
            O.trace_dopri5(media, off, r, 1.0, rtol=rtol, atol=1e-9, t_max=2.5, radius=0.0)
            assert (r.status == O.DONE).all()
            ys.append(r.y)
        moved[kind] = np.abs(ys[1] - ys[0]).max(axis=1)
    assert (moved["luneburg"] > 1e-9).mean() >= 0.05, (moved["luneburg"] > 1e-9).mean()
    assert moved["quadratic"].max() < 1e-12, moved["quadratic"].max()


# ---------------------------------------------------------------- sensitivities

def _adjoint_case(n_rays=3, n_blobs=3, n_steps=300, dt=1e-2):
    rng = np.random.default_rng(31)
    blobs = W.blob_table(rng, n_blobs, 0.05)
    blobs[:, 1:4] = rng.uniform(-0.3, 0.3, (n_blobs, 3))
    blobs[:, 4] = rng.uniform(0.2, 0.4, n_blobs)
    x0, d = W.plane_disk_rays(rng, n_rays, 0.5)
    x0[:, 0] = -0.9
    return blobs, x0, d, n_steps, dt


def test_tangent_sensitivities_match_trace_differences():
    """dy_N/dA_j from the tangent-linear RK4 vs central differences of whole
    oracle traces (brute force), on a Luneburg + blob medium whose rays stay
    clear of the kink (catches any Jacobian or dF/dA term error)."""
    for kind in ("quadratic", "grin"):
        blobs, x0, d, n, dt = _adjoint_case()
        if kind == "grin":
            x0[:, 1:] *= 0.1
        m = O.medium(kind=kind, blobs=blobs)
        k0, _ = O.onshell(m, x0, d)
        r = O.make_rays(x0, k0)
        S = O.tangent_rk4(m, r, 1.0, dt, n)
        ref = O.make_rays(x0, k0)
        O.trace_rk4(m, ref, 1.0, dt, n)
        assert np.array_equal(r.y, ref.y)
        h = 1e-6
        for j in range(blobs.shape[0]):
            bp, bm = blobs.copy(), blobs.copy()
            bp[j, 0] += h
            bm[j, 0] -= h
            rp = O.make_rays(x0, k0)
            O.trace_rk4(O.medium(kind=kind, blobs=bp), rp, 1.0, dt, n)
            rm = O.make_rays(x0, k0)
            O.trace_rk4(O.medium(kind=kind, blobs=bm), rm, 1.0, dt, n)
            fd = (rp.y - rm.y) / (2 * h)
            np.testing.assert_allclose(S[:, :, j], fd, atol=2e-7 * (1 + np.abs(fd).max()))


def test_loss_gradient_matches_loss_differences():
    """dL/dA for L = sum |x_N - x*|^2 vs central differences of L."""
    blobs, x0, d, n, dt = _adjoint_case(n_rays=5, n_blobs=4, n_steps=200)
    m = O.medium(kind="quadratic", blobs=blobs)
    k0, _ = O.onshell(m, x0, d)
    xstar = x0 + 1.0

    def loss(b):
        r = O.make_rays(x0, k0)
        O.trace_rk4(O.medium(kind="quadratic", blobs=b), r, 1.0, dt, n)
        return ((r.y[:, :3] - xstar) ** 2).sum()

    r = O.make_rays(x0, k0)
    S = O.tangent_rk4(m, r, 1.0, dt, n)
    g = O.loss_grad(r.y, xstar, S)
    h = 1e-6
    for j in range(4):
        bp, bm = blobs.copy(), blobs.copy()
        bp[j, 0] += h
        bm[j, 0] -= h
        fd = (loss(bp) - loss(bm)) / (2 * h)
        assert abs(g[j] - fd) < 1e-6 * max(1.0, abs(fd))


# ---------------------------------------------------------------- Newton k_x

def test_newton_kx_finds_the_closed_form_roots():
    """Isotropic: k_x = +-sqrt(w^2 n^2 - k_y^2 - k_z^2), the sign of the guess
    picks the branch; |D| below the paper's 1e-15 (Sec. 4) or at rounding."""
    m = O.medium(kind="grin", n0=1.5, a=2.0, blobs=W.blob_table(np.random.default_rng(7), 4, 0.01))
    rng = np.random.default_rng(8)
    x = rng.uniform(-0.2, 0.2, (40, 3))
    kyz = rng.uniform(-0.5, 0.5, (40, 2))
    n2 = O.eval_dispersion(m, x, np.zeros((40, 3)), 1.3)[:, 8]
    exact = np.sqrt(1.3 ** 2 * n2 - (kyz ** 2).sum(1))
    for sign in (1.0, -1.0):
        k = np.column_stack([sign * np.full(40, 0.7), kyz])
        kk, st, it = O.newton_kx(m, x, k, 1.3)
        assert (st == O.ACTIVE).all() and (it < 12).all()
        np.testing.assert_allclose(kk[:, 0], sign * exact, rtol=1e-15)
        np.testing.assert_array_equal(kk[:, 1:], kyz)
        assert np.abs(O.eval_dispersion(m, x, kk, 1.3)[:, 0]).max() <= 8e-15


def test_newton_kx_spline_quadratic_roots_and_no_root():
    """Spline medium: D is quadratic in k_x, M11 k_x^2 + 2 b k_x + c = 0 with
    b = M12 k_y + M13 k_z, c = M22 k_y^2 + 2 M23 k_y k_z + M33 k_z^2 - w^2 eps;
    rays with k_y, k_z too large have no real root and get the cut-off status."""
    grid = W.aniso_grid(np.random.default_rng(9), g=16, n_modes=6)
    m = O.medium(kind="spline", grid=grid)
    rng = np.random.default_rng(10)
    x = rng.uniform(-1, 1, (30, 3))
    kyz = rng.uniform(-0.3, 0.3, (30, 2))
    ev = O.eval_dispersion(m, x, np.column_stack([np.ones(30), np.zeros((30, 2))]), 1.0)
    # D(k_x = 1, 0, 0) = M11 - eps and D_k = 2 M e_x give M11, M12, M13; probe the rest
    M = np.empty((30, 3, 3))
    for c in range(3):
        e = np.zeros((30, 3))
        e[:, c] = 1.0
        M[:, :, c] = O.eval_dispersion(m, x, e, 1.0)[:, 4:7] / 2
    eps = ev[:, 8]
    b = M[:, 0, 1] * kyz[:, 0] + M[:, 0, 2] * kyz[:, 1]
    c = (M[:, 1, 1] * kyz[:, 0] ** 2 + 2 * M[:, 1, 2] * kyz[:, 0] * kyz[:, 1]
         + M[:, 2, 2] * kyz[:, 1] ** 2 - eps)
    disc = np.sqrt(b * b - M[:, 0, 0] * c)
    roots = {1.0: (-b + disc) / M[:, 0, 0], -1.0: (-b - disc) / M[:, 0, 0]}
    for sign in (1.0, -1.0):
        kk, st, _ = O.newton_kx(m, x, np.column_stack([np.full(30, 3 * sign), kyz]))
        assert (st == O.ACTIVE).all()
        np.testing.assert_allclose(kk[:, 0], roots[sign], rtol=1e-13, atol=1e-15)
    kk, st, it = O.newton_kx(m, x[:3], np.column_stack([np.ones(3), np.full((3, 2), 3.0)]), max_iter=60)
    assert (st == O.CUTOFF).all()


# ---------------------------------------------------------------- cold plasma

COLD2 = dict(kind="cold", species=((0.45, -0.6), (0.03, 0.08)), profile=(1.0, 0.1, 1.0, 0.05))
COLD_E = dict(kind="cold", species=((0.3, -0.5),), profile=(1.0, 0.1, 1.0, 0.0))


def _cold_det(spec, x, k, w):
    """det(eps + n n - n^2 I) with the dielectric tensor of Eqs. 7-10, complex numpy."""
    f0, f1, g0, g1 = spec["profile"]
    out = []
    for xi, ki in zip(x, k):
        f, g = f0 + f1 * xi[0], g0 + g1 * xi[0]
        e11 = 1 - sum(wp2 * f / w ** 2 / (1 - (om * g) ** 2 / w ** 2) for wp2, om in spec["species"])
        e12 = -1j * sum((om * g / w) * (wp2 * f / w ** 2) / (1 - (om * g) ** 2 / w ** 2)
                        for wp2, om in spec["species"])
        e33 = 1 - sum(wp2 * f / w ** 2 for wp2, _ in spec["species"])
        eps = np.array([[e11, e12, 0], [-e12, e11, 0], [0, 0, e33]])
        n = ki / w
        out.append(np.linalg.det(eps + np.outer(n, n) - (n @ n) * np.eye(3)))
    return np.array(out)


def test_cold_plasma_D_equals_the_determinant():
    """The Stix-form D against the determinant of Eq. 5 built from Eqs. 6-10
    (catches a wrong sign of eps12, a swapped S/P, a wrong n_parallel axis)."""
    rng = np.random.default_rng(20)
    x = rng.uniform(-3, 3, (25, 3))
    k = rng.uniform(-1.5, 1.5, (25, 3))
    for w in (1.0, 1.7):
        D = O.eval_dispersion(O.medium(**COLD2), x, k, w)[:, 0]
        det = _cold_det(COLD2, x, k, w)
        assert np.abs(det.imag).max() < 1e-12
        np.testing.assert_allclose(D, det.real, rtol=1e-12, atol=1e-12)


def test_cold_plasma_partials_match_central_differences():
    m = O.medium(**COLD2)
    rng = np.random.default_rng(21)
    x = rng.uniform(-3, 3, (12, 3))
    k = rng.uniform(-1.5, 1.5, (12, 3))
    w, h = 1.3, 1e-4
    ev = O.eval_dispersion(m, x, k, w)
    Dx = _fd5(lambda xx: O.eval_dispersion(m, xx, k, w)[:, 0], x, h)
    Dk = _fd5(lambda kk: O.eval_dispersion(m, x, kk, w)[:, 0], k, h)
    Dw = (-O.eval_dispersion(m, x, k, w + 2 * h)[:, 0] + 8 * O.eval_dispersion(m, x, k, w + h)[:, 0]
          - 8 * O.eval_dispersion(m, x, k, w - h)[:, 0] + O.eval_dispersion(m, x, k, w - 2 * h)[:, 0]) / (12 * h)
    scale = 1 + np.abs(ev[:, 1:8]).max()
    np.testing.assert_allclose(ev[:, 1:4], Dx, atol=1e-8 * scale)
    np.testing.assert_allclose(ev[:, 4:7], Dk, atol=1e-8 * scale)
    np.testing.assert_allclose(ev[:, 7], Dw, atol=1e-8 * scale)


def test_cold_plasma_newton_finds_O_and_X_roots():
    """For k_z = 0, D = (S a - R L)(a - P): the O root a = P and the X root
    a = R L / S; Newton from a guess near each returns it (Sec. 4: the guess
    selects the branch)."""
    m = O.medium(**COLD_E)
    x = np.array([[0.0, 0, 0], [2.0, 0, 0], [-1.0, 0, 0]])
    ky = np.array([0.1, 0.3, 0.0])
    f = 1 + 0.1 * x[:, 0]
    P = 1 - 0.3 * f
    R, L = 1 - 0.3 * f / 0.5, 1 - 0.3 * f / 1.5
    S = (R + L) / 2
    kO = np.sqrt(P - ky ** 2)
    kX = np.sqrt(R * L / S - ky ** 2)
    for guess, exact in ((kO + 0.05, kO), (kX - 0.05, kX)):
        k, st, _ = O.newton_kx(m, x, np.column_stack([guess, ky, np.zeros(3)]))
        assert (st == O.ACTIVE).all()
        np.testing.assert_allclose(k[:, 0], exact, rtol=1e-13)


def test_cold_plasma_O_mode_parabola_is_exact():
    """O-mode in the x-y plane of the linear-density slab (Eq. 4): on the O
    branch the ray equations reduce to dx/dt = k / w, dk_x/dt = w P_x / 2 with
    P_x constant, so the ray is a parabola in t -- reproduced by RK4 to
    rounding; k_y, k_z = 0 and D are conserved; the ray turns where k_x = 0."""
    m = O.medium(**COLD2)
    w = 1.0
    x0 = np.array([[0.0, 0.2, 0.0], [-1.0, 0.0, 0.0], [0.5, -0.3, 0.0]])
    ky = np.array([0.2, 0.0, -0.15])
    f = 1 + 0.1 * x0[:, 0]
    Wsum = 0.45 + 0.03
    P = 1 - Wsum * f / w ** 2
    k0 = np.column_stack([np.sqrt(w ** 2 * P - ky ** 2), ky, np.zeros(3)])
    assert np.abs(O.eval_dispersion(m, x0, k0, w)[:, 0]).max() < 1e-14
    r = O.make_rays(x0, k0)
    T, n = 60.0, 6000                                 # turns near t = 29
    O.trace_rk4(m, r, w, T / n, n)
    c = -Wsum * 0.1 / (2 * w)                         # dk_x/dt = w P_x / 2
    kx = k0[:, 0] + c * T
    xx = x0[:, 0] + (k0[:, 0] * T + c * T * T / 2) / w
    yy = x0[:, 1] + ky * T / w
    np.testing.assert_allclose(r.y[:, 3], kx, atol=1e-12)
    np.testing.assert_allclose(r.y[:, 0], xx, atol=1e-11)
    np.testing.assert_allclose(r.y[:, 1], yy, atol=1e-11)
    assert (r.y[:, 5] == 0).all() and (r.y[:, 2] == 0).all()
    assert (kx < 0).all()                             # reflected off the P = k_y^2/w^2 cut-off
    assert r.dmax.max() < 1e-12


def test_cold_plasma_X_mode_reflects_at_R_cutoff():
    """X-mode launched along +x into rising density (uniform B) turns at the
    R = 0 cut-off, f(x_R) = w (w + Omega_e) / w_pe^2, well before the upper
    hybrid resonance (S = 0) and the O cut-off (P = 0)."""
    m = O.medium(**COLD_E)
    x0 = np.zeros((1, 3))
    k, st, _ = O.newton_kx(m, x0, np.array([[0.7, 0.0, 0.0]]))
    f = 1.0
    R, L, P = 1 - 0.3 * f / 0.5, 1 - 0.3 * f / 1.5, 1 - 0.3 * f
    S = (R + L) / 2
    np.testing.assert_allclose(k[0, 0], np.sqrt(R * L / S), rtol=1e-13)
    xR = (1.0 * (1.0 - 0.5) / 0.3 - 1.0) / 0.1
    xs = []
    r = O.make_rays(x0, k)
    for _ in range(400):
        O.trace_rk4(m, r, 1.0, 0.01, 10)
        xs.append(r.y[0, 0])
    xs = np.array(xs)
    assert abs(xs.max() - xR) < 1e-3, (xs.max(), xR)
    assert xs[-1] < xs.max() - 0.03 and r.y[0, 3] < 0     # on its way back
    assert r.dmax.max() < 1e-9 and r.status[0] == O.ACTIVE
