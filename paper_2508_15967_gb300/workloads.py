"""Seeded synthetic inputs for the ray-tracing workloads.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no dispersion relation, no gradient, no integrator).  It
is the one module that both the CUDA path and the CPU oracle consume.

Every array is produced by ``numpy.random.default_rng(seed)`` with
``seed = 250815967 + workload index`` (1 = Luneburg lens, 2 = GRIN fibre,
3 = anisotropic spline, 4 = batched media, 5 = adjoint), and the hidden
adjoint target amplitudes use ``seed + 1000``.

Rays are returned as launch points ``x0`` (n, 3) and launch directions ``d``
(n, 3) in float64; the on-shell wave vector k0 = s * d is computed by the
library (``gf_rays_onshell``) or by the oracle, never here, because it needs
the medium.

Blob tables are (n_blobs, 5) float64 rows ``(A, cx, cy, cz, w)``: a Gaussian
A * exp(-|x - c|^2 / (2 w^2)) added to the squared refractive index.

The anisotropic grid is (g, g, g, 8) float32, x fastest:
``grid[iz, iy, ix] = (M11, M12, M13, M22, M23, M33, eps, 0)`` at node
``(-1 + ix*h, -1 + iy*h, -1 + iz*h)``, h = 2/g, periodic with period 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 250815967

LUNEBURG, GRIN, ANISO, BATCHED, ADJOINT, COLD = 1, 2, 3, 4, 5, 6


def rng_for(index: int, offset: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + index + offset)


# --------------------------------------------------------------------------- rays

def plane_disk_rays(rng: np.random.Generator, n: int, radius: float, x_plane: float = -1.0):
    """Launch points on the plane x = x_plane, (y, z) uniform in a disk; direction +x."""
    r = radius * np.sqrt(rng.random(n))
    phi = 2.0 * math.pi * rng.random(n)
    x0 = np.empty((n, 3))
    x0[:, 0] = x_plane
    x0[:, 1] = r * np.cos(phi)
    x0[:, 2] = r * np.sin(phi)
    d = np.zeros((n, 3))
    d[:, 0] = 1.0
    return x0, d


def morton_order(p: np.ndarray) -> np.ndarray:
    """Permutation listing 2-D points p (n, 2) along a Z-order (Morton) curve of
    a 2^16 x 2^16 grid over their bounding box: consecutive points are
    neighbours, as when a launcher sweeps its aperture, so that a warp traces
    rays that stay close together (the same set of rays in another order)."""
    if len(p) == 0:
        return np.zeros(0, dtype=np.int64)
    lo = p.min(axis=0)
    span = np.maximum(p.max(axis=0) - lo, 1e-300)
    q = np.minimum((p - lo) / span * 65536.0, 65535.0).astype(np.uint64)

    def spread(v):   # bit i of v moves to bit 2 i
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
        return (v | (v << np.uint64(1))) & np.uint64(0x55555555)

    code = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1))
    return np.argsort(code, kind="stable")


def aperture_rays(rng: np.random.Generator, n: int, radius: float, morton: bool = True):
    """plane_disk_rays listed in Morton order of their launch points (y0, z0),
    or in the order drawn (morton = False)."""
    x0, d = plane_disk_rays(rng, n, radius)
    if not morton:
        return x0, d
    o = morton_order(x0[:, 1:])
    return x0[o], d[o]


def cone_directions(rng: np.random.Generator, n: int, half_angle_deg: float):
    """Unit vectors uniform in solid angle on the cap of the given half-angle about +x."""
    cmin = math.cos(math.radians(half_angle_deg))
    c = 1.0 - rng.random(n) * (1.0 - cmin)
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    phi = 2.0 * math.pi * rng.random(n)
    return np.stack([c, s * np.cos(phi), s * np.sin(phi)], axis=1)


def sphere_directions(rng: np.random.Generator, n: int):
    """Unit vectors uniform on S^2."""
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def blob_table(rng: np.random.Generator, n_blobs: int, amp_sigma: float,
               centre_half: float = 0.5, w_lo: float = 0.05, w_hi: float = 0.2):
    """(n_blobs, 5) rows (A, cx, cy, cz, w): A ~ N(0, amp_sigma), c ~ U[-h, h]^3, w ~ U[w_lo, w_hi]."""
    A = rng.normal(0.0, amp_sigma, n_blobs)
    c = rng.uniform(-centre_half, centre_half, (n_blobs, 3))
    w = rng.uniform(w_lo, w_hi, n_blobs)
    return np.column_stack([A, c, w]).astype(np.float64)


# --------------------------------------------------------------------------- grid

def fourier_field(rng: np.random.Generator, axis: np.ndarray, n_modes: int = 32, kmax: int = 3):
    """sum_m a_m cos(pi kappa_m . x + phi_m) on the tensor grid axis^3 (index [iz, iy, ix]).

    kappa_m integer in [-kmax, kmax]^3 minus the origin, a_m ~ N(0,1)/sqrt(n_modes),
    phi_m ~ U[0, 2 pi).  Periodic with period 2 along every axis.
    """
    kap = np.zeros((n_modes, 3), dtype=np.int64)
    for m in range(n_modes):
        while True:
            v = rng.integers(-kmax, kmax + 1, 3)
            if np.any(v != 0):
                kap[m] = v
                break
    amp = rng.standard_normal(n_modes) / math.sqrt(n_modes)
    ph = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    g = axis.size
    # separable evaluation: cos(pi kappa.x + phi) = Re(e^{i phi} e^{i pi kx x} e^{i pi ky y} e^{i pi kz z})
    E = [np.exp(1j * math.pi * kap[:, c, None] * axis[None, :]) for c in range(3)]   # (m, g) each
    T = (amp * np.exp(1j * ph))[:, None, None] * E[2][:, :, None] * E[1][:, None, :]  # (m, z, y)
    out = (T.reshape(n_modes, g * g).T @ E[0]).real                                   # (z*y, x)
    return out.reshape(g, g, g)


def aniso_grid(rng: np.random.Generator, g: int = 128, n_modes: int = 32):
    """(g, g, g, 8) float32 nodes (M11, M12, M13, M22, M23, M33, eps, 0).

    M = I + 0.2 S S^T with S a 3x3 field of smooth random scalars, eps = exp(0.2 phi).
    Fields are sampled in float64 and rounded once to float32.
    """
    axis = -1.0 + (2.0 / g) * np.arange(g)
    S = np.empty((3, 3, g, g, g))
    for i in range(3):
        for j in range(3):
            S[i, j] = fourier_field(rng, axis, n_modes)
    phi = fourier_field(rng, axis, n_modes)
    M = np.einsum("ik...,jk...->ij...", S, S) * 0.2
    for i in range(3):
        M[i, i] += 1.0
    grid = np.zeros((g, g, g, 8), dtype=np.float32)
    grid[..., 0] = M[0, 0]
    grid[..., 1] = M[0, 1]
    grid[..., 2] = M[0, 2]
    grid[..., 3] = M[1, 1]
    grid[..., 4] = M[1, 2]
    grid[..., 5] = M[2, 2]
    grid[..., 6] = np.exp(0.2 * phi)
    return grid


def constant_grid(g: int, M=(1.0, 0.0, 0.0, 1.0, 0.0, 1.0), eps: float = 1.0):
    grid = np.zeros((g, g, g, 8), dtype=np.float32)
    grid[..., :6] = np.asarray(M, dtype=np.float32)
    grid[..., 6] = eps
    return grid


# --------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    medium: dict                      # keyword arguments of a medium description
    x0: np.ndarray                    # (n, 3) launch points
    d: np.ndarray                     # (n, 3) launch directions
    omega: float = 1.0
    dt: float = 0.0
    n_steps: int = 0
    radius: float = 0.0               # termination radius, 0 = none
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.x0.shape[0]


def luneburg(n: int = 1024, n_steps: int = 2000, dt: float = 1e-3) -> Workload:
    """Luneburg lens, no blobs; launch plane x = -1, disk radius 0.9, along +x
    (rays in Morton order of their launch points)."""
    rng = rng_for(LUNEBURG)
    x0, d = aperture_rays(rng, n, 0.9)
    return Workload("luneburg", dict(kind="luneburg"), x0, d, 1.0, dt, n_steps)


def grin(n: int = 1 << 20, n_steps: int = 10000, dt: float = 5e-4, n_blobs: int = 16,
         shard: int = 0) -> Workload:
    """Parabolic GRIN fibre n0 = 1.5, a = 2, plus Gaussian blobs.

    Launch points (-1, y0, z0) with (y0, z0) uniform in a disk of radius 0.05;
    directions uniform in solid angle within 10 degrees of +x.  The blob table
    is drawn first so that it does not depend on n.  ``shard`` > 0 draws an
    independent batch of rays in the same medium (one per GPU).
    """
    rng = rng_for(GRIN)
    blobs = blob_table(rng, n_blobs, 0.01)
    rr = rng_for(GRIN, 7 + 1000 * shard)
    x0, _ = plane_disk_rays(rr, n, 0.05)
    d = cone_directions(rr, n, 10.0)
    med = dict(kind="grin", n0=1.5, a=2.0, blobs=blobs)
    return Workload("grin", med, x0, d, 1.0, dt, n_steps)


def aniso(n: int = 262144, n_steps: int = 4000, dt: float = 1e-3, g: int = 128,
          n_modes: int = 32) -> Workload:
    """Anisotropic D = k^T M k - w^2 eps on a periodic g^3 tricubic B-spline grid."""
    rng = rng_for(ANISO)
    grid = aniso_grid(rng, g, n_modes)
    rr = rng_for(ANISO, 7)
    x0 = rr.uniform(-1.0, 1.0, (n, 3))
    d = sphere_directions(rr, n)
    return Workload("aniso", dict(kind="spline", grid=grid), x0, d, 1.0, dt, n_steps)


def batched(n_media: int = 4096, n_blobs: int = 8, e_lo: int = 4, e_hi: int = 14,
            scale_counts: float = 1.0, morton: bool = True, shard: int = 0) -> Workload:
    """Many Luneburg+blob media with power-of-two ray counts 2^U{e_lo..e_hi}.

    Rays of medium m occupy [offsets[m], offsets[m+1]) and launch as in the
    Luneburg workload (each medium's rays in Morton order of their launch
    points, or in the order drawn with ``morton = False``).  ``scale_counts``
    < 1 shrinks every count (at least 1 ray) for test-sized cases while
    keeping the unevenness.  ``shard`` > 0 draws an independent batch (media
    and rays) of the same shape, one per GPU of a weak-scaling run.
    """
    rng = rng_for(BATCHED) if shard == 0 else rng_for(BATCHED, 3 + 1000 * shard)
    exps = rng.integers(e_lo, e_hi + 1, n_media)
    counts = np.maximum(1, np.round((2.0 ** exps) * scale_counts)).astype(np.int64)
    blobs = np.stack([blob_table(rng, n_blobs, 0.02) for _ in range(n_media)])
    offsets = np.zeros(n_media + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    rr = rng_for(BATCHED, 7 + 1000 * shard)
    x0, d = plane_disk_rays(rr, int(offsets[-1]), 0.9)
    for m in range(n_media if morton else 0):
        lo, hi = int(offsets[m]), int(offsets[m + 1])
        o = morton_order(x0[lo:hi, 1:])
        x0[lo:hi], d[lo:hi] = x0[lo:hi][o], d[lo:hi][o]
    wl = Workload("batched", dict(kind="luneburg"), x0, d, 1.0, 1e-3, 0, 1.5)
    wl.extra = dict(blobs=blobs, offsets=offsets, counts=counts,
                    rtol=1e-9, atol=1e-9, h0=1e-3, t_max=10.0, max_steps=100000)
    return wl


def adjoint(n: int = 65536, n_steps: int = 4000, dt: float = 1e-3, n_blobs: int = 64,
            checkpoint_every: int = 64, morton: bool = True, shard: int = 0) -> Workload:
    """Luneburg base + n_blobs Gaussian blobs whose amplitudes theta are the parameters.

    theta ~ N(0, 0.01) (seed 250815967+5), hidden theta* from seed + 1000;
    centres and widths are shared by both.  Rays launch as in the Luneburg
    workload, in Morton order of their launch points (or in the order drawn
    with ``morton = False``).  ``shard`` > 0 draws an independent set of rays
    for the same medium and parameters (one per GPU of a weak-scaling run).
    """
    rng = rng_for(ADJOINT)
    blobs = blob_table(rng, n_blobs, 0.01)
    theta_star = rng_for(ADJOINT, 1000).normal(0.0, 0.01, n_blobs)
    rr = rng_for(ADJOINT, 7 + 1000 * shard)
    x0, d = aperture_rays(rr, n, 0.9, morton)
    wl = Workload("adjoint", dict(kind="luneburg", blobs=blobs), x0, d, 1.0, dt, n_steps)
    wl.extra = dict(theta=blobs[:, 0].copy(), theta_star=theta_star,
                    checkpoint_every=checkpoint_every)
    return wl


def cold(n: int = 1 << 20, n_steps: int = 1500, dt: float = 1e-2) -> Workload:
    """Cold magnetised plasma slab (Sec. 4.1): electrons and ions with squared
    plasma frequencies 0.7 and 0.02 times the density f(x) = 1 + 0.1 x (the
    linear gradient of Eq. 4) and cyclotron frequencies -0.5 and 0.05 times
    g(x) = 1 + 0.05 x, w = 1.  Rays start at (x, y, 0) with x, y uniform in
    [-1, 1), k_y uniform in +-0.25, k_z in +-0.2; k_x is the O-branch root
    found by Newton from k_x = 1.2 (extra["k_start"] holds the start).  By
    t = 15 most rays have reflected at the O-mode cut-off (x ~ 4.3) and the
    density stays positive along every ray."""
    rr = rng_for(COLD, 7)
    x0 = np.column_stack([rr.uniform(-1.0, 1.0, n), rr.uniform(-1.0, 1.0, n), np.zeros(n)])
    k_start = np.column_stack([np.full(n, 1.2), rr.uniform(-0.25, 0.25, n), rr.uniform(-0.2, 0.2, n)])
    med = dict(kind="cold", species=((0.7, -0.5), (0.02, 0.05)), profile=(1.0, 0.1, 1.0, 0.05))
    wl = Workload("cold", med, x0, np.zeros_like(x0), 1.0, dt, n_steps)
    wl.extra = dict(k_start=k_start)
    return wl
