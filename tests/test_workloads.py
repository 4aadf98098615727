"""Seeded input generators: determinism and the Morton ordering of aperture
launches (a permutation that keeps consecutive rays close)."""
from __future__ import annotations

import numpy as np

from paper_2508_15967_gb300 import workloads as W


def test_morton_order_is_a_locality_preserving_permutation():
    rng = np.random.default_rng(0)
    p = rng.uniform(-1, 1, (4096, 2))
    o = W.morton_order(p)
    assert sorted(o.tolist()) == list(range(len(p)))
    step_sorted = np.linalg.norm(np.diff(p[o], axis=0), axis=1).mean()
    step_random = np.linalg.norm(np.diff(p, axis=0), axis=1).mean()
    assert step_sorted < 0.1 * step_random
    # the Z curve of the unit square's corners
    corners = np.array([[0.0, 0.0], [1.0, 1.0], [0.0, 1.0], [1.0, 0.0]])
    assert W.morton_order(corners).tolist() == [0, 3, 2, 1]
    assert W.morton_order(np.zeros((0, 2))).size == 0


def test_aperture_workloads_are_deterministic_and_reordered_only():
    a, b = W.adjoint(n=2048, n_steps=10), W.adjoint(n=2048, n_steps=10)
    assert np.array_equal(a.x0, b.x0) and np.array_equal(a.d, b.d)
    rr = W.rng_for(W.ADJOINT, 7)
    x0, _ = W.plane_disk_rays(rr, 2048, 0.9)
    key = lambda x: np.lexsort((x[:, 2], x[:, 1]))
    assert np.array_equal(x0[key(x0)], a.x0[key(a.x0)])        # same rays, other order
    bt = W.batched(n_media=6, scale_counts=1 / 64)
    off = bt.extra["offsets"]
    rr = W.rng_for(W.BATCHED, 7)
    xb, _ = W.plane_disk_rays(rr, int(off[-1]), 0.9)
    for m in range(6):                                           # reordered within each medium
        lo, hi = off[m], off[m + 1]
        assert np.array_equal(np.sort(xb[lo:hi, 1]), np.sort(bt.x0[lo:hi, 1]))
