"""Synthetic workload generators (host only): the uneven cell batch and the k-point
mesh match their stated recipes, deterministically."""
import math

import numpy as np

from paper_1603_04339_gb300 import synth


def test_cell_batch_recipe():
    cells = synth.config4()
    again = synth.config4()
    assert len(cells) == 16
    grids = {g for _, g in synth.CELL_GRIDS}
    for c, d in zip(cells, again):
        assert c.n in grids and c.h == (0.45, 0.45, 0.45)
        assert 8 <= len(c.atoms) <= 96 and 48 <= c.ns <= 384 and c.m in (16, 20, 24)
        assert c.proj.nproj == 4 * len(c.atoms)
        assert c.veff.shape == (c.nd,)
        assert np.array_equal(c.veff, d.veff) and c.ns == d.ns and c.m == d.m
        L = np.array(c.n) * 0.45
        if "slab" in c.name:
            assert np.all(np.abs(c.atoms[:, 2]) <= 0.25 * L[2] + 1e-12)
        if "wire" in c.name:
            assert np.all(np.abs(c.atoms[:, :2]) <= 0.25 * L[:2] + 1e-12)
    assert len({c.n for c in cells}) >= 4   # the batch is uneven


def test_separable_gaussian_potential_matches_the_image_sum():
    rng = np.random.default_rng(5)
    n, h = (9, 8, 7), (0.7, 0.6, 0.8)
    L = np.array([n[s] * h[s] for s in range(3)])
    sites = rng.uniform(-0.5, 0.5, (3, 3)) * L
    d, w = rng.uniform(-2, 0, 3), rng.uniform(0.8, 1.5, 3)
    v = synth.gaussian_veff(n, h, sites, d, w)
    xs = synth.node_coords(n, h)
    ref = np.zeros(n[::-1])
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                x = np.array([xs[0][i], xs[1][j], xs[2][k]])
                for R, dd, ww in zip(sites, d, w):
                    for t in np.ndindex(3, 3, 3):
                        r = x - R - (np.array(t) - 1) * L
                        ref[k, j, i] += dd * math.exp(-float(r @ r) / (ww * ww))
    assert np.max(np.abs(v - ref.reshape(-1))) < 1e-13
