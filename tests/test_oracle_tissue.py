"""Pins of the tissue-overlap elasticity factor (App. A.1): c_delta =
sum_k frac_k f_k + (1 - sum_k frac_k) f_0, frac_k counted over the voxel
centres of the tet's reference copy (exact association, reading R3).

- A mask of one tissue gives that tissue's factor to every tet that contains
  a voxel centre; a tet with none keeps the factor of its label.
- c_delta is linear in the factors.
- One large tet against a half-space mask: the count of voxel centres per
  tissue, done here in exact integer arithmetic with numpy (no tie lies on a
  face by construction), gives c_delta exactly; and it approaches the
  continuous volume fraction 1 - ((L - c) / L)^3 of the corner tet cut by
  the plane x = c.
"""

import numpy as np
import pytest

import oracle
import synth
from helpers import box_lattice, problem


def _with_mask(prob, mask, factors, labels=None):
    prob.tissue_mask = np.ascontiguousarray(mask, np.uint8)
    prob.tissue_factor = np.asarray(factors, np.float64)
    if labels is not None:
        prob.tet_label = np.asarray(labels, np.int32)
    return prob


def test_single_tissue_and_empty_tets(oracle_lib):
    n = 10
    img = np.zeros((n, n, n), np.float32)
    pts, tets = box_lattice(np.linspace(-0.5, n - 0.5, 3), np.linspace(-0.5, n - 0.5, 3), np.linspace(-0.5, n - 0.5, 3))
    # one extra sliver tet between voxel-centre planes: no voxel centre
    sliver = np.array([[2.1, 2.1, 2.1], [2.9, 2.2, 2.2], [2.2, 2.9, 2.3], [2.3, 2.3, 2.9]], np.float32)
    pts2 = np.concatenate([pts, sliver])
    tets2 = np.concatenate([tets, np.arange(len(pts), len(pts) + 4, dtype=np.int32)[None]])
    labels = np.zeros(len(tets2), np.int32)
    labels[-1] = 2
    prob = _with_mask(problem(img, img, pts2, tets2, g_mode=2), np.full((n, n, n), 1, np.uint8),
                      [1.0, 4.0, 7.0], labels)
    c = oracle.Oracle(prob).cdelta()
    assert (c[:-1] == 4.0).all()
    assert c[-1] == 7.0


def test_linear_in_the_factors(oracle_lib):
    p = synth.make_c0(n_sol=1)
    la, _ = synth.label_pair((32, 32, 32), synth.phantom.C0_ELLIPSOIDS, 2.0)
    L = int(la.max()) + 1
    rng = np.random.default_rng(3)
    f1, f2 = rng.uniform(0.5, 3.0, L), rng.uniform(0.5, 3.0, L)
    c1 = oracle.Oracle(_with_mask(p, la, f1)).cdelta()
    c2 = oracle.Oracle(_with_mask(p, la, f2)).cdelta()
    c12 = oracle.Oracle(_with_mask(p, la, f1 + f2)).cdelta()
    np.testing.assert_allclose(c12, c1 + c2, rtol=1e-12)
    assert len(np.unique(np.round(c1, 9))) > 2      # the organs split some tets


def _orient(a, b, c, d):
    u, v, w = b - a, c - a, d - a
    return (u[..., 0] * (v[..., 1] * w[..., 2] - v[..., 2] * w[..., 1])
            + u[..., 1] * (v[..., 2] * w[..., 0] - v[..., 0] * w[..., 2])
            + u[..., 2] * (v[..., 0] * w[..., 1] - v[..., 1] * w[..., 0]))


def test_half_space_closed_forms(oracle_lib):
    n, L, cut = 48, 40.0, 12
    off = np.array([1.296875, 1.203125, 1.109375])           # multiples of 2^-8: exact on the snap grid
    verts = np.array([[0, 0, 0], [L, 0, 0], [0, L, 0], [0, 0, L]]) + off
    img = np.zeros((n, n, n), np.float32)
    mask = np.zeros((n, n, n), np.uint8)
    mask[:, :, :cut + 1] = 1                                  # x <= cut
    f = np.array([1.0, 3.0])
    prob = _with_mask(problem(img, img, verts.astype(np.float32), np.array([[0, 1, 2, 3]], np.int32), g_mode=2),
                      mask, f)
    c = oracle.Oracle(prob).cdelta()[0]
    # exact count of voxel centres strictly inside, in integers (units of 2^-8 voxel)
    q = np.round((verts + 0.5) * 256).astype(np.int64)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    P = np.stack([i, j, k], -1).reshape(-1, 3).astype(np.int64) * 256 + 128
    D = _orient(*q)
    assert D > 0
    inside = np.ones(len(P), bool)
    for m in range(4):
        w = [np.broadcast_to(v, P.shape) for v in q]
        w[m] = P
        Dm = _orient(*w)
        assert (Dm != 0).all()                                # no tie by construction
        inside &= Dm > 0
    lab = mask.reshape(-1)[inside]
    want = (np.sum(lab == 0) * f[0] + np.sum(lab == 1) * f[1]) / inside.sum()
    assert c == want
    # ... and close to the continuous volume fraction of the plane x = cut + 1/2
    frac = 1.0 - ((L - (cut + 0.5 - off[0])) / L) ** 3
    assert abs(c - (f[0] + (f[1] - f[0]) * frac)) < 0.05
