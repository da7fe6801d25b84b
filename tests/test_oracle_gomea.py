"""Pins of the model-building oracle (readings R19-R21: selection,
clustering, estimation and sampling of FOS elements, adaptive steering;
Sec. 3 and Sec. 4.3.2).

Front ranks against a count of dominating solutions, farthest-first
leaders and balanced clusters on configurations whose answer is known by
hand, the estimate against a closed-form covariance, sampling on a
diagonal factor, and the steering window by hand."""

import math

import numpy as np
import pytest

from oracle import gomea as gm


def test_front_ranks_by_hand_and_by_peeling():
    obj = np.array([[1, 5, 0], [2, 4, 0], [3, 3, 0], [2, 5, 0], [3, 4, 0], [4, 4, 0], [1, 5, 0]], float)
    r = gm.front_ranks(obj)
    # front 0: the three staircase points and the duplicate of (1, 5)
    assert list(r) == [0, 0, 0, 1, 1, 2, 0]
    rng = np.random.default_rng(0)
    obj = rng.integers(0, 4, size=(40, 3)).astype(float)
    r = gm.front_ranks(obj)
    for i in range(40):
        doms = [j for j in range(40) if np.all(obj[j] <= obj[i]) and np.any(obj[j] < obj[i])]
        # rank 0 iff nothing dominates it; otherwise one more than the highest rank among its dominators
        assert r[i] == (0 if not doms else 1 + max(r[j] for j in doms))


def test_selection_takes_whole_fronts_in_index_order():
    obj = np.array([[5, 5, 5], [1, 1, 1], [2, 2, 2], [1, 1, 1], [3, 3, 3]], float)
    assert list(gm.select(obj, 0.35)) == [1, 3]          # ceil(1.75) = 2: the two copies of the best
    assert list(gm.select(obj, 0.6)) == [1, 3, 2]
    assert list(gm.select(obj, 1.0)) == [1, 3, 2, 4, 0]


def test_normaliser():
    f = gm.normaliser([[1, 10, 5], [3, 30, 5]])
    assert f([2, 20, 5]) == [0.5, 0.5, 0.0]


def test_farthest_first_on_a_line():
    pts = [[float(x), 0.0, 0.0] for x in (3, 0, 10, 6, 1)]
    # first: smallest f_0 (x = 0, index 1); then the farthest (x = 10); then the
    # point farthest from both (x = 6 is 4 from 10, x = 3 is 3 from 0)
    assert gm.leaders(pts, 3) == [1, 2, 3]


def test_balanced_clusters_on_two_blobs():
    rng = np.random.default_rng(1)
    a = rng.normal(0, 0.01, size=(6, 3))
    b = rng.normal(0, 0.01, size=(6, 3)) + [1.0, 1.0, 1.0]
    pts = [list(map(float, p)) for p in np.concatenate([a, b])]
    # k = 4: clusters of ceil(2 * 12 / 4) = 6, each exactly one blob, both blobs used
    members, means = gm.balanced_kmeans(pts, 4)
    assert {tuple(m) for m in members} == {tuple(range(6)), tuple(range(6, 12))}
    for mem, m in zip(members, means):
        np.testing.assert_allclose(m, np.mean([pts[i] for i in mem], axis=0), rtol=0, atol=1e-15)
    # k = 2: clusters of 12, i.e. everything (the clusters overlap)
    members, _ = gm.balanced_kmeans(pts, 2)
    assert all(m == list(range(12)) for m in members)


def test_assignment_to_the_nearest_mean():
    means = [[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
    pts = [[0.2, 0, 0], [0.8, 0, 0], [0.5, 0, 0]]
    assert list(gm.assign(pts, means)) == [0, 1, 0]      # the tie goes to the lower cluster


def test_clusters_cover_the_population():
    rng = np.random.default_rng(2)
    obj = rng.random((50, 3))
    sel, members, pc = gm.clusters(obj, 0.35, 5)
    assert len(sel) == 18 and len(members) == 5
    assert all(len(m) == 8 for m in members)              # ceil(2 * 18 / 5)
    assert set(i for m in members for i in m) <= set(sel.tolist())
    assert pc.min() >= 0 and pc.max() < 5


def test_estimate_closed_form():
    # mu0 +- s e_j for every free variable j: mean mu0, covariance (s^2 / n_free) I
    mu0 = np.arange(12, dtype=float)
    free = np.ones(12, bool)
    free[[2, 8]] = False                                  # a point's z fixed on both meshes
    idx = np.nonzero(free)[0]
    s = 2.0
    rows = []
    for j in idx:
        for sign in (1, -1):
            r = mu0.copy()
            r[j] += sign * s
            rows.append(r)
    mu, L = gm.estimate(np.array(rows), free)
    np.testing.assert_allclose(mu, mu0, atol=1e-14)
    var = s * s / len(idx)
    want = np.zeros((12, 12))
    want[idx, idx] = math.sqrt(var + gm.RIDGE)
    np.testing.assert_allclose(L, want, atol=1e-12)


def test_sampling():
    mu = np.arange(12, dtype=float)
    L = np.diag(np.linspace(0.5, 1.6, 12))
    free = np.ones(12, bool)
    free[0] = False
    parent = np.full(12, -7.0)
    z = np.linspace(-1, 1, 12)
    x = gm.sample(mu, L, z, 2.0, parent, free)
    want = (mu + 2.0 * np.diag(L) * z).astype(np.float32)
    want[0] = -7.0
    np.testing.assert_array_equal(x, want)
    np.testing.assert_array_equal(gm.sample(mu, L, np.zeros(12), 3.0, parent, np.ones(12, bool)),
                                  mu.astype(np.float32))


def test_element_values_layout():
    src = np.arange(30, dtype=np.float32).reshape(10, 3)
    tgt = -src
    v = gm.element_values(src, tgt, 2, 7)
    np.testing.assert_array_equal(v, [6, 7, 8, 21, 22, 23, -6, -7, -8, -21, -22, -23])
    fx = np.zeros((10, 3), bool)
    fx[7, 1] = True
    assert list(np.nonzero(~gm.free_mask(fx, 2, 7))[0]) == [4, 10]


def test_steering_window():
    arch = np.array([[1, 1, 4.0], [2, 1, 2.0], [0.5, 3, 3.0], [0.1, 9, 3.01]])
    kept = gm.steer(arch, 1.5)
    np.testing.assert_array_equal(kept, arch[[1, 2]])
    assert gm.steering_window(np.array([2.0, 5.0])) == (2.0, 3.0)
