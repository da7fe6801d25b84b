"""Host logic of the optimiser: exact hypervolume against brute-force cell
counting, Pareto filtering and the archive's acceptance rule (Sec. 3)."""

import itertools

import numpy as np
import pytest

from paper_2303_04873_gb300 import ea


def brute_hv(points, ref):
    pts = np.asarray(points, float)
    coords = [np.unique(np.concatenate([pts[:, a][pts[:, a] < ref[a]], [ref[a]]])) for a in range(3)]
    vol = 0.0
    for i, j, k in itertools.product(*(range(len(c) - 1) for c in coords)):
        lo = np.array([coords[0][i], coords[1][j], coords[2][k]])
        hi = np.array([coords[0][i + 1], coords[1][j + 1], coords[2][k + 1]])
        if np.any(np.all(pts <= lo, axis=1)):
            vol += np.prod(hi - lo)
    return vol


@pytest.mark.parametrize("seed", range(8))
def test_hv3d_matches_cell_counting(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 13))
    pts = rng.integers(0, 6, size=(n, 3)).astype(float)       # ties and duplicates
    pts[0] = [7.0, 1.0, 1.0]                                    # outside the box in x
    ref = np.array([6.5, 6.0, 5.5])
    assert ea.hv3d(pts, ref) == pytest.approx(brute_hv(pts, ref), rel=1e-12, abs=1e-12)


def test_hv_closed_forms():
    assert ea.hv3d(np.array([[1.0, 2.0, 3.0]]), [4.0, 4.0, 4.0]) == pytest.approx(3 * 2 * 1)
    assert ea.hv2d(np.array([[0.0, 2.0], [1.0, 1.0]]), [3.0, 3.0]) == pytest.approx(3 * 1 + 2 * 1)
    assert ea.hv3d(np.zeros((0, 3)), [1, 1, 1]) == 0.0


def test_nondominated_and_archive():
    pts = np.array([[1, 2, 3], [2, 1, 3], [2, 2, 3], [1, 2, 3], [0, 5, 5]], float)
    nd = ea.nondominated(pts)
    assert {tuple(r) for r in nd} == {(1, 2, 3), (2, 1, 3), (0, 5, 5)}
    arc = ea.Archive()
    for p in pts:
        arc.add(p)
    assert {tuple(r) for r in arc.pts} == {(1, 2, 3), (2, 1, 3), (0, 5, 5)}
    assert not arc.accepts(np.array([1.0, 2.0, 3.0]))          # duplicate
    assert not arc.accepts(np.array([3.0, 3.0, 3.0]))          # dominated
    assert arc.accepts(np.array([0.5, 3.0, 3.0]))              # non-dominated
    assert ea.dominates(np.array([1, 1, 1]), np.array([1, 2, 1]))
    assert not ea.dominates(np.array([1, 1, 1]), np.array([1, 1, 1]))


def test_bfs_orders_are_connected_neighbourhoods():
    import synth
    p = synth.make_c0(n_sol=1)
    orders = ea.bfs_orders(p.tets, p.n_points, 12)
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    for v in (0, 31, 62, 124):
        o = orders[v]
        assert o[0] == v and len(set(o)) == 12
        for k in range(1, 12):                                # each vertex touches an earlier one
            assert any(int(u) in adj[int(o[k])] for u in o[:k])


@pytest.mark.parametrize("seed", range(4))
def test_acceptance_margin_sign_matches_the_acceptance_rule(seed):
    rng = np.random.default_rng(seed)
    arch = ea.Archive()
    for o in rng.integers(0, 8, size=(40, 3)).astype(float):
        arch.add(o)
    parents = rng.integers(0, 8, size=(300, 3)).astype(float)
    cand = rng.integers(0, 8, size=(300, 3)).astype(float)
    scale = np.array([1.0, 2.0, 0.5])
    m = ea.acceptance_margin(cand, parents, arch.pts, scale)
    for y, p, s in zip(cand, parents, m):
        kept = arch.accepts(y) or ea.dominates(y, p)
        strictly_better = bool(np.all(y < p))
        # negative score: kept by the archive test or better in every objective
        assert (s < 0) == (arch.accepts(y) or strictly_better)
        if s < 0:
            assert kept
    # scaling an objective's unit does not change the sign
    m2 = ea.acceptance_margin(cand * 3.0, parents * 3.0, arch.pts * 3.0, scale * 3.0)
    np.testing.assert_allclose(m2, m, rtol=1e-12)
    assert np.all(ea.acceptance_margin(cand, parents, np.zeros((0, 3)), scale) == -np.inf)


def test_crowding_distance_closed_form():
    pts = np.array([[0.0, 4.0, 1.0], [1.0, 2.0, 1.0], [3.0, 1.0, 1.0], [4.0, 0.0, 1.0]])
    d = ea.crowding(pts)
    assert np.isinf(d[0]) and np.isinf(d[3])
    # point 1: x neighbours 0 and 3 (range 4), y neighbours 1 and 4 (range 4), z constant
    np.testing.assert_allclose(d[1:3], [3 / 4 + 3 / 4, 3 / 4 + 2 / 4])


def test_archive_cap_keeps_extremes_and_non_dominance():
    rng = np.random.default_rng(9)
    arch = ea.Archive(cap=50)
    t = rng.uniform(0, np.pi / 2, size=(400, 2))
    front = np.stack([np.cos(t[:, 0]) * np.cos(t[:, 1]), np.sin(t[:, 0]) * np.cos(t[:, 1]), np.sin(t[:, 1])], 1)
    for o in front:
        arch.add(o)
    assert len(arch.pts) <= 50 + 50 // 4
    nd = ea.nondominated(arch.pts)
    assert len(nd) == len(arch.pts)
    # the per-objective minima of the whole front survive pruning
    for k in range(3):
        assert arch.pts[:, k].min() == pytest.approx(front[:, k].min())
