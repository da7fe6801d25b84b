"""Pins of the linkage model and parallel groups (reading R16, Sec. 4.2.1).

Greedy set cover and DSATUR are checked by hand on tiny instances, against
known chromatic numbers (DSATUR is exact on bipartite graphs, cycles,
complete graphs and wheels), and by validity on meshes: every point is
covered, and the elements of a group never share a dependent tet."""

import numpy as np
import pytest

import synth
from oracle import fos


def test_edges_of_one_tet():
    assert fos.mesh_edges([[3, 1, 2, 0]]) == [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def test_set_cover_by_hand():
    path = [(0, 1), (1, 2), (2, 3), (3, 4)]
    # (0,1) and (2,3) cover two new points each; 4 is then covered by (3,4)
    assert fos.greedy_set_cover(5, path) == [(0, 1), (2, 3), (3, 4)]
    star = [(0, 1), (0, 2), (0, 3)]
    assert fos.greedy_set_cover(4, star) == [(0, 1), (0, 2), (0, 3)]
    with pytest.raises(ValueError):
        fos.greedy_set_cover(3, [(0, 1)])


def _cycle(n):
    return [{(i - 1) % n, (i + 1) % n} for i in range(n)]


@pytest.mark.parametrize("n,colors", [(6, 2), (8, 2), (5, 3), (7, 3)])
def test_dsatur_on_cycles(n, colors):
    c = fos.dsatur(_cycle(n))
    assert max(c) + 1 == colors
    assert all(c[i] != c[(i + 1) % n] for i in range(n))


def test_dsatur_on_complete_bipartite_and_wheel_graphs():
    k5 = [set(range(5)) - {i} for i in range(5)]
    assert sorted(fos.dsatur(k5)) == [0, 1, 2, 3, 4]
    # complete bipartite K(3,4): 2 colours
    kb = [set(range(3, 7)) for _ in range(3)] + [set(range(3)) for _ in range(4)]
    c = fos.dsatur(kb)
    assert max(c) + 1 == 2 and len({c[i] for i in range(3)}) == 1
    # wheels: hub + rim cycle; even rim -> 3 colours, odd rim -> 4
    for rim, want in ((6, 3), (5, 4)):
        adj = [set(range(1, rim + 1))] + [{0, 1 + (i - 1) % rim, 1 + (i + 1) % rim} for i in range(rim)]
        assert max(fos.dsatur(adj)) + 1 == want
    # a grid graph is bipartite: 2 colours
    w, h = 4, 3
    adj = [set() for _ in range(w * h)]
    for y in range(h):
        for x in range(w):
            i = y * w + x
            if x + 1 < w:
                adj[i].add(i + 1); adj[i + 1].add(i)
            if y + 1 < h:
                adj[i].add(i + w); adj[i + w].add(i)
    assert max(fos.dsatur(adj)) + 1 == 2


def test_first_choice_follows_the_tie_rules():
    # star K(1,3) plus an isolated vertex: the hub (degree 3) is coloured first with 0
    adj = [{1, 2, 3}, {0}, {0}, {0}, set()]
    assert fos.dsatur(adj) == [0, 1, 1, 1, 0]


def test_groups_on_the_mesh_are_valid():
    p = synth.make_c0(n_sol=1)
    el, grp = fos.parallel_groups(p.n_points, p.tets)
    covered = np.zeros(p.n_points, bool)
    covered[el.ravel()] = True
    assert covered.all()
    dep = fos.dependent_tets(p.tets, [tuple(e) for e in el])
    for g in range(grp.max() + 1):
        members = np.nonzero(grp == g)[0]
        seen = set()
        for m in members:
            assert not (dep[m] & seen)
            seen |= dep[m]
    # every element is a mesh edge
    edges = set(fos.mesh_edges(p.tets))
    assert all((int(a), int(b)) in edges for a, b in el)
