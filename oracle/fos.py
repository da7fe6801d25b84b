"""Linkage model and parallel groups of the partial evaluations (Sec. 4.2.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain Python loops.

Reading R16 (the paper names the algorithms, not their tie rules):
  - FOS elements are mesh edges: unordered point pairs (a < b) that share a
    tet, sorted lexicographically.
  - Greedy set cover of the points by edges: repeatedly take the edge that
    covers the most still-uncovered points, the first in sorted order on
    ties, until every point is covered.
  - The dependent tets of an element are the tets that contain one of its
    points (the tets a partial evaluation of that element re-evaluates).
  - Two elements interact when their dependent tets overlap.
  - DSATUR colouring of the interaction graph (Brelaz 1979): repeatedly
    colour the uncoloured element with the most distinct colours among its
    neighbours, then the largest degree, then the lowest index, with the
    smallest colour no neighbour has.  Elements of one colour (a parallel
    group) have disjoint dependent tets and can be evaluated together.
Elements are numbered in the order the set cover takes them.
"""

from __future__ import annotations

from typing import List, Tuple

import numpy as np


def mesh_edges(tets) -> List[Tuple[int, int]]:
    edges = set()
    for t in np.asarray(tets):
        for i in range(4):
            for j in range(i + 1, 4):
                a, b = int(t[i]), int(t[j])
                edges.add((min(a, b), max(a, b)))
    return sorted(edges)


def greedy_set_cover(n_points: int, edges) -> List[Tuple[int, int]]:
    covered = [False] * n_points
    left = n_points
    chosen = []
    while left > 0:
        best, best_gain = None, 0
        for e in edges:
            gain = (not covered[e[0]]) + (not covered[e[1]])
            if gain > best_gain:
                best, best_gain = e, gain
                if gain == 2:
                    break
        if best is None:
            raise ValueError("a point belongs to no edge")
        chosen.append(best)
        for v in best:
            if not covered[v]:
                covered[v] = True
                left -= 1
    return chosen


def dependent_tets(tets, elements) -> List[set]:
    star = {}
    for t, tv in enumerate(np.asarray(tets)):
        for v in tv:
            star.setdefault(int(v), set()).add(t)
    return [star.get(a, set()) | star.get(b, set()) for a, b in elements]


def interaction_graph(dep) -> List[set]:
    n = len(dep)
    adj = [set() for _ in range(n)]
    for i in range(n):
        for j in range(i + 1, n):
            if dep[i] & dep[j]:
                adj[i].add(j)
                adj[j].add(i)
    return adj


def dsatur(adj) -> List[int]:
    n = len(adj)
    color = [-1] * n
    for _ in range(n):
        best, key = -1, None
        for v in range(n):
            if color[v] >= 0:
                continue
            sat = len({color[u] for u in adj[v] if color[u] >= 0})
            k = (sat, len(adj[v]), -v)
            if key is None or k > key:
                best, key = v, k
        used = {color[u] for u in adj[best] if color[u] >= 0}
        c = 0
        while c in used:
            c += 1
        color[best] = c
    return color


def parallel_groups(n_points: int, tets):
    """(elements [m][2], group id per element) of the edge FOS."""
    elements = greedy_set_cover(n_points, mesh_edges(tets))
    groups = dsatur(interaction_graph(dependent_tets(tets, elements)))
    return np.array(elements, np.int32).reshape(-1, 2), np.array(groups, np.int32)
