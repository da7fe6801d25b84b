"""Model building of MO-RV-GOMEA as MOREA uses it (Sec. 3; Sec. 4.3.2):
selection, clustering, per-cluster estimation and sampling of the FOS
elements' distributions, and adaptive steering.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain Python loops
over solutions and clusters; numpy only for small vector arithmetic.

The paper describes these steps in one paragraph each and refers to the
MO-RV-GOMEA literature for the rest; the readings below fix what it leaves
open.

Reading R19 (selection and clustering, Sec. 3):
  - Fronts: rank 0 is the non-dominated set of the population; rank r the
    non-dominated set of what remains after ranks < r are removed
    (minimisation; equal vectors are mutually non-dominated).
  - Selection: the ceil(tau n) solutions first in (rank, index) order.
  - Objective space: every objective is scaled by the range of the
    selection, (f - min) / (max - min) (a zero range maps to 0); distances
    are squared Euclidean in that space.
  - k leaders by farthest-first traversal: the first is the selected
    solution with the smallest normalised f_0 (lowest index on ties); each
    next is the selected solution farthest from its nearest leader (lowest
    index on ties).
  - Balanced k-means: every cluster holds the c = min(|S|, ceil(2 |S| / k))
    selected solutions nearest to its mean (ties by lower index); the means
    start at the leaders and are recomputed as the plain mean of the
    members, for at most `iters` iterations or until no membership changes.
    Clusters may overlap, so they are equally sized.
  - Every population member joins the cluster with the nearest mean (lowest
    cluster index on ties).

Reading R20 (estimation and sampling of a FOS element, Sec. 3): an element
(a, b) has 12 variables: source a (x, y, z), source b, target a, target b.
Variables whose axis is fixed for that point (points on the image box
faces) are not estimated and keep the parent's value.  Per cluster and
element: mu = the mean over the cluster's members (summed in member
order), Sigma = the maximum-likelihood covariance (1/n), L = the Cholesky
factor of Sigma + 1e-6 I (restricted to the free variables); a new value is
mu + c L z with z the caller's standard normal draws and c the cluster's
distribution multiplier, rounded to float.

Reading R21 (adaptive steering, Sec. 4.3.2): from the activation
generation on, only solutions with f_guidance in [s_G, factor * s_G] are
kept, s_G the best f_guidance in the elitist archive: the archive is
filtered and a candidate outside the window is not accepted.
"""

from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

RIDGE = 1e-6


def _dominates(a, b) -> bool:
    return all(x <= y for x, y in zip(a, b)) and any(x < y for x, y in zip(a, b))


def front_ranks(obj) -> np.ndarray:
    obj = [tuple(float(v) for v in row) for row in np.asarray(obj, np.float64)]
    n = len(obj)
    rank = [-1] * n
    left = set(range(n))
    r = 0
    while left:
        front = [i for i in sorted(left) if not any(_dominates(obj[j], obj[i]) for j in left if j != i)]
        for i in front:
            rank[i] = r
        left -= set(front)
        r += 1
    return np.array(rank, np.int32)


def select(obj, tau: float) -> np.ndarray:
    n = len(obj)
    ranks = front_ranks(obj)
    size = int(math.ceil(tau * n))
    order = sorted(range(n), key=lambda i: (int(ranks[i]), i))
    return np.array(order[:size], np.int32)


def normaliser(obj_sel):
    lo = [min(float(r[m]) for r in obj_sel) for m in range(3)]
    hi = [max(float(r[m]) for r in obj_sel) for m in range(3)]

    def f(o):
        out = []
        for m in range(3):
            span = hi[m] - lo[m]
            out.append((float(o[m]) - lo[m]) / span if span > 0 else 0.0)
        return out
    return f


def sqdist(a, b) -> float:
    d0, d1, d2 = a[0] - b[0], a[1] - b[1], a[2] - b[2]
    return (d0 * d0 + d1 * d1) + d2 * d2


def leaders(pts: List[List[float]], k: int) -> List[int]:
    first = min(range(len(pts)), key=lambda i: (pts[i][0], i))
    chosen = [first]
    near = [sqdist(p, pts[first]) for p in pts]
    while len(chosen) < min(k, len(pts)):
        nxt = max(range(len(pts)), key=lambda i: (near[i], -i))
        chosen.append(nxt)
        near = [min(near[i], sqdist(pts[i], pts[nxt])) for i in range(len(pts))]
    while len(chosen) < k:                       # more clusters than solutions: repeat
        chosen.append(chosen[len(chosen) % len(pts)])
    return chosen


def balanced_kmeans(pts: List[List[float]], k: int, iters: int = 10):
    """Cluster member lists (indices into pts, ascending) and their means."""
    n = len(pts)
    c = min(n, int(math.ceil(2 * n / k)))
    means = [list(pts[i]) for i in leaders(pts, k)]
    members = None
    for _ in range(max(1, iters)):
        new = []
        for m in means:
            order = sorted(range(n), key=lambda i: (sqdist(pts[i], m), i))
            new.append(sorted(order[:c]))
        if new == members:
            break
        members = new
        means = []
        for mem in members:
            s = [0.0, 0.0, 0.0]
            for i in mem:
                for a in range(3):
                    s[a] = s[a] + pts[i][a]
            means.append([s[a] / len(mem) for a in range(3)])
    return members, means


def assign(pts: List[List[float]], means) -> np.ndarray:
    return np.array([min(range(len(means)), key=lambda c: (sqdist(p, means[c]), c)) for p in pts], np.int32)


def clusters(obj, tau: float, k: int, iters: int = 10):
    """(selected indices, cluster member lists as population indices, the
    cluster of every population member)."""
    sel = select(obj, tau)
    norm = normaliser([obj[i] for i in sel])
    pts = [norm(obj[i]) for i in sel]
    members, means = balanced_kmeans(pts, k, iters)
    pop_cluster = assign([norm(o) for o in obj], means)
    return sel, [[int(sel[i]) for i in mem] for mem in members], pop_cluster


def element_values(src, tgt, a: int, b: int) -> np.ndarray:
    """The 12 variables of element (a, b) of one solution."""
    return np.concatenate([src[a], src[b], tgt[a], tgt[b]]).astype(np.float64)


def free_mask(fixed_axes, a: int, b: int) -> np.ndarray:
    f = np.asarray(fixed_axes, bool)
    return ~np.concatenate([f[a], f[b], f[a], f[b]])


def estimate(samples: np.ndarray, free: np.ndarray):
    """mu (12), Cholesky factor L (12 x 12, zero outside the free block)."""
    x = np.asarray(samples, np.float64)
    n = len(x)
    mu = np.zeros(12)
    for row in x:
        mu = mu + row
    mu = mu / n
    cov = np.zeros((12, 12))
    for row in x:
        d = row - mu
        cov = cov + np.outer(d, d)
    cov = cov / n
    idx = np.nonzero(free)[0]
    L = np.zeros((12, 12))
    if len(idx):
        sub = cov[np.ix_(idx, idx)] + RIDGE * np.eye(len(idx))
        L[np.ix_(idx, idx)] = np.linalg.cholesky(sub)
    return mu, L


def sample(mu, L, z, cmult: float, parent: np.ndarray, free: np.ndarray) -> np.ndarray:
    x = mu + cmult * (L @ np.asarray(z, np.float64))
    out = np.where(free, x, parent)
    return out.astype(np.float32)


def steering_window(guid: np.ndarray, factor: float = 1.5) -> Tuple[float, float]:
    s = float(np.min(guid))
    return s, factor * s


def steer(archive_obj: np.ndarray, factor: float = 1.5) -> np.ndarray:
    """The archive rows kept by adaptive steering (f_guidance is column 2)."""
    a = np.asarray(archive_obj, np.float64)
    if len(a) == 0:
        return a
    lo, hi = steering_window(a[:, 2], factor)
    return a[(a[:, 2] >= lo) & (a[:, 2] <= hi)]
