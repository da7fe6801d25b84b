"""A GOMEA-style optimiser on top of the evaluator, plain or surrogate-screened.

Host-side driver used to measure the surrogate pre-screen (not a hot path).
Each generation runs ``rounds`` optimal-mixing rounds: every solution gets one
linkage subset (a breadth-first mesh neighbourhood of 4-32 points, the
"dependent variables" of Sec. 4.2.1) moved by a Gaussian step on both
meshes; the partial solution is accepted if it dominates its parent or is
non-dominated with respect to the elitist archive, and is not folded (Sec. 3;
folded solutions are discarded, Sec. 4.3.1).  With a surrogate, all
candidates of a round are first scored by the network (the predicted change
of each objective, as the difference of the network's outputs for the
candidate and for its parent) and only the best ``screen`` fraction is
evaluated exactly; the rest are dropped unevaluated.

Hypervolume: exact 3-D, by sweeping the third objective over exact 2-D
staircase areas.
"""

from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np
import torch


# ---------------------------------------------------------------------------
# Pareto utilities
# ---------------------------------------------------------------------------

def dominates(a, b) -> bool:
    return bool(np.all(a <= b) and np.any(a < b))


def nondominated(points: np.ndarray) -> np.ndarray:
    """Rows of ``points`` not dominated by any other row (duplicates kept once)."""
    pts = np.unique(np.asarray(points, np.float64), axis=0)
    keep = np.ones(len(pts), bool)
    for i in range(len(pts)):
        if not keep[i]:
            continue
        dom = np.all(pts <= pts[i], axis=1) & np.any(pts < pts[i], axis=1)
        if dom.any():
            keep[i] = False
    return pts[keep]


def hv2d(xy: np.ndarray, ref) -> float:
    """Area dominated by points (minimisation) inside the box below ``ref``."""
    p = xy[(xy[:, 0] < ref[0]) & (xy[:, 1] < ref[1])]
    if len(p) == 0:
        return 0.0
    p = p[np.lexsort((p[:, 1], p[:, 0]))]
    # staircase: each point adds (ref_x - x) times how far it lowers the best y so far
    best_before = np.concatenate([[ref[1]], np.minimum.accumulate(p[:, 1])[:-1]])
    gain = np.maximum(best_before - p[:, 1], 0.0)
    return float(np.sum((ref[0] - p[:, 0]) * gain))


def hv3d(points: np.ndarray, ref) -> float:
    """Exact hypervolume of a 3-objective point set w.r.t. ``ref``."""
    p = np.asarray(points, np.float64)
    p = p[np.all(p < np.asarray(ref), axis=1)]
    if len(p) == 0:
        return 0.0
    p = p[np.argsort(p[:, 2], kind="stable")]
    vol = 0.0
    for i in range(len(p)):
        z_next = p[i + 1, 2] if i + 1 < len(p) else ref[2]
        if z_next > p[i, 2]:
            vol += hv2d(p[:i + 1, :2], ref) * (z_next - p[i, 2])
    return vol


def crowding(points: np.ndarray) -> np.ndarray:
    """Crowding distance of each point: the sum over objectives of the gap
    between its two neighbours in that objective, divided by the objective's
    range; the extremes of every objective get infinity."""
    n, m = points.shape
    d = np.zeros(n)
    for k in range(m):
        order = np.argsort(points[:, k], kind="stable")
        v = points[order, k]
        span = v[-1] - v[0]
        d[order[0]] = d[order[-1]] = np.inf
        if n > 2 and span > 0:
            d[order[1:-1]] += (v[2:] - v[:-2]) / span
    return d


class Archive:
    """Elitist archive of non-dominated objective vectors.

    Bounded by ``cap``: when it holds more than cap + cap // 4 points, the
    points with the smallest crowding distance are dropped (recomputed after
    each tenth of the excess) until cap remain, so the extremes and the
    spread of the front are kept.
    """

    def __init__(self, cap: int = 2000):
        self.cap = cap
        self.pts = np.zeros((0, 3))

    def accepts(self, o: np.ndarray) -> bool:
        """True if no archived point is at least as good as o in every objective."""
        if len(self.pts) == 0:
            return True
        le = np.all(self.pts <= o, axis=1)
        return not bool(np.any(le))

    def add(self, o: np.ndarray) -> bool:
        if not self.accepts(o):
            return False
        keep = ~(np.all(o <= self.pts, axis=1) & np.any(o < self.pts, axis=1))
        self.pts = np.vstack([self.pts[keep], o[None]])
        if len(self.pts) > self.cap + self.cap // 4:
            self.prune()
        return True

    def prune(self):
        step = max(1, (len(self.pts) - self.cap) // 10)
        while len(self.pts) > self.cap:
            k = min(step, len(self.pts) - self.cap)
            drop = np.argsort(crowding(self.pts), kind="stable")[:k]
            self.pts = np.delete(self.pts, drop, axis=0)


# ---------------------------------------------------------------------------
# the optimiser
# ---------------------------------------------------------------------------

def bfs_orders(tets: np.ndarray, n_points: int, depth: int = 32) -> np.ndarray:
    """For every vertex, the first ``depth`` vertices of a breadth-first walk over mesh edges."""
    adj = [set() for _ in range(n_points)]
    for t in tets:
        for a in t:
            for b in t:
                if a != b:
                    adj[int(a)].add(int(b))
    adj = [sorted(x) for x in adj]
    out = np.full((n_points, depth), -1, np.int32)
    for v in range(n_points):
        seen, head = [v], 0
        mark = {v}
        while len(seen) < depth and head < len(seen):
            for nb in adj[seen[head]]:
                if nb not in mark and len(seen) < depth:
                    mark.add(nb)
                    seen.append(nb)
            head += 1
        out[v, :len(seen)] = seen
    return out


def acceptance_margin(pred: np.ndarray, parent: np.ndarray, archive: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Predicted distance of each candidate from the acceptance test (lower is better).

    A candidate is kept if it dominates its parent or no archived point
    dominates it.  In units of ``scale`` per objective: max_k (y_k - p_k) is
    negative when y is better than the parent p in every objective, and the
    maximum over archived a of min_k (y_k - a_k) is negative exactly when no
    archived point is at least as good as y in every objective (the archive
    test).  The score is the smaller of the two, so the candidates that the
    network places deepest inside the acceptance region come first.
    """
    y = pred / scale
    m_parent = (y - parent / scale).max(axis=1)
    if len(archive) == 0:
        return np.full(len(y), -np.inf)
    a = archive / scale
    m_arch = (y[:, None, :] - a[None, :, :]).min(axis=2).max(axis=1)
    return np.minimum(m_parent, m_arch)


@dataclasses.dataclass
class Surrogate:
    """Trained network + the standardisation of its targets."""
    net: object
    mean: np.ndarray
    std: np.ndarray

    def predict(self, feats: torch.Tensor) -> np.ndarray:
        y = self.net.forward(feats).cpu().numpy().astype(np.float64)
        return y * self.std + self.mean


def run(gp, prob, generations: int, rounds: int, seed: int, step_scale: np.ndarray,
        surrogate: Optional[Surrogate] = None, screen: float = 0.25, ref: Optional[np.ndarray] = None,
        hv_every: int = 10, log: Optional[List] = None, orders: Optional[np.ndarray] = None,
        min_pts: int = 4, max_pts: int = 32, random_screen: bool = False, differential: bool = True,
        screen_rule: str = "sum") -> Dict:
    """Run the optimiser on the problem held by ``gp`` starting from ``prob``'s population.

    step_scale: per-vertex standard deviation of a move (voxels).
    differential: predict a candidate's objectives as its parent's exact
    objectives plus net(candidate) - net(parent) instead of net(candidate).
    screen_rule: "sum" ranks by the predicted sum of standardised objective
    changes (lowest first), "margin" by ``acceptance_margin``.
    random_screen: without a surrogate, evaluate a random ``screen`` fraction
    of the candidates (the same exact budget as the screened run, without the
    network's choice).  log: if a
    list is given, (features, objectives) of every exact partial evaluation
    are appended (features as a device tensor).  Returns the archive, the
    hypervolume history, and the number of exact evaluations.
    """
    dev = torch.device("cuda")
    rng = np.random.default_rng(seed)
    P, V = prob.n_solutions, prob.n_points
    if orders is None:
        orders = bfs_orders(prob.tets, V, max_pts)
    cur_s = prob.sol_src.astype(np.float32).copy()
    cur_t = prob.sol_tgt.astype(np.float32).copy()
    obj, folded, _ = gp.eval_full(torch.as_tensor(cur_s).to(dev), torch.as_tensor(cur_t).to(dev))
    obj = obj.cpu().numpy()
    folded = folded.cpu().numpy().astype(bool)
    if ref is None:
        ref = 1.1 * obj[~folded].max(axis=0)
    archive = Archive()
    for i in range(P):
        if not folded[i]:
            archive.add(obj[i])
    exact = P
    hist = [(0, exact, hv3d(archive.pts, ref))]
    slots_all = np.arange(P, dtype=np.int32)
    fixed = prob.fixed_axes
    for g in range(1, generations + 1):
        for _ in range(rounds):
            m = rng.integers(min_pts, max_pts + 1, size=P)
            seeds = rng.integers(0, V, size=P)
            ids = [np.sort(orders[seeds[i], :m[i]][orders[seeds[i], :m[i]] >= 0]) for i in range(P)]
            off = np.zeros(P + 1, np.int32)
            off[1:] = np.cumsum([len(x) for x in ids])
            pts = np.concatenate(ids).astype(np.int32)
            owner = np.repeat(slots_all, np.diff(off))
            step = step_scale[pts][:, None, None] * rng.normal(size=(len(pts), 2, 3))
            step[fixed[pts][:, None, :].repeat(2, axis=1)] = 0.0
            new_s = (cur_s[owner, pts] + step[:, 0]).astype(np.float32)
            new_t = (cur_t[owner, pts] + step[:, 1]).astype(np.float32)
            chosen = slots_all
            feats = None
            if surrogate is not None or log is not None:
                dv = [torch.as_tensor(a).to(dev) for a in (slots_all, off, pts, new_s, new_t)]
                feats = gp.partial_features(*dv)
            if surrogate is not None:
                if differential:
                    # the parent's own field through the same network: its
                    # error is shared by parent and candidate and cancels
                    dv = [torch.as_tensor(a).to(dev) for a in (slots_all, off, pts, cur_s[owner, pts],
                                                               cur_t[owner, pts])]
                    pred = obj + surrogate.predict(feats) - surrogate.predict(gp.partial_features(*dv))
                else:
                    pred = surrogate.predict(feats)
                if screen_rule == "margin":
                    score = acceptance_margin(pred, obj, archive.pts, surrogate.std)
                else:
                    score = ((pred - obj) / surrogate.std).sum(axis=1)
                k = max(1, int(round(screen * P)))
                chosen = np.sort(np.argsort(score, kind="stable")[:k]).astype(np.int32)
            elif random_screen:
                k = max(1, int(round(screen * P)))
                chosen = np.sort(rng.choice(P, size=k, replace=False)).astype(np.int32)
            # exact partial evaluation of the chosen candidates
            sub_off = np.zeros(len(chosen) + 1, np.int32)
            sub_off[1:] = np.cumsum(np.diff(off)[chosen])
            sel = np.concatenate([np.arange(off[i], off[i + 1]) for i in chosen])
            args = [torch.as_tensor(a).to(dev) for a in (chosen.astype(np.int32), sub_off, pts[sel], new_s[sel],
                                                         new_t[sel])]
            o, f, _ = gp.eval_partial(*args)
            o = o.cpu().numpy()
            f = f.cpu().numpy().astype(bool)
            exact += len(chosen)
            if log is not None:
                log.append((feats[torch.as_tensor(chosen).to(dev).long()].clone(), o.copy()))
            acc = np.zeros(len(chosen), np.uint8)
            for j, i in enumerate(chosen):
                if f[j] or not np.all(np.isfinite(o[j])):
                    continue
                if dominates(o[j], obj[i]) or archive.accepts(o[j]):
                    acc[j] = 1
                    archive.add(o[j])
                    obj[i] = o[j]
                    a, b = off[i], off[i + 1]
                    cur_s[i, pts[a:b]] = new_s[a:b]
                    cur_t[i, pts[a:b]] = new_t[a:b]
            gp.commit_partial(torch.as_tensor(acc).to(dev))
        if g % hv_every == 0 or g == generations:
            hist.append((g, exact, hv3d(archive.pts, ref)))
    return {"archive": archive.pts, "history": hist, "exact": exact, "ref": ref, "hv": hist[-1][2],
            "objectives": obj}


def train_surrogate(net, feats: torch.Tensor, targets: np.ndarray, epochs: int = 20, lr: float = 1e-3,
                    holdout: float = 0.1, seed: int = 0) -> Dict:
    """Fit ``net`` (morea.Mlp) on standardised targets; MAE and R^2 per objective on a held-out split."""
    n = int(feats.shape[0])
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    n_val = max(1, int(holdout * n))
    val, tr = perm[:n_val], perm[n_val:]
    mean = targets[tr].mean(axis=0)
    std = targets[tr].std(axis=0) + 1e-12
    T = torch.as_tensor(((targets - mean) / std).astype(np.float32)).cuda()
    bs = net.max_batch
    tr_t = torch.as_tensor(tr).cuda()
    for ep in range(epochs):
        order = tr_t[torch.randperm(len(tr), generator=torch.Generator().manual_seed(seed + ep)).cuda()]
        for a in range(0, len(tr) - bs + 1, bs):
            idx = order[a:a + bs]
            net.train_step(feats[idx].contiguous(), T[idx].contiguous(), lr)
    val_t = torch.as_tensor(val).cuda()
    pred = net.forward(feats[val_t].contiguous()).cpu().numpy() * std + mean
    truth = targets[val]
    mae = np.abs(pred - truth).mean(axis=0)
    r2 = 1.0 - ((pred - truth) ** 2).sum(axis=0) / ((truth - truth.mean(axis=0)) ** 2).sum(axis=0)
    return {"surrogate": Surrogate(net, mean, std), "mae": mae, "r2": r2, "n_train": len(tr), "n_val": n_val}
