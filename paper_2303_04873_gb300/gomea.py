"""MO-RV-GOMEA generations as MOREA runs them (Sec. 3, Sec. 4.2-4.3), driven
from the host over the library's device calls.

A generation:
  1. selection and balanced clustering of the population in objective space
     (``morea.cluster``, host);
  2. for every parallel group of FOS elements (mesh edges from a greedy set
     cover, coloured by DSATUR, ``morea.parallel_groups``): one request per
     (solution, element of the group), drawn from the distribution of that
     element in the solution's cluster (``Problem.sample_elements``,
     device), all evaluated by one batched partial evaluation (device);
  3. a request is accepted if its partial solution is unfolded and dominates
     its parent or is not dominated by the elitist archive (Sec. 3); under
     adaptive steering its f_guidance must also stay within the window
     (Sec. 4.3.2); accepted requests are committed (device) and the
     solutions' objectives re-read from the committed totals (device);
  4. with repair on (the paper's configuration), after each group's commit
     every solution's first folded candidate of the group is repaired
     (Sec. 4.3.1; reading R20): rebuilt on the solution as committed,
     repaired with ``Problem.repair_folds`` (one call per group), and, if
     the repair (which keeps the fixed axes) leaves it unfolded,
     re-evaluated as a partial request over every point that differs from
     the solution and accepted by the same rule;
  5. the archive takes the new solutions; the distribution multiplier of a
     cluster grows by 10 % after a generation with an accepted request of
     that cluster and shrinks by 10 % otherwise, within [0.1, 10]
     (reading R20); from the steering generation on the archive keeps only
     f_guidance in [s_G, factor s_G] (reading R21).

The initial population comes from ``Problem.init_noise`` (Sec. 4.2.2).
Without repair, folded candidates are discarded (Sec. 4.3.1).

Optional learned pre-screen (not in the paper): with a ``surrogate``
(``ea.Surrogate``) only the ``screen`` fraction of each group's requests
with the best predicted change -- net(candidate) - net(parent), summed over
objectives in units of the training targets' standard deviation, lowest
first (reading R11) -- is evaluated exactly; the others count as rejected.
``random_screen`` evaluates a random fraction of the same size instead.
``log`` collects (features, objectives) of up to ``log_per_group`` exactly
evaluated requests per group, for training a surrogate.
"""

from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import morea
from .ea import Archive, hv3d


@dataclasses.dataclass
class GomeaConfig:
    tau: float = 0.35                # selection fraction
    clusters: int = 10               # the paper's runs use 10 clusters
    kmeans_iters: int = 10
    archive_cap: int = 2000          # the paper's archive capacity
    steer_at: int = 100              # adaptive steering from this generation on
    steer_factor: float = 1.5
    cmult0: float = 1.0
    init_kernels: int = 8            # Gaussian kernels per mesh for the initial noise
    init_rounds: int = 50
    init_sigma: tuple = (8.0, 24.0)
    init_strength: tuple = (0.02, 0.15)
    repair: bool = True              # the paper's runs repair folded candidates
    repair_points: int = 16          # repair visits per candidate


def fixed_bits(fixed_axes: np.ndarray) -> np.ndarray:
    f = np.asarray(fixed_axes, bool).astype(np.uint8)
    return (f[:, 0] | (f[:, 1] << 1) | (f[:, 2] << 2)).astype(np.uint8)


def max_changed(cfg: Optional[GomeaConfig] = None) -> int:
    """The changed-point capacity a Problem needs for Gomea: the two points of
    an element, plus one per repair visit."""
    cfg = cfg or GomeaConfig()
    return 2 + (cfg.repair_points if cfg.repair else 0)


def max_requests(prob, n_pop: int) -> int:
    """The request capacity a Problem needs for Gomea: one request per
    (solution, element) of the largest parallel group."""
    _, grp = morea.parallel_groups(prob.n_points, prob.tets)
    return int(n_pop) * int(np.bincount(grp).max())


class Gomea:
    """``gp`` must hold at least n_pop slots, max_requests(prob, n_pop)
    requests and max_changed(cfg) changed points per request."""

    def __init__(self, gp: "morea.Problem", prob, n_pop: int, cfg: Optional[GomeaConfig] = None, seed: int = 0,
                 start_src: Optional[np.ndarray] = None, start_tgt: Optional[np.ndarray] = None,
                 surrogate=None, screen: float = 0.25, random_screen: bool = False, log: Optional[list] = None,
                 log_per_group: int = 128):
        self.gp, self.cfg = gp, cfg or GomeaConfig()
        self.surrogate, self.screen, self.random_screen = surrogate, float(screen), bool(random_screen)
        self.log, self.log_per_group = log, int(log_per_group)
        self.exact = 0                   # exact evaluations (requests, repaired candidates, the initial population)
        self.rng = np.random.default_rng(seed)
        self.dev_rng = torch.Generator(device="cuda")     # the repair's trial draws
        self.dev_rng.manual_seed(int(seed))
        self.dev = torch.device("cuda")
        self.n, self.V = int(n_pop), prob.n_points
        el, grp = morea.parallel_groups(prob.n_points, prob.tets)
        self.elements = torch.as_tensor(el).to(self.dev).contiguous()
        self.el_host = el
        self.groups = [np.nonzero(grp == g)[0].astype(np.int32) for g in range(int(grp.max()) + 1)]
        # each group's element pairs on the device: the models are estimated per group
        self.group_el = [torch.as_tensor(el[g]).to(self.dev).contiguous() for g in self.groups]
        self.fixed = torch.as_tensor(fixed_bits(prob.fixed_axes)).to(self.dev)
        # initial population: the reference mesh with Gaussian-attraction noise
        if start_src is None:
            ref = np.broadcast_to(prob.ref_points.astype(np.float32), (self.n, self.V, 3)).copy()
            S = torch.as_tensor(ref).to(self.dev)
            T = S.clone()
            c = self.cfg
            box = np.array([prob.nx, prob.ny, prob.nz], np.float64) - 1
            K = c.init_kernels
            ker = np.concatenate([self.rng.uniform(0, 1, (self.n, 2, K, 3)) * box,
                                  self.rng.uniform(*c.init_sigma, (self.n, 2, K, 1)),
                                  self.rng.uniform(*c.init_strength, (self.n, 2, K, 1))], -1).astype(np.float32)
            gp.init_noise(S, T, torch.as_tensor(ker).to(self.dev), c.init_rounds, fixed=self.fixed)
        else:
            S = torch.as_tensor(np.ascontiguousarray(start_src, np.float32)).to(self.dev)
            T = torch.as_tensor(np.ascontiguousarray(start_tgt, np.float32)).to(self.dev)
        self.S, self.T = S, T
        obj, folded, _ = gp.eval_full(S, T)
        self.exact += self.n
        self.obj = obj.cpu().numpy()
        self.folded = folded.cpu().numpy().astype(bool)
        self.archive = Archive(self.cfg.archive_cap)
        for i in range(self.n):
            if not self.folded[i]:
                self.archive.add(self.obj[i])
        self.cmult = np.full(self.cfg.clusters, self.cfg.cmult0, np.float64)
        self.generation_index = 0
        self.requests = 0
        self.accepted = 0
        self.repair_calls = 0            # groups whose folded candidates went through the repair
        self.repaired = 0                # repaired candidates re-evaluated
        self.repaired_accepted = 0
        biggest = max(len(g) for g in self.groups)
        self.work = torch.empty((morea.sample_elements_workspace(self.cfg.clusters, biggest),), dtype=torch.uint8,
                                device=self.dev)

    def steering(self) -> bool:
        return self.generation_index >= self.cfg.steer_at

    def window_hi(self) -> float:
        if len(self.archive.pts) == 0:
            return np.inf
        return self.cfg.steer_factor * float(self.archive.pts[:, 2].min())

    def _archive_accepts(self, o: np.ndarray, chunk: int = 2048) -> np.ndarray:
        """Per row of o: no archived point is at least as good in every objective."""
        a = self.archive.pts
        out = np.ones(len(o), bool)
        if len(a) == 0:
            return out
        for s in range(0, len(o), chunk):
            out[s:s + chunk] = ~np.any(np.all(a[None, :, :] <= o[s:s + chunk, None, :], axis=2), axis=1)
        return out

    def _refresh(self, changed: np.ndarray):
        """Re-read the committed objectives of the changed solutions and offer
        them to the archive."""
        if len(changed) == 0:
            return
        obj, _, _ = self.gp.slot_objectives(self.n)
        obj = obj.cpu().numpy()
        for i in changed:
            self.obj[i] = obj[i]
            self.archive.add(self.obj[i])

    def _accept(self, o: np.ndarray, f: np.ndarray, sol: np.ndarray, hi: float) -> np.ndarray:
        ok = ~f & np.all(np.isfinite(o), axis=1) & (o[:, 2] <= hi)
        par = self.obj[sol]
        better = np.all(o <= par, axis=1) & np.any(o < par, axis=1)
        return ok & (better | self._archive_accepts(o))

    def _repair(self, sols: np.ndarray, ab: torch.Tensor, cs2: torch.Tensor, ct2: torch.Tensor, hi: float):
        """Repair one folded candidate per solution ``sols`` (element points ab
        [k][2], their coordinates cs2 / ct2 [k][2][3]), then evaluate, accept
        and commit the repaired candidates.  Returns the solutions changed
        and the numbers re-evaluated and accepted."""
        c = self.cfg
        k = len(sols)
        sol_d = torch.as_tensor(sols).to(self.dev).long()
        Cs, Ct = self.S[sol_d].clone(), self.T[sol_d].clone()
        ar = torch.arange(k, device=self.dev)
        for j in range(2):
            Cs[ar, ab[:, j]] = cs2[:, j]
            Ct[ar, ab[:, j]] = ct2[:, j]
        self.repair_calls += 1
        noise = torch.randn((k, c.repair_points, 64, 3), generator=self.dev_rng, device=self.dev)
        self.gp.repair_folds(Cs, Ct, noise, c.repair_points, fixed=self.fixed)
        folded, _ = self.gp.check_folds(Cs, Ct)          # a degenerate tet is folded without severity
        diff = ((Cs != self.S[sol_d]) | (Ct != self.T[sol_d])).any(dim=2)
        n_diff = diff.sum(dim=1)
        good = (folded == 0) & (n_diff > 0) & (n_diff <= self.gp.max_changed)
        keep = np.nonzero(good.cpu().numpy())[0]
        if len(keep) == 0:
            return np.zeros(0, np.int64), 0, 0
        keep_d = torch.as_tensor(keep).to(self.dev)
        sub = diff[keep_d]
        qi, pi = torch.nonzero(sub, as_tuple=True)           # (candidate, point), candidate-major
        counts = sub.sum(dim=1).cpu().numpy()
        off = np.zeros(len(keep) + 1, np.int32)
        off[1:] = np.cumsum(counts)
        own = keep_d[qi]
        cs, ct = Cs[own, pi].contiguous(), Ct[own, pi].contiguous()
        slots = sol_d[keep_d].int()
        o, f, _ = self.gp.eval_partial(slots, torch.as_tensor(off).to(self.dev), pi.int().contiguous(), cs, ct)
        o = o.cpu().numpy()
        f = f.cpu().numpy().astype(bool)
        acc = self._accept(o, f, sols[keep], hi).astype(np.uint8)
        self.gp.commit_partial(torch.as_tensor(acc).to(self.dev))
        if acc.any():
            sel = torch.as_tensor(np.repeat(acc, counts).astype(bool)).to(self.dev)
            self.S[sol_d[own[sel]], pi[sel]] = cs[sel]
            self.T[sol_d[own[sel]], pi[sel]] = ct[sel]
        return sols[keep][acc.astype(bool)], len(keep), int(acc.sum())

    def _features(self, sol: torch.Tensor, pts: torch.Tensor, cs: torch.Tensor, ct: torch.Tensor,
                  chunk: int = 4096) -> list:
        """Displacement features of two-point requests (solution sol[r], points
        pts[2r:2r+2] moved to cs / ct), in chunks of `chunk` requests."""
        out = []
        n = int(sol.shape[0])
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            off = torch.arange(0, 2 * (b - a) + 1, 2, dtype=torch.int32, device=self.dev)
            out.append(self.gp.partial_features(sol[a:b].int().contiguous(), off, pts[2 * a:2 * b].contiguous(),
                                                cs[2 * a:2 * b].contiguous(), ct[2 * a:2 * b].contiguous()))
        return out

    def _screen(self, d, gel, new_s, new_t, n_req: int) -> np.ndarray:
        """Indices of the requests to evaluate exactly (all without a screen)."""
        if self.surrogate is None and not self.random_screen:
            return np.arange(n_req)
        k = max(1, int(round(self.screen * n_req)))
        if self.surrogate is None:
            return np.sort(self.rng.choice(n_req, size=k, replace=False))
        sur = self.surrogate
        # each solution's own field through the network (its committed slot; the
        # "change" of one point to its current value leaves it as it is)
        sol_all = torch.arange(self.n, dtype=torch.int32, device=self.dev)
        off1 = torch.arange(0, self.n + 1, dtype=torch.int32, device=self.dev)
        p0 = torch.zeros(self.n, dtype=torch.int32, device=self.dev)
        parent = sur.predict(self.gp.partial_features(sol_all, off1, p0, self.S[:, 0].contiguous(),
                                                      self.T[:, 0].contiguous()))
        pts = gel[d[2].long()].reshape(-1)
        cand = np.concatenate([sur.predict(f) for f in self._features(d[0], pts, new_s, new_t)])
        req_sol = d[0].cpu().numpy()
        score = ((cand - parent[req_sol]) / sur.std).sum(axis=1)
        return np.sort(np.argsort(score, kind="stable")[:k])

    def step(self) -> dict:
        """One generation; returns its counts."""
        c = self.cfg
        _, members, pop_cluster = morea.cluster(self.obj, c.tau, c.clusters, c.kmeans_iters)
        mem_d = torch.as_tensor(members).to(self.dev).contiguous()
        cm_d = torch.as_tensor(self.cmult.astype(np.float32)).to(self.dev)
        hit = np.zeros(c.clusters, bool)
        n_req_total = n_acc_total = 0
        steer = self.steering()
        for grp, gel in zip(self.groups, self.group_el):
            m = len(grp)
            req_sol = np.repeat(np.arange(self.n, dtype=np.int32), m)
            req_el = np.tile(np.arange(m, dtype=np.int32), self.n)          # index into this group's elements
            req_cl = pop_cluster[req_sol].astype(np.int32)
            n_req = len(req_sol)
            z = self.rng.standard_normal((n_req, 12)).astype(np.float32)
            d = [torch.as_tensor(a).to(self.dev) for a in (req_sol, req_cl, req_el, z)]
            new_s, new_t = self.gp.sample_elements(self.S, self.T, mem_d, gel, cm_d, d[0], d[1], d[2], d[3],
                                                   fixed=self.fixed, work=self.work)
            chosen = self._screen(d, gel, new_s, new_t, n_req)
            if len(chosen) < n_req:          # only the screened requests are evaluated exactly
                ch = torch.as_tensor(chosen).to(self.dev)
                rows2 = torch.stack([2 * ch, 2 * ch + 1], 1).reshape(-1)
                d = [x[ch] for x in d]
                new_s, new_t = new_s[rows2].contiguous(), new_t[rows2].contiguous()
                req_sol, req_el, req_cl = req_sol[chosen], req_el[chosen], req_cl[chosen]
                n_req = len(chosen)
            off = torch.arange(0, 2 * n_req + 1, 2, dtype=torch.int32, device=self.dev)
            pts = gel[d[2].long()].reshape(-1).contiguous()
            o, f, _ = self.gp.eval_partial(d[0], off, pts, new_s, new_t)
            self.exact += n_req
            o = o.cpu().numpy()
            f = f.cpu().numpy().astype(bool)
            if self.log is not None:         # a sample of this group's exact evaluations, before the commit
                okr = np.nonzero(np.all(np.isfinite(o), axis=1))[0]
                take = np.sort(self.rng.choice(okr, size=min(self.log_per_group, len(okr)), replace=False))
                if len(take):
                    tk = torch.as_tensor(take).to(self.dev)
                    rows2 = torch.stack([2 * tk, 2 * tk + 1], 1).reshape(-1)
                    fe = self._features(d[0][tk], pts[rows2], new_s[rows2], new_t[rows2])
                    self.log.append((torch.cat(fe), o[take].copy()))
            hi = self.window_hi() if steer else np.inf
            acc = self._accept(o, f, req_sol, hi).astype(np.uint8)
            self.gp.commit_partial(torch.as_tensor(acc).to(self.dev))
            changed = np.unique(req_sol[acc.astype(bool)])
            if acc.any():
                rows = torch.as_tensor(np.nonzero(acc)[0]).to(self.dev)
                sol = d[0][rows].long()
                ab = gel[d[2][rows].long()].long()
                for j in range(2):
                    self.S[sol, ab[:, j]] = new_s.view(n_req, 2, 3)[rows, j]
                    self.T[sol, ab[:, j]] = new_t.view(n_req, 2, 3)[rows, j]
                hit[np.unique(req_cl[acc.astype(bool)])] = True
            n_acc = int(acc.sum())
            self._refresh(changed)
            fr = np.nonzero(f & np.all(np.isfinite(o), axis=1))[0]
            if c.repair and len(fr):
                fs, first = np.unique(req_sol[fr], return_index=True)      # each solution's first folded one
                rows_d = torch.as_tensor(fr[first]).to(self.dev).long()
                rsol, n_rep, n_racc = self._repair(fs, gel[d[2][rows_d].long()].long(),
                                                   new_s.view(n_req, 2, 3)[rows_d], new_t.view(n_req, 2, 3)[rows_d],
                                                   self.window_hi() if steer else np.inf)
                self._refresh(rsol)
                if n_racc:
                    hit[np.unique(pop_cluster[rsol])] = True
                self.repaired += n_rep
                self.repaired_accepted += n_racc
                self.exact += n_rep
                n_acc += n_racc
            n_req_total += n_req
            n_acc_total += n_acc
        self.cmult = np.where(hit, np.minimum(self.cmult * 1.1, 10.0), np.maximum(self.cmult * 0.9, 0.1))
        self.generation_index += 1
        if self.steering() and len(self.archive.pts):
            pts = self.archive.pts
            s_g = float(pts[:, 2].min())
            self.archive.pts = pts[pts[:, 2] <= c.steer_factor * s_g]
        self.requests += n_req_total
        self.accepted += n_acc_total
        return {"requests": n_req_total, "accepted": n_acc_total, "repaired": self.repaired,
                "repaired_accepted": self.repaired_accepted}

    def hypervolume(self, ref) -> float:
        return hv3d(self.archive.pts, ref)
