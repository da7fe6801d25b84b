"""MO-RV-GOMEA model building and generations on the GPU (readings
R19-R21, Sec. 3 and Sec. 4.3.2).

Sampled FOS elements against the oracle's estimate and draw (within one
float ulp: both sides compute in FP64, the oracle's Cholesky and matrix
product round in a different order), objectives of committed slots
against evaluations, and short generations checked by their invariants."""

import numpy as np
import pytest
import torch

import synth
from oracle import gomea as gm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def fixed_bits(fa):
    f = fa.astype(np.uint8)
    return (f[:, 0] | (f[:, 1] << 1) | (f[:, 2] << 2)).astype(np.uint8)


@pytest.mark.parametrize("seed", range(3))
def test_sampled_elements_match_the_oracle(mo, seed):
    p = synth.make_c0(n_sol=12)
    rng = np.random.default_rng(seed)
    n = p.n_solutions
    obj = rng.random((n, 3))
    k = 3
    _, members, pc = mo.cluster(obj, 0.6, k)
    el, _ = mo.parallel_groups(p.n_points, p.tets)
    n_req = 40
    req_sol = rng.integers(0, n, n_req).astype(np.int32)
    req_el = rng.integers(0, len(el), n_req).astype(np.int32)
    req_cl = pc[req_sol].astype(np.int32)
    z = rng.standard_normal((n_req, 12)).astype(np.float32)
    cmult = rng.uniform(0.5, 2.0, k).astype(np.float32)
    gp = mo.Problem(p, max_solutions=1)
    dv = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    new_s, new_t = gp.sample_elements(dv(p.sol_src), dv(p.sol_tgt), dv(members), dv(el), dv(cmult), dv(req_sol),
                                      dv(req_cl), dv(req_el), dv(z), fixed=dv(fixed_bits(p.fixed_axes)))
    got = np.concatenate([new_s.cpu().numpy().reshape(n_req, 6), new_t.cpu().numpy().reshape(n_req, 6)], 1)
    for r in range(n_req):
        a, b = el[req_el[r]]
        c = req_cl[r]
        vals = np.array([gm.element_values(p.sol_src[i], p.sol_tgt[i], a, b) for i in members[c]])
        free = gm.free_mask(p.fixed_axes, a, b)
        mu, L = gm.estimate(vals, free)
        parent = gm.element_values(p.sol_src[req_sol[r]], p.sol_tgt[req_sol[r]], a, b)
        want = gm.sample(mu, L, z[r], float(cmult[c]), parent, free)
        ulp = np.spacing(np.abs(want)).astype(np.float32)
        assert np.all(np.abs(got[r] - want) <= ulp), (r, got[r], want)
        np.testing.assert_array_equal(got[r][~free], parent[~free].astype(np.float32))


def test_bad_indices_give_nan_rows(mo):
    p = synth.make_c0(n_sol=4)
    el, _ = mo.parallel_groups(p.n_points, p.tets)
    gp = mo.Problem(p, max_solutions=1)
    dv = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    members = np.array([[0, 1], [2, 99]], np.int32)          # cluster 1 names a solution out of range
    req_sol = np.array([0, 0, 7, 1], np.int32)
    req_cl = np.array([0, 1, 0, 0], np.int32)
    req_el = np.array([0, 0, 0, len(el)], np.int32)
    z = np.zeros((4, 12), np.float32)
    new_s, new_t = gp.sample_elements(dv(p.sol_src), dv(p.sol_tgt), dv(members), dv(el), dv(np.ones(2, np.float32)),
                                      dv(req_sol), dv(req_cl), dv(req_el), dv(z))
    s = new_s.cpu().numpy().reshape(4, 6)
    assert np.isfinite(s[0]).all()
    assert np.isnan(s[1]).all() and np.isnan(s[2]).all() and np.isnan(s[3]).all()


def test_slot_objectives_follow_commits(mo):
    p = synth.make_c0(n_sol=4)
    n = 4
    gp = mo.Problem(p, max_solutions=n, max_requests=n, max_changed=4)
    S = torch.as_tensor(p.sol_src).cuda()
    T = torch.as_tensor(p.sol_tgt).cuda()
    obj, folded, sev = gp.eval_full(S, T)
    o2, f2, s2 = gp.slot_objectives(n)
    np.testing.assert_array_equal(o2.cpu().numpy(), obj.cpu().numpy())
    np.testing.assert_array_equal(f2.cpu().numpy(), folded.cpu().numpy())
    rng = np.random.default_rng(1)
    cur_s, cur_t = p.sol_src.copy(), p.sol_tgt.copy()
    pts = np.array([20, 21, 40, 62], np.int32)
    off = np.array([0, 1, 2, 3, 4], np.int32)
    slots = np.arange(n, dtype=np.int32)
    new_s = (cur_s[slots, pts] + rng.normal(0, 0.5, (n, 3)) * ~p.fixed_axes[pts]).astype(np.float32)
    new_t = (cur_t[slots, pts] + rng.normal(0, 0.5, (n, 3)) * ~p.fixed_axes[pts]).astype(np.float32)
    dv = lambda a: torch.as_tensor(a).cuda()
    gp.eval_partial(dv(slots), dv(off), dv(pts), dv(new_s), dv(new_t))
    acc = np.array([1, 0, 1, 1], np.uint8)
    gp.commit_partial(dv(acc))
    for i in np.nonzero(acc)[0]:
        cur_s[i, pts[i]] = new_s[i]
        cur_t[i, pts[i]] = new_t[i]
    o3, f3, _ = gp.slot_objectives(n)
    fresh = mo.Problem(p, max_solutions=n)
    o4, f4, _ = fresh.eval_full(torch.as_tensor(cur_s).cuda(), torch.as_tensor(cur_t).cuda())
    np.testing.assert_allclose(o3.cpu().numpy(), o4.cpu().numpy(), rtol=1e-9)
    np.testing.assert_array_equal(f3.cpu().numpy(), f4.cpu().numpy())


def _pareto_ok(pts):
    for i in range(len(pts)):
        for j in range(len(pts)):
            if i != j:
                assert not (np.all(pts[j] <= pts[i]) and np.any(pts[j] < pts[i]))


def test_generations_keep_their_invariants(mo):
    from paper_2303_04873_gb300 import gomea
    p = synth.make_c0(n_sol=1)
    n = 16
    cfg = gomea.GomeaConfig(clusters=4, steer_at=1000, init_kernels=4, init_rounds=20, init_sigma=(3.0, 9.0),
                            init_strength=(0.05, 0.2))
    gp = mo.Problem(p, max_solutions=n, max_requests=gomea.max_requests(p, n), max_changed=gomea.max_changed(cfg))
    run = gomea.Gomea(gp, p, n, cfg, seed=4)
    ref = 1.1 * run.obj.max(axis=0)
    hv = [run.hypervolume(ref)]
    for _ in range(4):
        st = run.step()
        assert st["requests"] > 0
        hv.append(run.hypervolume(ref))
    assert run.accepted > 0
    assert all(b >= a - 1e-12 for a, b in zip(hv, hv[1:]))          # no pruning at this size
    _pareto_ok(run.archive.pts)
    # the device coordinates are the committed solutions: a fresh evaluation agrees
    fresh = mo.Problem(p, max_solutions=n)
    o, f, _ = fresh.eval_full(run.S, run.T)
    np.testing.assert_allclose(o.cpu().numpy(), run.obj, rtol=1e-9)
    assert not f.cpu().numpy().any()
    assert gp.device_status() == 0


def test_adaptive_steering_window(mo):
    from paper_2303_04873_gb300 import gomea
    p = synth.make_c0(n_sol=1)
    n = 16
    cfg = gomea.GomeaConfig(clusters=4, steer_at=2, init_kernels=4, init_rounds=20, init_sigma=(3.0, 9.0),
                            init_strength=(0.05, 0.2))
    gp = mo.Problem(p, max_solutions=n, max_requests=gomea.max_requests(p, n), max_changed=gomea.max_changed(cfg))
    run = gomea.Gomea(gp, p, n, cfg, seed=5)
    for _ in range(4):
        run.step()
    g = run.archive.pts[:, 2]
    assert np.all(g <= 1.5 * g.min() + 1e-15)


def test_folded_candidates_are_repaired(mo):
    """A large distribution multiplier makes many candidates fold, and the
    repair path runs every generation.  Acceptance is widened to every
    unfolded candidate (the rule itself is tested above), so repaired
    candidates are committed too: the committed objectives must still equal
    a fresh evaluation, with every boundary axis in place."""
    from paper_2303_04873_gb300 import gomea
    p = synth.make_c0(n_sol=1)
    n = 16
    cfg = gomea.GomeaConfig(clusters=4, steer_at=1000, init_kernels=4, init_rounds=20, init_sigma=(3.0, 9.0),
                            init_strength=(0.05, 0.2), cmult0=6.0, repair_points=8)
    gp = mo.Problem(p, max_solutions=n, max_requests=gomea.max_requests(p, n), max_changed=gomea.max_changed(cfg))
    run = gomea.Gomea(gp, p, n, cfg, seed=6)
    run._accept = lambda o, f, sol, hi: ~f & np.all(np.isfinite(o), axis=1)
    for _ in range(3):
        run.step()
    assert run.repaired > 0 and run.repaired_accepted > 0
    fresh = mo.Problem(p, max_solutions=n)
    o, f, _ = fresh.eval_full(run.S, run.T)
    np.testing.assert_allclose(o.cpu().numpy(), run.obj, rtol=1e-9)
    assert not f.cpu().numpy().any()
    fx = p.fixed_axes
    for X in (run.S.cpu().numpy(), run.T.cpu().numpy()):
        np.testing.assert_array_equal(X[:, fx], np.broadcast_to(p.ref_points[fx], (n,) + p.ref_points[fx].shape))
    _pareto_ok(run.archive.pts)
    assert gp.device_status() == 0


def test_generations_on_the_full_size_problem(mo):
    """Two generations on the 128x128x96 problem (population 32, the paper's
    10 clusters, repair on): committed objectives equal a fresh evaluation
    of the device coordinates, nothing is folded, boundary axes stay."""
    from paper_2303_04873_gb300 import gomea
    p = synth.make_c1(n_sol=1)
    n = 32
    cfg = gomea.GomeaConfig()
    gp = mo.Problem(p, max_solutions=n, max_requests=gomea.max_requests(p, n), max_changed=gomea.max_changed(cfg))
    run = gomea.Gomea(gp, p, n, cfg, seed=9)
    for _ in range(2):
        st = run.step()
        assert st["requests"] == n * len(run.el_host)
    assert run.accepted > 0
    fresh = mo.Problem(p, max_solutions=n)
    o, f, _ = fresh.eval_full(run.S, run.T)
    np.testing.assert_allclose(o.cpu().numpy(), run.obj, rtol=1e-9)
    assert not f.cpu().numpy().any()
    fx = p.fixed_axes
    for X in (run.S.cpu().numpy(), run.T.cpu().numpy()):
        np.testing.assert_array_equal(X[:, fx], np.broadcast_to(p.ref_points[fx], (n,) + p.ref_points[fx].shape))
    _pareto_ok(run.archive.pts)
    assert gp.device_status() == 0


def test_screened_generations(mo):
    """The learned and the random pre-screen evaluate exactly round(0.25 n m)
    requests per group of m elements (plus the population and the repaired
    candidates), and the committed objectives still equal a fresh
    evaluation of the device coordinates."""
    from paper_2303_04873_gb300 import ea, gomea
    p = synth.make_c0(n_sol=1)
    n = 16
    cfg = gomea.GomeaConfig(clusters=4, steer_at=1000, init_kernels=4, init_rounds=20, init_sigma=(3.0, 9.0),
                            init_strength=(0.05, 0.2), repair=False)
    gp = mo.Problem(p, max_solutions=n, max_requests=gomea.max_requests(p, n), max_changed=gomea.max_changed(cfg))
    log = []
    data = gomea.Gomea(gp, p, n, cfg, seed=7, log=log, log_per_group=64)
    for _ in range(3):
        data.step()
    feats = torch.cat([f for f, _ in log])
    targ = np.concatenate([o for _, o in log])
    assert feats.shape == (len(targ), 3 * p.n_points)
    net = mo.Mlp(3 * p.n_points, 64, 64, 3, max_batch=256, seed=0)
    tr = ea.train_surrogate(net, feats, targ, epochs=2, lr=1e-3)
    per_gen = sum(max(1, int(round(0.25 * n * len(g)))) for g in data.groups)
    for kind in ("surrogate", "random"):
        run = gomea.Gomea(gp, p, n, cfg, seed=8, surrogate=tr["surrogate"] if kind == "surrogate" else None,
                          random_screen=kind == "random")
        for _ in range(2):
            st = run.step()
            assert st["requests"] == per_gen
        assert run.exact == n + 2 * per_gen
        fresh = mo.Problem(p, max_solutions=n)
        o, f, _ = fresh.eval_full(run.S, run.T)
        np.testing.assert_allclose(o.cpu().numpy(), run.obj, rtol=1e-9)
        assert not f.cpu().numpy().any()
        _pareto_ok(run.archive.pts)
    assert gp.device_status() == 0
