"""Parallel groups on the GPU (Sec. 4.2.1): one morea_eval_partial call
carries a request for every element of a group on every solution, so a
slot gets many requests at once.  Each request's objectives equal the
oracle's partial evaluation against the same parent, and after the
accepted requests are committed, the totals equal a fresh full evaluation
of the resulting coordinates."""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def test_group_requests_on_shared_slots(mo):
    p = synth.make_c0(n_sol=3)
    n = 3
    el, grp = mo.parallel_groups(p.n_points, p.tets)
    biggest = int(np.bincount(grp).max())
    gp = mo.Problem(p, max_solutions=n, max_requests=n * biggest, max_changed=2)
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits, trunc_radius=gp.trunc_radius)
    cur_s, cur_t = p.sol_src.copy(), p.sol_tgt.copy()
    S = torch.as_tensor(cur_s).cuda()
    T = torch.as_tensor(cur_t).cuda()
    gp.eval_full(S, T)
    res = [orc.eval(cur_s[i], cur_t[i]) for i in range(n)]
    rng = np.random.default_rng(5)
    fixed = p.fixed_axes
    for g in range(int(grp.max()) + 1):
        members = el[grp == g]
        m = len(members)
        slots = np.repeat(np.arange(n, dtype=np.int32), m)
        pts = np.tile(members, (n, 1)).reshape(-1).astype(np.int32)
        off = np.arange(0, 2 * n * m + 1, 2, dtype=np.int32)
        step = rng.normal(0, 0.8, size=(len(pts), 2, 3))
        step[np.repeat(fixed[pts][:, None, :], 2, axis=1)] = 0.0
        owner = slots.repeat(2)
        new_s = (cur_s[owner, pts] + step[:, 0]).astype(np.float32)
        new_t = (cur_t[owner, pts] + step[:, 1]).astype(np.float32)
        dv = [torch.as_tensor(a).cuda() for a in (slots, off, pts, new_s, new_t)]
        obj, folded, _ = gp.eval_partial(*dv)
        obj, folded = obj.cpu().numpy(), folded.cpu().numpy()
        accept = (rng.random(n * m) < 0.6).astype(np.uint8)
        gp.commit_partial(torch.as_tensor(accept).cuda())
        assert gp.device_status() == 0
        # every request against its parent, in the oracle (a sample of them)
        for r in rng.choice(n * m, size=min(6, n * m), replace=False):
            s = int(slots[r])
            ids = pts[off[r]:off[r + 1]]
            ns, nt = cur_s[s].copy(), cur_t[s].copy()
            ns[ids] = new_s[off[r]:off[r + 1]]
            nt[ids] = new_t[off[r]:off[r + 1]]
            want = orc.eval_partial(cur_s[s], cur_t[s], ns, nt, ids, res[s])
            np.testing.assert_allclose(obj[r, :2], want["obj"][:2], rtol=1e-5)
            np.testing.assert_allclose(obj[r, 2], want["obj"][2], rtol=1e-5, atol=1e-10)
            assert int(folded[r]) == want["folded"]
        # apply the accepted requests (their points are disjoint within a slot)
        for r in np.nonzero(accept)[0]:
            s = int(slots[r])
            ids = pts[off[r]:off[r + 1]]
            cur_s[s, ids] = new_s[off[r]:off[r + 1]]
            cur_t[s, ids] = new_t[off[r]:off[r + 1]]
        res = [orc.eval(cur_s[i], cur_t[i]) for i in range(n)]
    tot = gp.read_totals(n)
    fresh = mo.Problem(p, max_solutions=n)
    obj2, _, _ = fresh.eval_full(torch.as_tensor(cur_s).cuda(), torch.as_tensor(cur_t).cuda())
    tot2 = fresh.read_totals(n)
    np.testing.assert_array_equal(tot["n_vox"], tot2["n_vox"])
    np.testing.assert_array_equal(tot["sev"], tot2["sev"])
    for f in ("s_img", "s_guid", "s_mag"):
        np.testing.assert_allclose(tot[f], tot2[f], rtol=1e-9, atol=1e-12)
    for i in range(n):
        np.testing.assert_allclose(obj2.cpu().numpy()[i, :2], res[i]["obj"][:2], rtol=1e-5)
