"""Large tet copies: every copy of a coarse mesh is an item that the ordered
image pass of a partial evaluation takes first.

On a 96x96x64 image with a 3x3x3 lattice every tet copy's bounding box holds
48 x 48 x 32 = 73 728 voxel centres, so every item of every partial round is
on the entry pass's list of large items.  The checks, in four modes (FP32
with continuous guidance, FP16 with the foreground/background h and pair
transfer, a narrow guidance band, no guidance): the full evaluation against
the FP64 oracle per tet; every partial request against the oracle's partial
evaluation; and, after rounds of commits, the committed per-tet records equal
a fresh full evaluation's bit for bit (the full evaluation takes the items in
tet-major order, the partial ones from the list)."""

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import assert_obj_close, check_against_oracle, gpu_full

pytestmark = pytest.mark.gpu

LARGE_ELLIPSOIDS = [
    (30.0, 36.0, 32.0, 18.0, 15.0, 14.0, 40.0),
    (63.0, 54.0, 28.0, 15.0, 21.0, 12.0, 80.0),
    (48.0, 66.0, 44.0, 12.0, 12.0, 10.0, 120.0),
]


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def large_problem(n_sol, **kw):
    args = dict(name="large_96x96x64", shape_xyz=(96, 96, 64), ellipsoids=LARGE_ELLIPSOIDS, background=0.0,
                amp=3.0, noise_sigma=5.0, dtype="f32", xs=np.linspace(-0.5, 95.5, 3), ys=np.linspace(-0.5, 95.5, 3),
                zs=np.linspace(-0.5, 63.5, 3), n_guid=200, n_sol=n_sol, jitter=1.5, tissue=[1.0, 0.5, 2.0, 4.0],
                seeds=(3, 4, 5))
    args.update(kw)
    return synth.make_problem(**args)


@pytest.mark.parametrize("kw", [dict(), dict(dtype="f16", h_mode=1, g_mode=1), dict(trunc_radius=1.0),
                                dict(g_mode=2)], ids=["f32-continuous", "f16-fg-pairs", "narrow-band", "no-guidance"])
def test_large_items_match_oracle_and_full(mo, kw):
    n = 4
    p = large_problem(n, **kw)
    gp, orc, _ = check_against_oracle(mo, p)
    gp.close()
    gp = mo.Problem(p, max_solutions=n, max_requests=n, max_changed=32)
    cur_s, cur_t = p.sol_src.copy(), p.sol_tgt.copy()
    gpu_full(gp, cur_s, cur_t)
    cur_res = [orc.eval(cur_s[i], cur_t[i]) for i in range(n)]
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rng = np.random.default_rng(11)
    rounds = synth.partial_requests(p, adj, 5, 1, 4, 1.5, 13)
    for rd in rounds:
        off = rd["chg_off"]
        for k in range(n):
            ids = rd["chg_pts"][off[k]:off[k + 1]]
            rd["chg_src"][off[k]:off[k + 1]] += cur_s[k, ids] - p.sol_src[k, ids]
            rd["chg_tgt"][off[k]:off[k + 1]] += cur_t[k, ids] - p.sol_tgt[k, ids]
        dv = {kk: torch.as_tensor(v).cuda() for kk, v in rd.items()}
        accept = (rng.random(n) < 0.6).astype(np.uint8)
        obj, folded, sev = gp.eval_partial(dv["slot"], dv["chg_off"], dv["chg_pts"], dv["chg_src"], dv["chg_tgt"])
        gp.commit_partial(torch.as_tensor(accept).cuda())
        obj, folded, sev = obj.cpu().numpy(), folded.cpu().numpy(), sev.cpu().numpy()
        assert gp.device_status() == 0
        for k in range(n):
            ids = rd["chg_pts"][off[k]:off[k + 1]]
            ns, nt = cur_s[k].copy(), cur_t[k].copy()
            ns[ids] = rd["chg_src"][off[k]:off[k + 1]]
            nt[ids] = rd["chg_tgt"][off[k]:off[k + 1]]
            r = orc.eval_partial(cur_s[k], cur_t[k], ns, nt, ids, cur_res[k])
            assert int(folded[k]) == r["folded"]
            assert sev[k] == r["severity"]
            if not r["folded"]:
                assert_obj_close(obj[k], r["obj"], f"request {k}")
            if accept[k]:
                cur_s[k], cur_t[k], cur_res[k] = ns, nt, r
    committed = gp.read_records(n)
    tot_before = gp.read_totals(n)
    gpu_full(gp, cur_s, cur_t)
    fresh = gp.read_records(n)
    for f in ("e_img", "e_guid", "n_vox", "n_gp", "e_mag", "folded", "sev"):
        np.testing.assert_array_equal(committed[f], fresh[f], err_msg=f)
    tot_after = gp.read_totals(n)
    for f in ("n_vox", "n_folded", "sev"):
        np.testing.assert_array_equal(tot_before[f], tot_after[f])
    for f in ("s_img", "s_guid", "s_mag"):
        np.testing.assert_allclose(tot_before[f], tot_after[f], rtol=1e-12, atol=1e-12)
    assert gp.device_status() == 0
