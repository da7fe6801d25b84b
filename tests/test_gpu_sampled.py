"""GPU parity of the sampled estimator (App. A.2, estimator SAMPLED) against
the oracle's restatement (reading R13), through the C ABI.

Bars as for the voxel estimator: sample counts (the records' n_vox), fold
flags and severities bit-exact; per-tet sums within 1e-4 and objectives
within 1e-5 relative error.  The kernel computes -log, the barycentric
coordinates and the sample positions in FP32, the oracle in FP64."""

import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import _random_case, assert_obj_close, check_against_oracle, gpu_full

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def sampled(p, rate=1.0, **kw):
    q = dataclasses.replace(p, estimator=1, sampling_rate=rate) if dataclasses.is_dataclass(p) else p
    if not dataclasses.is_dataclass(p):
        q.estimator, q.sampling_rate = 1, rate
    for k, v in kw.items():
        setattr(q, k, v)
    return q


@pytest.mark.parametrize("rate", [1.0, 0.37, 3.0])
def test_c0_sampled_full_parity(mo, rate):
    p = sampled(synth.make_c0(), rate)
    gp, orc, obj = check_against_oracle(mo, p)
    recs = gp.read_records(8)
    assert recs["n_vox"].sum() > 0


@pytest.mark.parametrize("over", [dict(g_mode=2), dict(trunc_radius=4.0)])
def test_c0_sampled_modes(mo, over):
    check_against_oracle(mo, sampled(synth.make_c0(n_sol=4)), **over)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_sampled_random_small_meshes(mo, seed, dtype):
    prob = _random_case(seed, dtype=dtype, g_mode=0 if seed % 2 == 0 else 2, h_mode=0)
    check_against_oracle(mo, sampled(prob, 0.8 + 0.3 * seed))


def test_sampled_folded_solutions(mo):
    prob = _random_case(51, fold=True)
    check_against_oracle(mo, sampled(prob, 1.0))


def test_sampled_counts_follow_the_volume(mo):
    p = sampled(synth.make_c0(n_sol=2), 2.0)
    gp = mo.Problem(p, max_solutions=2)
    gpu_full(gp, p.sol_src, p.sol_tgt)
    tot = gp.read_totals(2)
    # the sum of the copies' volumes is the box volume for an unfolded,
    # box-spanning mesh, so the total count is near rate * 2 * volume
    want = 2.0 * 2 * p.voxels()
    assert abs(tot["n_vox"][0] - want) < 0.5 * 2 * p.n_tets + 1


def test_sampled_partial_matches_oracle_and_full(mo):
    p = sampled(synth.make_c0(n_sol=6), 0.75)
    n = 6
    gp = mo.Problem(p, max_solutions=n, max_requests=n)
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits, trunc_radius=gp.trunc_radius)
    cur_s, cur_t = p.sol_src.copy(), p.sol_tgt.copy()
    gpu_full(gp, cur_s, cur_t)
    cur_res = [orc.eval(cur_s[i], cur_t[i]) for i in range(n)]
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rng = np.random.default_rng(11)
    for rd in synth.partial_requests(p, adj, 6, 4, 24, 1.0, 5):
        off = rd["chg_off"]
        for k in range(n):
            ids = rd["chg_pts"][off[k]:off[k + 1]]
            rd["chg_src"][off[k]:off[k + 1]] += cur_s[k, ids] - p.sol_src[k, ids]
            rd["chg_tgt"][off[k]:off[k + 1]] += cur_t[k, ids] - p.sol_tgt[k, ids]
        dv = {kk: torch.as_tensor(v).cuda() for kk, v in rd.items()}
        accept = (rng.random(n) < 0.5).astype(np.uint8)
        obj, folded, sev = gp.eval_partial(dv["slot"], dv["chg_off"], dv["chg_pts"], dv["chg_src"], dv["chg_tgt"])
        gp.commit_partial(torch.as_tensor(accept).cuda())
        obj, folded = obj.cpu().numpy(), folded.cpu().numpy()
        assert gp.device_status() == 0
        for k in range(n):
            ids = rd["chg_pts"][off[k]:off[k + 1]]
            ns, nt = cur_s[k].copy(), cur_t[k].copy()
            ns[ids] = rd["chg_src"][off[k]:off[k + 1]]
            nt[ids] = rd["chg_tgt"][off[k]:off[k + 1]]
            r = orc.eval_partial(cur_s[k], cur_t[k], ns, nt, ids, cur_res[k])
            assert int(folded[k]) == r["folded"]
            assert_obj_close(obj[k], r["obj"], f"request {k}")
            if accept[k]:
                cur_s[k], cur_t[k], cur_res[k] = ns, nt, r
    tot_before = gp.read_totals(n)
    obj2, _, _ = gpu_full(gp, cur_s, cur_t)
    tot_after = gp.read_totals(n)
    np.testing.assert_array_equal(tot_before["n_vox"], tot_after["n_vox"])
    for f in ("s_img", "s_guid", "s_mag"):
        np.testing.assert_allclose(tot_before[f], tot_after[f], rtol=1e-9, atol=1e-12)
    for k in range(n):
        assert_obj_close(obj2[k], cur_res[k]["obj"], f"final {k}")


def test_sampled_batch_equals_single_problem(mo):
    probs = [sampled(synth.make_c0(n_sol=3, seeds=(s, s + 1, s + 2)), 1.0) for s in (0, 3)]
    gps = [mo.Problem(p, max_solutions=3) for p in probs]
    single = [gpu_full(g, p.sol_src, p.sol_tgt)[0] for g, p in zip(gps, probs)]
    b = mo.Batch(gps)
    srcs = [torch.as_tensor(p.sol_src).cuda() for p in probs]
    tgts = [torch.as_tensor(p.sol_tgt).cuda() for p in probs]
    outs = b.eval_full(srcs, tgts)
    torch.cuda.synchronize()
    for (obj, _, _), want in zip(outs, single):
        np.testing.assert_array_equal(obj.cpu().numpy(), want)
