"""GPU parity: libmorea (through the C ABI) against the FP64 oracle.

Bars: voxel coverage counts, fold flags and severities bit-exact; objectives
within 1e-5 relative error of the oracle; per-tet sums within 1e-4.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import GAMMA_POS, GAMMA_VAL, MAX_AMBIGUOUS, box_lattice, problem, random_image

pytestmark = pytest.mark.gpu

RTOL_OBJ = 1e-5
RTOL_TET = 1e-4


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def gpu_full(gp, src, tgt, slots=None):
    S = torch.as_tensor(np.ascontiguousarray(src, np.float32)).cuda()
    T = torch.as_tensor(np.ascontiguousarray(tgt, np.float32)).cuda()
    sl = None if slots is None else torch.as_tensor(np.asarray(slots, np.int32)).cuda()
    obj, folded, sev = gp.eval_full(S, T, sl)
    torch.cuda.synchronize()
    return obj.cpu().numpy(), folded.cpu().numpy(), sev.cpu().numpy()


def assert_obj_close(g, o, what=""):
    np.testing.assert_allclose(g[:2], o[:2], rtol=RTOL_OBJ, atol=0, err_msg=what)
    np.testing.assert_allclose(g[2], o[2], rtol=RTOL_OBJ, atol=1e-10, err_msg=what)


def check_against_oracle(mo, prob, idx=None, **over):
    """Full evaluation of prob.sol_src/sol_tgt on the GPU; oracle on ``idx``.

    In the foreground/background mode of h the oracle decides each case on
    the exact sample (R9).  Voxels whose exact sample lies within the FP32
    error bound of 0 (helpers.GAMMA_*) are ambiguous: a tet's e_img may then
    differ by the spread of h they allow (``amb_slack``) on top of the FP32
    rounding tolerance; every other voxel must take the oracle's case.  The
    ambiguous voxels must stay below MAX_AMBIGUOUS of the covered ones."""
    n = prob.sol_src.shape[0]
    gp = mo.Problem(prob, max_solutions=n, **over)
    orc = oracle.Oracle(prob, **{**over, "subvoxel_bits": gp.subvoxel_bits, "trunc_radius": gp.trunc_radius})
    orc.set_perturbation(GAMMA_POS, GAMMA_VAL)
    obj, folded, sev = gpu_full(gp, prob.sol_src, prob.sol_tgt)
    recs = gp.read_records(n)
    for i in (range(n) if idx is None else idx):
        r = orc.eval(prob.sol_src[i], prob.sol_tgt[i], with_tets=True)
        ot = r["tets"]
        np.testing.assert_array_equal(recs[i]["n_vox"], ot["n_vox"])
        np.testing.assert_array_equal(recs[i]["n_gp"], ot["n_gp"])
        np.testing.assert_array_equal(recs[i]["folded"], ot["folded"])
        np.testing.assert_array_equal(recs[i]["sev"], ot["sev"])
        slack = ot["amb_slack"]
        assert ot["amb_n"].sum() <= MAX_AMBIGUOUS * max(1, ot["n_vox"].sum()), "too many ambiguous voxels"
        err = np.abs(recs[i]["e_img"].astype(np.float64) - ot["e_img"])
        assert (err <= RTOL_TET * np.abs(ot["e_img"]) + 1e-3 + slack).all(), f"e_img of solution {i}"
        np.testing.assert_allclose(recs[i]["e_mag"], ot["e_mag"], rtol=RTOL_TET, atol=1e-9)
        assert int(folded[i]) == r["folded"]
        assert sev[i] == r["severity"]
        total_slack = slack.sum() / max(1, r["n_vox"])
        if total_slack == 0.0:
            assert_obj_close(obj[i], r["obj"], f"solution {i}")
        else:
            assert abs(obj[i][0] - r["obj"][0]) <= RTOL_OBJ * abs(r["obj"][0]) + total_slack, f"solution {i}"
            assert_obj_close(np.r_[r["obj"][0], obj[i][1:]], r["obj"], f"solution {i}")
    return gp, orc, obj


def test_c0_full_parity(mo):
    p = synth.make_c0()
    gp, orc, obj = check_against_oracle(mo, p)
    tot = gp.read_totals(8)
    assert (tot["n_vox"] == 2 * p.voxels()).all()          # every voxel centre exactly once per side


@pytest.mark.parametrize("over", [
    dict(h_mode=1), dict(g_mode=1), dict(g_mode=2), dict(trunc_radius=4.0), dict(trunc_radius=4.0, h_mode=1),
])
def test_c0_modes(mo, over):
    p = synth.make_c0(n_sol=4)
    if over.get("h_mode") == 1:
        # two-level foreground images: the FG case split is exercised, and
        # every sample is either exactly 0 or clearly positive
        p.image_s = np.where(p.image_s > 20, p.image_s, 0).astype(np.float32)
        p.image_t = np.where(p.image_t > 20, p.image_t, 0).astype(np.float32)
    check_against_oracle(mo, p, **over)


def test_identity_gives_zero_magnitude_and_plain_ssd(mo):
    p = synth.make_c0(n_sol=2)
    p.sol_src = np.stack([p.ref_points] * 2)
    p.sol_tgt = np.stack([p.ref_points] * 2)
    gp = mo.Problem(p, max_solutions=2)
    obj, folded, sev = gpu_full(gp, p.sol_src, p.sol_tgt)
    ssd = ((p.image_s.astype(np.float64) - p.image_t.astype(np.float64)) ** 2).mean()
    assert obj[0, 1] == 0.0
    np.testing.assert_allclose(obj[0, 0], ssd, rtol=1e-6)
    assert folded.tolist() == [0, 0]


def test_adversarial_ties_each_voxel_once(mo):
    nx, ny, nz = 12, 10, 9
    pts, tets = box_lattice([-0.5, 3.0, 7.0, 11.5], [-0.5, 4.0, 9.5], [-0.5, 2.0, 5.0, 8.5])
    rng = np.random.default_rng(3)
    interior = np.all((pts > -0.5) & (pts < np.array([nx, ny, nz]) - 0.5), axis=1)
    sols = []
    for s in range(4):
        q = pts.copy()
        q[interior] += rng.integers(-1, 2, size=(interior.sum(), 3)) * 0.5
        sols.append(q)
    sols = np.stack(sols).astype(np.float32)
    img = random_image((nz, ny, nx), 4)
    img2 = random_image((nz, ny, nx), 5)
    prob = problem(img, img2, pts, tets, sol_src=sols, sol_tgt=sols[::-1].copy())
    gp, orc, obj = check_against_oracle(mo, prob)
    tot = gp.read_totals(4)
    assert (tot["n_vox"] == 2 * nx * ny * nz).all()


def _random_case(seed, dtype=np.float32, fold=False, g_mode=0, h_mode=0):
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(v) for v in rng.integers(8, 17, size=3))
    cx, cy, cz = (int(v) for v in rng.integers(1, 4, size=3))
    xs = np.linspace(-0.5, nx - 0.5, cx + 1)
    ys = np.linspace(-0.5, ny - 0.5, cy + 1)
    zs = np.linspace(-0.5, nz - 0.5, cz + 1)
    pts, tets = box_lattice(xs, ys, zs, flip_x=bool(rng.integers(0, 2)))
    fixed = np.zeros(pts.shape, bool)
    for a, n in enumerate((nx, ny, nz)):
        fixed[:, a] = (pts[:, a] == np.float32(-0.5)) | (pts[:, a] == np.float32(n - 0.5))
    P = 6
    amp = 0.6 * min(nx / cx, ny / cy, nz / cz) * (0.9 if fold else 0.2)
    src = pts[None] + rng.uniform(-amp, amp, size=(P,) + pts.shape)
    tgt = pts[None] + rng.uniform(-amp, amp, size=(P,) + pts.shape)
    src[:, fixed] = pts[fixed]
    tgt[:, fixed] = pts[fixed]
    # some coordinates exactly on voxel centres / half voxels (ties)
    m = rng.random(src.shape) < 0.3
    src[m] = np.round(src[m] * 2) / 2
    img_s = random_image((nz, ny, nx), seed + 100).astype(dtype)
    img_t = random_image((nz, ny, nx), seed + 200).astype(dtype)
    if h_mode == 1:
        img_s = np.where(img_s > 0, img_s, 0).astype(dtype)
        img_t = np.where(img_t > 0, img_t, 0).astype(dtype)
    ng = 24
    gs = rng.uniform(0, [nx - 1, ny - 1, nz - 1], size=(ng, 3))
    gt = gs + rng.normal(0, 0.8, size=gs.shape)
    label = rng.integers(0, 3, size=len(tets)).astype(np.int32)
    return problem(img_s, img_t, pts, tets, label=label, tissue=[1.0, 0.5, 3.0], guid_s=gs, guid_t=gt,
                   guid_group=(np.arange(ng) % 3).astype(np.int32), trunc_radius=3.0, g_mode=g_mode,
                   h_mode=h_mode, sol_src=src.astype(np.float32), sol_tgt=tgt.astype(np.float32))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_random_small_meshes(mo, seed, dtype):
    prob = _random_case(seed, dtype=dtype, g_mode=seed % 3, h_mode=seed % 2)
    check_against_oracle(mo, prob)


@pytest.mark.parametrize("seed", range(4))
def test_folded_solutions(mo, seed):
    prob = _random_case(50 + seed, fold=True)
    gp, orc, obj = check_against_oracle(mo, prob)
    # the fold-only entry point agrees with the full evaluation
    S = torch.as_tensor(prob.sol_src).cuda()
    T = torch.as_tensor(prob.sol_tgt).cuda()
    folded, sev = gp.check_folds(S, T)
    torch.cuda.synchronize()
    for i in range(prob.sol_src.shape[0]):
        r = orc.eval(prob.sol_src[i], prob.sol_tgt[i])
        assert int(folded[i]) == r["folded"]
        assert float(sev[i]) == r["severity"]


def test_tet_without_voxel_centres(mo):
    # a sliver between voxel-centre planes covers no centre; a lone tet in a
    # large box leaves most voxels uncovered
    img = random_image((10, 10, 10), 1)
    pts = np.array([[2.1, 2.1, 2.1], [2.9, 2.2, 2.2], [2.2, 2.9, 2.3], [2.3, 2.3, 2.9],
                    [1.0, 1.0, 1.0], [8.0, 1.0, 1.0], [1.0, 8.0, 1.0], [1.0, 1.0, 8.0]], np.float32)
    tets = np.array([[0, 1, 2, 3], [4, 5, 6, 7]], np.int32)
    prob = problem(img, img, pts, tets, sol_src=pts[None].copy(), sol_tgt=(pts[None] + 0.25).astype(np.float32))
    gp, orc, obj = check_against_oracle(mo, prob)
    recs = gp.read_records(1)
    assert recs[0]["n_vox"][0].tolist() == [0, 0]


def test_partial_matches_oracle_and_full(mo):
    p = synth.make_c0(n_sol=8)
    n = 8
    gp = mo.Problem(p, max_solutions=n, max_requests=n)
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits, trunc_radius=gp.trunc_radius)
    cur_s, cur_t = p.sol_src.copy(), p.sol_tgt.copy()
    gpu_full(gp, cur_s, cur_t)
    cur_res = [orc.eval(cur_s[i], cur_t[i]) for i in range(n)]
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rng = np.random.default_rng(7)
    rounds = synth.partial_requests(p, adj, 12, 4, 32, 1.0, 3)
    for rd in rounds:
        # moves are relative to the current committed solutions
        off = rd["chg_off"]
        for k in range(n):
            ids = rd["chg_pts"][off[k]:off[k + 1]]
            rd["chg_src"][off[k]:off[k + 1]] += cur_s[k, ids] - p.sol_src[k, ids]
            rd["chg_tgt"][off[k]:off[k + 1]] += cur_t[k, ids] - p.sol_tgt[k, ids]
        dv = {kk: torch.as_tensor(v).cuda() for kk, v in rd.items()}
        accept = (rng.random(n) < 0.5).astype(np.uint8)
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
            assert_obj_close(obj[k], r["obj"], f"request {k}")
            if accept[k]:
                cur_s[k], cur_t[k], cur_res[k] = ns, nt, r
    # committed state == a fresh full evaluation of the committed coordinates
    tot_before = gp.read_totals(n)
    obj2, _, _ = gpu_full(gp, cur_s, cur_t)
    tot_after = gp.read_totals(n)
    np.testing.assert_array_equal(tot_before["n_vox"], tot_after["n_vox"])
    np.testing.assert_array_equal(tot_before["n_folded"], tot_after["n_folded"])
    np.testing.assert_array_equal(tot_before["sev"], tot_after["sev"])
    for f in ("s_img", "s_guid", "s_mag"):
        np.testing.assert_allclose(tot_before[f], tot_after[f], rtol=1e-9, atol=1e-12)
    for k in range(n):
        assert_obj_close(obj2[k], cur_res[k]["obj"], f"final {k}")


def test_partial_commit_flag_equals_commit_call(mo):
    p = synth.make_c0(n_sol=4)
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rd = synth.partial_requests(p, adj, 1, 4, 16, 1.0, 9)[0]
    dv = {k: torch.as_tensor(v).cuda() for k, v in rd.items()}
    outs = []
    for mode in ("flag", "call"):
        gp = mo.Problem(p, max_solutions=4)
        gpu_full(gp, p.sol_src, p.sol_tgt)
        acc = torch.tensor([1, 0, 1, 1], dtype=torch.uint8, device="cuda")
        if mode == "flag":
            gp.eval_partial(dv["slot"], dv["chg_off"], dv["chg_pts"], dv["chg_src"], dv["chg_tgt"], commit=acc)
        else:
            gp.eval_partial(dv["slot"], dv["chg_off"], dv["chg_pts"], dv["chg_src"], dv["chg_tgt"])
            gp.commit_partial(acc)
        outs.append((gp.read_totals(4), gp.read_records(4)))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_device_status_for_bad_requests(mo):
    p = synth.make_c0(n_sol=2)
    gp = mo.Problem(p, max_solutions=2, max_changed=8)
    gpu_full(gp, p.sol_src, p.sol_tgt)
    dev = "cuda"
    slot = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    off = torch.tensor([0, 2, 4], dtype=torch.int32, device=dev)
    pts = torch.tensor([3, 10_000, 5, 6], dtype=torch.int32, device=dev)       # request 0: bad id
    xyz = torch.zeros((4, 3), dtype=torch.float32, device=dev) + 5.0
    obj, folded, sev = gp.eval_partial(slot, off, pts, xyz, xyz)
    bits = gp.device_status()
    assert bits & mo.DEV_BAD_POINT
    o = obj.cpu().numpy()
    assert np.isnan(o[0]).all() and np.isfinite(o[1]).all()
    # duplicates and over-long requests
    pts2 = torch.tensor([3, 3, 5, 6], dtype=torch.int32, device=dev)
    gp.eval_partial(slot, off, pts2, xyz, xyz)
    assert gp.device_status() & mo.DEV_DUPLICATE
    off3 = torch.tensor([0, 0, 20], dtype=torch.int32, device=dev)
    pts3 = torch.arange(20, dtype=torch.int32, device=dev)
    xyz3 = torch.zeros((20, 3), dtype=torch.float32, device=dev) + 5.0
    gp.eval_partial(slot, off3, pts3, xyz3, xyz3)
    assert gp.device_status() & mo.DEV_TOO_MANY
    # the handle stays usable
    obj, folded, sev = gpu_full(gp, p.sol_src, p.sol_tgt)
    assert np.isfinite(obj).all() and gp.device_status() == 0


def test_c1_full_size_sampled(mo):
    """The benchmark's configuration: 128x128x96 FP32, 2304 tets, population
    128, full evaluation plus one round of 128 partial requests; the oracle
    checks sampled solutions and requests."""
    p = synth.make_c1()
    n = p.n_solutions
    gp = mo.Problem(p, max_solutions=n, max_requests=n)
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits, trunc_radius=gp.trunc_radius)
    obj, folded, sev = gpu_full(gp, p.sol_src, p.sol_tgt)
    recs = gp.read_records(n)
    res = {}
    for i in (0, 77, 127):
        r = orc.eval(p.sol_src[i], p.sol_tgt[i], with_tets=True)
        res[i] = r
        np.testing.assert_array_equal(recs[i]["n_vox"], r["tets"]["n_vox"])
        np.testing.assert_array_equal(recs[i]["folded"], r["tets"]["folded"])
        assert_obj_close(obj[i], r["obj"], f"c1 solution {i}")
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rd = synth.partial_requests(p, adj, 1, 4, 32, 1.0, 3)[0]
    dv = {k: torch.as_tensor(v).cuda() for k, v in rd.items()}
    pobj, pf, ps = gp.eval_partial(dv["slot"], dv["chg_off"], dv["chg_pts"], dv["chg_src"], dv["chg_tgt"])
    pobj = pobj.cpu().numpy()
    assert gp.device_status() == 0
    off = rd["chg_off"]
    for k in (0, 77):
        ids = rd["chg_pts"][off[k]:off[k + 1]]
        ns, nt = p.sol_src[k].copy(), p.sol_tgt[k].copy()
        ns[ids] = rd["chg_src"][off[k]:off[k + 1]]
        nt[ids] = rd["chg_tgt"][off[k]:off[k + 1]]
        r = orc.eval_partial(p.sol_src[k], p.sol_tgt[k], ns, nt, ids, res[k])
        assert_obj_close(pobj[k], r["obj"], f"c1 request {k}")


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_short_and_long_rows(mo, dtype):
    """One mesh with cells of 1.5 voxels (rows of one or two voxel centres,
    more than 32 row starts in 64 voxels, so the image pass falls back to
    32-voxel windows) beside cells of 24 voxels (long rows, taken 64 voxels
    per window two voxels a lane).  Per-tet sums against the oracle."""
    img_s = random_image((40, 40, 40), 21, dtype=dtype)
    img_t = random_image((40, 40, 40), 22, dtype=dtype)
    axis = np.concatenate([np.arange(-0.5, 15.0, 1.5), [15.5, 39.5]])
    pts, tets = box_lattice(axis, axis, axis)
    rng = np.random.default_rng(23)
    interior = np.all((pts > 0.0) & (pts < 39.0), axis=1)
    n = 2
    src = np.repeat(pts[None], n, axis=0).astype(np.float32)
    tgt = src.copy()
    tgt[:, interior] += rng.uniform(-0.2, 0.2, size=(n, int(interior.sum()), 3)).astype(np.float32)
    prob = problem(img_s, img_t, pts, tets, g_mode=2, sol_src=src, sol_tgt=tgt)
    gp, orc, _ = check_against_oracle(mo, prob)
    recs = gp.read_records(n)
    vox = recs["n_vox"].sum(axis=2)
    assert vox.min() <= 2 and vox.max() > 2000        # both kinds of tets are present
    assert gp.device_status() == 0
