"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to a library routine, a closed form, an
exact-rational computation or an invariant of the mathematics, chosen so that
a plausible slip (dropped term, wrong sign, transposed operand, wrong spoke
edges, off-by-one in the voxel association) fails at least one of them.

Oracle function            pinned by
-------------------------  -----------------------------------------------
snap (R1)                  hand-computed half-even ties, clamping
orient (R2)                numpy.linalg.det, unit-tet volume, odd swaps
inside_sos (R3)            exact rational perturbation p + (e, e^2, e^3)
coverage (R3)              each voxel centre in exactly one tet (ties on
                           vertices/faces), sum of counts = voxel count
trilinear (R4)             scipy.ndimage.map_coordinates(order=1, nearest)
h, both modes              closed forms on two-level images
barycentric map            global affine deformation vs scipy sampling and
                           two different tetrahedralisations
f_intensity                identity = numpy mean SSD; linear image under a
                           translation = (a.t)^2
f_magnitude (R5)           scaling closed form via sum(spokes^2) =
                           sum(edges^2)/4; rigid translation / 90-degree
                           rotation give exactly 0; tissue factor scales
distance maps (R7)         scipy.spatial.cKDTree
f_guidance continuous      identity and translation closed forms built on
                           cKDTree maps and scipy sampling
f_guidance pair (R8)       translation with dyadic offsets: mean |e|^2
fold + severity (R2, R6)   vertex pushed through the opposite face: flips
                           exactly at the crossing; |det|/6 from numpy
partial evaluation         equals a fresh full evaluation
"""

from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage, spatial

import synth
from helpers import box_lattice, problem, random_image

S8 = 256


@pytest.fixture(scope="module")
def orc(oracle_lib):
    return oracle_lib


# ---------------------------------------------------------------------------
# R1 snap
# ---------------------------------------------------------------------------

def test_snap_ties_and_clamp(orc):
    n = 32
    assert orc.snap1(-0.5, n, 8) == 0
    assert orc.snap1(n - 0.5, n, 8) == n * S8
    assert orc.snap1(-3.0, n, 8) == 0
    assert orc.snap1(1e9, n, 8) == n * S8
    assert orc.snap1(0.0, n, 8) == 128          # voxel centre 0 -> (0 + 1/2) 2^8
    assert orc.snap1(5.0, n, 8) == 5 * 256 + 128
    # exact ties (x + 1/2) 2^8 = m + 1/2 go to the even neighbour
    for m in (10, 11, 12, 13, 200, 201):
        x = (m + 0.5) / 256.0 - 0.5
        assert np.float32(x) == x
        want = m if m % 2 == 0 else m + 1
        assert orc.snap1(x, n, 8) == want, m
    assert orc.snap1(float("nan"), n, 8) == 0   # NaN clamps to the low face


# ---------------------------------------------------------------------------
# R2 orientation
# ---------------------------------------------------------------------------

def test_orient_matches_numpy_det(orc):
    rng = np.random.default_rng(1)
    for _ in range(300):
        v = rng.integers(-50, 50, size=(4, 3))
        want = np.linalg.det((v[1:] - v[0]).astype(np.float64))
        got = orc.orient(v[0], v[1], v[2], v[3])
        assert got == int(round(want))
        assert orc.orient(v[1], v[0], v[2], v[3]) == -got
        assert orc.orient(v[0], v[2], v[3], v[1]) == got     # even permutation
    assert orc.orient([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]) == 1


# ---------------------------------------------------------------------------
# R3 inside test with ties
# ---------------------------------------------------------------------------

def _det3(m):
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def _orient_frac(a, b, c, d):
    return _det3([[b[i] - a[i] for i in range(3)], [c[i] - a[i] for i in range(3)],
                  [d[i] - a[i] for i in range(3)]])


def _inside_perturbed(v, p):
    eps = Fraction(1, 2 ** 60)
    pp = (Fraction(int(p[0])) + eps, Fraction(int(p[1])) + eps ** 2, Fraction(int(p[2])) + eps ** 3)
    for i in range(4):
        w = [tuple(Fraction(int(c)) for c in x) for x in v]
        w[i] = pp
        if _orient_frac(*w) <= 0:
            return False
    return True


def test_inside_sos_matches_rational_perturbation(orc):
    rng = np.random.default_rng(2)
    checked = 0
    while checked < 40:
        v = rng.integers(0, 7, size=(4, 3))
        d = orc.orient(*v)
        if d == 0:
            continue
        if d < 0:
            v = v[[0, 1, 3, 2]]
        checked += 1
        lo, hi = v.min(0), v.max(0)
        for x in range(lo[0] - 1, hi[0] + 2):
            for y in range(lo[1] - 1, hi[1] + 2):
                for z in range(lo[2] - 1, hi[2] + 2):
                    p = (x, y, z)
                    assert orc.inside(v, p) == _inside_perturbed([tuple(r) for r in v], p), (v, p)


def _snap_all(orc, pts, shape_xyz, k=8):
    return np.array([[orc.snap1(float(c), shape_xyz[a], k) for a, c in enumerate(p)] for p in pts],
                    dtype=np.int64)


@pytest.mark.parametrize("flip", [False, True])
def test_each_voxel_centre_in_exactly_one_tet(orc, flip):
    # vertices on voxel centres and faces through rows of voxel centres
    nx, ny, nz = 12, 10, 9
    xs = [-0.5, 3.0, 7.0, 11.5]
    ys = [-0.5, 4.0, 9.5]
    zs = [-0.5, 2.0, 5.0, 8.5]
    pts, tets = box_lattice(xs, ys, zs, flip_x=flip)
    rng = np.random.default_rng(3)
    # move interior vertices to other voxel centres / half-voxel positions (ties)
    interior = np.all((pts > -0.5) & (pts < np.array([nx, ny, nz]) - 0.5), axis=1)
    pts = pts.copy()
    pts[interior] += rng.integers(-1, 2, size=(interior.sum(), 3)) * 0.5
    q = _snap_all(orc, pts, (nx, ny, nz))
    tq = q[tets]
    for t in range(len(tets)):
        if orc.orient(*tq[t]) < 0:
            tq[t] = tq[t][[0, 1, 3, 2]]
        assert orc.orient(*tq[t]) > 0
    H = S8 // 2
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = (i * S8 + H, j * S8 + H, k * S8 + H)
                c = sum(orc.inside(tq[t], p) for t in range(len(tets)))
                assert c == 1, (i, j, k, c)
    img = random_image((nz, ny, nx), 4)
    prob = problem(img, img, pts, tets)
    o = orc.Oracle(prob)
    r = o.eval(pts, pts, with_tets=True)
    assert r["n_vox"] == 2 * nx * ny * nz
    assert int(r["tets"]["n_vox"][:, 0].sum()) == nx * ny * nz


# ---------------------------------------------------------------------------
# R4 trilinear sampling, h
# ---------------------------------------------------------------------------

def test_trilinear_matches_scipy(orc):
    img = random_image((5, 6, 7), 5).astype(np.float64)
    rng = np.random.default_rng(6)
    ys = rng.uniform(-1.5, 8.0, size=(400, 3))
    ys[:20] = np.floor(ys[:20])              # integer positions, including the last cell
    ys[20] = [6.0, 5.0, 4.0]
    for y in ys:
        want = ndimage.map_coordinates(img, [[y[2]], [y[1]], [y[0]]], order=1, mode="nearest")[0]
        assert orc.trilinear(img, y) == pytest.approx(want, rel=1e-12, abs=1e-9)


def test_h_modes_closed_form(orc):
    # identity mesh: each side contributes sum_p h(I_s(p), I_t(p)); the
    # two-level images give 0 / 1 / (30-50)^2 per column by construction
    nx, ny, nz = 16, 4, 3
    img_s = np.zeros((nz, ny, nx), np.float32)
    img_t = np.zeros((nz, ny, nx), np.float32)
    img_s[:, :, 6:] = 30.0
    img_t[:, :, 8:] = 50.0
    pts, tets = box_lattice([-0.5, 7.5, 15.5], [-0.5, 3.5], [-0.5, 2.5])
    prob = problem(img_s, img_t, pts, tets, h_mode=1, g_mode=2)
    r = orc.Oracle(prob).eval(pts, pts)
    assert r["obj"][0] == pytest.approx((2 * 1 + 8 * 400) / 16.0, rel=1e-15)
    prob0 = problem(img_s, img_t, pts, tets, h_mode=0, g_mode=2)
    r0 = orc.Oracle(prob0).eval(pts, pts)
    assert r0["obj"][0] == pytest.approx((2 * 900 + 8 * 400) / 16.0, rel=1e-15)
    # negative intensities fall in the "otherwise" case
    img_s2 = img_s.copy()
    img_s2[:, :, :6] = -5.0
    r2 = orc.Oracle(problem(img_s2, img_t, pts, tets, h_mode=1, g_mode=2)).eval(pts, pts)
    assert r2["obj"][0] == pytest.approx((8 * 1 + 8 * 400) / 16.0, rel=1e-15)
    assert orc.h(1, 0.0, 0.0) == 0.0 and orc.h(1, 2.0, 0.0) == 1.0 and orc.h(1, 3.0, 1.0) == 4.0


# ---------------------------------------------------------------------------
# f_intensity and the barycentric map
# ---------------------------------------------------------------------------

def test_identity_c0(orc):
    p = synth.make_c0(n_sol=1)
    o = orc.Oracle(p)
    r = o.eval(p.ref_points, p.ref_points, with_tets=True)
    ssd = ((p.image_s.astype(np.float64) - p.image_t.astype(np.float64)) ** 2).mean()
    assert r["obj"][1] == 0.0
    assert r["obj"][0] == pytest.approx(ssd, rel=1e-12)
    assert r["n_vox"] == 2 * p.voxels()
    assert r["folded"] == 0 and r["severity"] == 0.0


def test_linear_image_translation_closed_form(orc):
    nx, ny, nz = 28, 26, 24
    a = np.array([0.5, -1.25, 2.0])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    img = (a[0] * x + a[1] * y + a[2] * z + 3.0).astype(np.float32)
    pts, tets = box_lattice([4.0, 12.0, 20.0], [4.0, 12.0, 20.0], [4.0, 12.0, 20.0])
    t = np.array([1.5, -0.75, 0.375])
    prob = problem(img, img, pts, tets, g_mode=2)
    r = orc.Oracle(prob).eval(pts, pts + t.astype(np.float32))
    assert r["n_vox"] == 2 * 16 ** 3
    assert r["obj"][0] == pytest.approx(float(a @ t) ** 2, rel=1e-12)
    assert r["obj"][1] == 0.0


def _affine_case(flip):
    nx, ny, nz = 30, 28, 26
    img_s = random_image((nz, ny, nx), 7)
    img_t = ndimage.gaussian_filter(random_image((nz, ny, nx), 8), 1.5).astype(np.float32)
    xs = [4.0, 12.0, 20.0]
    pts, tets = box_lattice(xs, xs, xs, flip_x=flip)
    A = np.array([[1.0 + 1 / 16, 1 / 32, 0.0], [-1 / 32, 1.0 - 1 / 16, 1 / 32], [0.0, 1 / 16, 1.0]])
    b = np.array([0.75 + 1 / 256, -0.5 + 3 / 256, 1.25 + 5 / 256])
    tgt = (pts.astype(np.float64) @ A.T + b)
    assert np.all(np.round(tgt * 256) == tgt * 256)
    return img_s, img_t, pts, tets, A, b, tgt.astype(np.float32)


def test_global_affine_map_closed_form_and_mesh_independence(orc):
    img_s, img_t, pts, tets, A, b, tgt = _affine_case(False)
    nz, ny, nx = img_s.shape
    r1 = orc.Oracle(problem(img_s, img_t, pts, tets, g_mode=2)).eval(pts, tgt)
    _, _, pts2, tets2, _, _, tgt2 = _affine_case(True)
    r2 = orc.Oracle(problem(img_s, img_t, pts2, tets2, g_mode=2)).eval(pts2, tgt2)
    assert r1["n_vox"] == r2["n_vox"]
    assert r1["obj"][0] == pytest.approx(r2["obj"][0], rel=1e-12)
    # independent closed form: side 0 over the source box, side 1 over A.box + b
    Is = img_s.astype(np.float64)
    It = img_t.astype(np.float64)
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1)
    g = g.reshape(-1, 3).astype(np.float64)
    in_s = np.all((g >= 4.0) & (g < 20.0), axis=1)
    ps = g[in_s]
    ys = ps @ A.T + b
    s0 = ((Is[ps[:, 2].astype(int), ps[:, 1].astype(int), ps[:, 0].astype(int)]
           - ndimage.map_coordinates(It, [ys[:, 2], ys[:, 1], ys[:, 0]], order=1, mode="nearest")) ** 2).sum()
    pre = (g - b) @ np.linalg.inv(A).T
    in_t = np.all((pre > 4.0) & (pre < 20.0), axis=1)
    assert not np.any(np.isclose(pre, 4.0) | np.isclose(pre, 20.0))
    qt = g[in_t]
    back = pre[in_t]
    s1 = ((It[qt[:, 2].astype(int), qt[:, 1].astype(int), qt[:, 0].astype(int)]
           - ndimage.map_coordinates(Is, [back[:, 2], back[:, 1], back[:, 0]], order=1, mode="nearest")) ** 2).sum()
    assert r1["n_vox"] == in_s.sum() + in_t.sum()
    assert r1["obj"][0] == pytest.approx((s0 + s1) / (in_s.sum() + in_t.sum()), rel=1e-11)


# ---------------------------------------------------------------------------
# f_magnitude
# ---------------------------------------------------------------------------

def test_magnitude_scaling_closed_form(orc):
    img = np.zeros((40, 40, 40), np.float32)
    tet_pts = np.array([[3.0, 4.0, 5.0], [13.0, 5.0, 6.0], [5.0, 15.0, 7.0], [6.0, 7.0, 17.0]], np.float32)
    tets = np.array([[0, 1, 2, 3]], np.int32)
    for s, c in ((1.5, 1.0), (0.75, 3.5)):
        tgt = (tet_pts.astype(np.float64) * s).astype(np.float32)
        assert np.all(np.round(tgt * 256) == tgt * 256)
        prob = problem(img, img, tet_pts, tets, tissue=[c], g_mode=2)
        r = orc.Oracle(prob).eval(tet_pts, tgt)
        e6 = sum(float(np.sum((tet_pts[j] - tet_pts[i]).astype(np.float64) ** 2))
                 for i in range(4) for j in range(i + 1, 4))
        # spokes: sum_i |v_i - centroid|^2 = (1/4) sum_edges |v_i - v_j|^2
        want = c * (1.0 - s) ** 2 * (e6 * 1.25) / 10.0
        assert r["obj"][1] == pytest.approx(want, rel=1e-12)


def test_magnitude_rigid_motions_are_zero(orc):
    # interior jittered mesh (nothing clamped) translated by a grid multiple
    img = np.zeros((40, 40, 40), np.float32)
    pts, tets = box_lattice([8.0, 14.0, 20.0], [8.0, 14.0, 20.0], [8.0, 14.0, 20.0])
    rng = np.random.default_rng(13)
    src = (pts + rng.uniform(-1, 1, size=pts.shape)).astype(np.float32)
    shift = np.array([3 / 256, -5 / 256, 17 / 256], np.float32)
    r = orc.Oracle(problem(img, img, pts, tets, g_mode=2)).eval(src, src + shift)
    assert r["obj"][1] == 0.0
    # interior mesh rotated by 90 degrees about a grid point
    c = np.array([14.0, 14.0, 14.0])
    rot = ((pts - c) @ np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]).T + c).astype(np.float32)
    r2 = orc.Oracle(problem(img, img, pts, tets, g_mode=2)).eval(pts, rot)
    assert r2["obj"][1] == 0.0


# ---------------------------------------------------------------------------
# guidance
# ---------------------------------------------------------------------------

def _guid_problem(g_mode, r=4.0):
    nx, ny, nz = 24, 22, 20
    img_s = random_image((nz, ny, nx), 9)
    img_t = random_image((nz, ny, nx), 10)
    pts, tets = box_lattice([3.0, 11.0, 19.0], [3.0, 10.0, 17.0], [3.0, 9.0, 15.0])
    rng = np.random.default_rng(11)
    gs = rng.uniform(6.0, 14.0, size=(30, 3)).astype(np.float32)
    gt = (gs + rng.normal(0, 0.7, size=gs.shape)).astype(np.float32)
    grp = (np.arange(30) % 3).astype(np.int32)
    return problem(img_s, img_t, pts, tets, guid_s=gs, guid_t=gt, guid_group=grp,
                   trunc_radius=r, g_mode=g_mode)


def _kdtree_maps(prob, side):
    pts = prob.guid_s if side == 0 else prob.guid_t
    g = np.stack(np.meshgrid(np.arange(prob.nz), np.arange(prob.ny), np.arange(prob.nx), indexing="ij"), -1)
    xyz = g[..., ::-1].reshape(-1, 3).astype(np.float64)
    out = []
    for k in range(int(prob.guid_group.max()) + 1):
        tree = spatial.cKDTree(pts[prob.guid_group == k].astype(np.float64))
        d, _ = tree.query(xyz)
        out.append(d.reshape(prob.nz, prob.ny, prob.nx))
    return out


def test_distance_maps_match_kdtree(orc):
    prob = _guid_problem(0)
    o = orc.Oracle(prob)
    for side in (0, 1):
        want = _kdtree_maps(prob, side)
        for k in range(3):
            np.testing.assert_allclose(o.distance_map(side, k), want[k], rtol=0, atol=1e-12)


def test_guidance_continuous_translation_closed_form(orc):
    prob = _guid_problem(0)
    o = orc.Oracle(prob)
    pts = prob.ref_points
    t = np.array([0.5, -0.25, 0.75])
    r = o.eval(pts, (pts + t).astype(np.float32))
    Ds, Dt = _kdtree_maps(prob, 0), _kdtree_maps(prob, 1)
    w = np.bincount(prob.guid_group) / len(prob.guid_group)
    rr = prob.trunc_radius

    def side_sum(own_maps, oth_maps, lo, hi, shift):
        tot = 0.0
        zz, yy, xx = np.meshgrid(np.arange(prob.nz), np.arange(prob.ny), np.arange(prob.nx), indexing="ij")
        m = (xx >= lo[0]) & (xx < hi[0]) & (yy >= lo[1]) & (yy < hi[1]) & (zz >= lo[2]) & (zz < hi[2])
        for k in range(3):
            a = own_maps[k][m]
            sel = a < rr
            c = [zz[m][sel] + shift[2], yy[m][sel] + shift[1], xx[m][sel] + shift[0]]
            d = ndimage.map_coordinates(oth_maps[k], c, order=1, mode="nearest")
            tot += w[k] * np.sum((rr - a[sel]) / rr * (a[sel] - d) ** 2)
        return tot, int(m.sum())

    lo = np.array([3.0, 3.0, 3.0])
    hi = np.array([19.0, 17.0, 15.0])
    s0, n0 = side_sum(Ds, Dt, lo, hi, t)
    s1, n1 = side_sum(Dt, Ds, np.ceil(lo + t), np.ceil(hi + t), -t)
    assert r["n_vox"] == n0 + n1
    assert r["obj"][2] == pytest.approx((s0 + s1) / (n0 + n1), rel=1e-11)


def test_guidance_pair_transfer_closed_form(orc):
    prob = _guid_problem(1)
    rng = np.random.default_rng(12)
    t = np.array([1.25, -0.5, 0.75])
    gs = (np.round(rng.uniform(6.0, 13.0, size=(30, 3)) * 256) / 256)
    e = np.round(rng.normal(0, 0.5, size=gs.shape) * 256) / 256
    gt = gs + t + e
    prob.guid_s = gs.astype(np.float32)
    prob.guid_t = gt.astype(np.float32)
    o = orc.Oracle(prob)
    pts = prob.ref_points
    r = o.eval(pts, (pts + t).astype(np.float32))
    assert r["n_gp"] == 60
    assert r["obj"][2] == pytest.approx(float(np.mean(np.sum(e ** 2, axis=1))), rel=1e-12)


# ---------------------------------------------------------------------------
# fold constraint
# ---------------------------------------------------------------------------

def test_fold_flip_at_crossing_and_severity(orc):
    img = np.zeros((20, 20, 20), np.float32)
    base = np.array([[2.0, 2.0, 8.0], [12.0, 2.0, 8.0], [2.0, 12.0, 8.0], [4.0, 4.0, 12.0]])
    tets = np.array([[0, 1, 2, 3]], np.int32)
    prob = problem(img, img, base.astype(np.float32), tets, g_mode=2)
    o = orc.Oracle(prob)
    for dz in np.arange(-6.0, 6.0 + 1e-9, 0.25):
        tgt = base.copy()
        tgt[3, 2] = 8.0 + dz                 # apex pushed through the base plane z = 8
        r = o.eval(base.astype(np.float32), tgt.astype(np.float32), with_tets=True)
        vol = np.linalg.det(tgt[1:] - tgt[0]) / 6.0
        assert r["folded"] == (1 if dz <= 0 else 0)
        assert r["tets"]["folded"][0] == (2 if dz <= 0 else 0)
        assert r["severity"] == pytest.approx(abs(vol) if dz <= 0 else 0.0, abs=1e-12)
        if dz <= 0:
            assert r["tets"]["n_vox"][0, 1] == 0          # a folded copy is not rasterised


def test_reference_orientation_is_normalised(orc):
    p = synth.make_c0(n_sol=1)
    rev = p.tets[:, ::-1].copy()
    a = orc.Oracle(p).eval(p.sol_src[0], p.sol_tgt[0])
    b = orc.Oracle(p, tets=rev).eval(p.sol_src[0], p.sol_tgt[0])
    assert a["n_vox"] == b["n_vox"]
    np.testing.assert_allclose(a["obj"], b["obj"], rtol=1e-12)


def test_setup_rejects_bad_problems(orc):
    p = synth.make_c0(n_sol=1)
    with pytest.raises(orc.OracleError):
        orc.Oracle(p, tets=np.array([[0, 1, 2, 2]], np.int32))        # degenerate
    with pytest.raises(orc.OracleError):
        orc.Oracle(p, tet_label=np.full(p.n_tets, 9, np.int32))       # label out of range
    with pytest.raises(orc.OracleError):
        orc.Oracle(p, subvoxel_bits=12)                                 # 32 * 2^12 > 2^16


# ---------------------------------------------------------------------------
# partial evaluation
# ---------------------------------------------------------------------------

def test_partial_equals_full(orc):
    p = synth.make_c0(n_sol=2)
    o = orc.Oracle(p)
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    src, tgt = p.sol_src[0].copy(), p.sol_tgt[0].copy()
    cur = o.eval(src, tgt)
    for rd in synth.partial_requests(p, adj, 6, 4, 20, 1.0, 3, slots=np.array([0])):
        ns, nt = src.copy(), tgt.copy()
        ns[rd["chg_pts"]] = rd["chg_src"]
        nt[rd["chg_pts"]] = rd["chg_tgt"]
        part = o.eval_partial(src, tgt, ns, nt, rd["chg_pts"], cur)
        full = o.eval(ns, nt)
        assert part["n_vox"] == full["n_vox"] and part["n_folded"] == full["n_folded"]
        assert part["sev_raw"] == full["sev_raw"]
        np.testing.assert_allclose(part["obj"], full["obj"], rtol=1e-12)
        assert 0 < part["n_affected"] < p.n_tets
        src, tgt, cur = ns, nt, part
