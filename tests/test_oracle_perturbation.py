"""Pins of the oracle's perturbation report (test support for readings R9
and R15): the decisions it marks as open under the FP32 error model of
``helpers.GAMMA_*``, against closed forms and against an independent FP32
evaluation written here in numpy.

- The report never changes a returned value, and is all zero when off.
- An integer translation (map rows in {-1, 0, 1}) is exact in FP32: nothing
  is open, and the labels are those at p + t.
- A doubling map, foreground/background h: a voxel is open exactly when its
  sample is a stored 0 with a nonzero value in the 3x3x3 neighbourhood of
  its mapped position; the spread is |a^2 - 1| (a > 0) or 1 (a = 0).
- A doubling map shifted by half a voxel, labels: every covered voxel's
  mapped x is a half-integer, the exact tie goes to the even neighbour, and
  both neighbours are allowed.
- Soundness: per tet and side, the oracle's sum equals the exact-decision
  sum computed here in rationals (Fraction), and an FP32 evaluation of T(p)
  and of the sample (numpy, no fused operations) changes the case of h only
  at voxels the report counts, and the sum of h by at most the reported
  spread; its nearest voxel is one of the reported candidates.
"""

from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage

import oracle
from helpers import GAMMA_POS, GAMMA_VAL, box_lattice, problem


def _two_level(shape, seed, frac=0.35, lo=20.0, hi=120.0):
    rng = np.random.default_rng(seed)
    v = rng.uniform(lo, hi, size=shape)
    return np.where(rng.random(shape) < frac, v, 0.0).astype(np.float32)


def _full_box(nx, ny, nz, cells=(2, 2, 2)):
    xs = np.linspace(-0.5, nx - 0.5, cells[0] + 1)
    ys = np.linspace(-0.5, ny - 0.5, cells[1] + 1)
    zs = np.linspace(-0.5, nz - 0.5, cells[2] + 1)
    return box_lattice(xs, ys, zs)


def test_report_changes_no_value(oracle_lib):
    nz, ny, nx = 9, 10, 11
    img_s, img_t = _two_level((nz, ny, nx), 1), _two_level((nz, ny, nx), 2)
    pts, tets = _full_box(nx, ny, nz)
    rng = np.random.default_rng(3)
    interior = np.all((pts > -0.5) & (pts < np.array([nx, ny, nz]) - 0.5), axis=1)
    src = pts.copy()
    src[interior] += rng.uniform(-0.7, 0.7, size=(interior.sum(), 3))
    tgt = pts.copy()
    tgt[interior] += rng.uniform(-0.7, 0.7, size=(interior.sum(), 3))
    prob = problem(img_s, img_t, pts, tets, h_mode=1, g_mode=2)
    o = oracle.Oracle(prob)
    off = o.eval(src, tgt, with_tets=True)
    lab = (img_t > 0).astype(np.uint8) + 1
    w_off = o.warp_labels(src, tgt, 0, lab)
    assert (off["tets"]["amb_n"] == 0).all() and (off["tets"]["amb_slack"] == 0).all()
    o.set_perturbation(GAMMA_POS, GAMMA_VAL)
    on = o.eval(src, tgt, with_tets=True)
    w_on, cand = o.warp_labels(src, tgt, 0, lab, candidates=True)
    for f in ("e_img", "e_guid", "n_vox", "e_mag", "sev", "folded"):
        np.testing.assert_array_equal(on["tets"][f], off["tets"][f])
    np.testing.assert_array_equal(on["obj"], off["obj"])
    np.testing.assert_array_equal(w_on, w_off)
    cov = w_on != 255
    assert (cand[cov] == w_on[cov][:, None]).any(-1).all()     # the exact label is a candidate
    assert (cand[~cov] == 255).all()
    o.set_perturbation(0.0, 0.0)
    again = o.eval(src, tgt, with_tets=True)
    assert (again["tets"]["amb_n"] == 0).all()


def _inner_box(nx, ny, nz, cells=(2, 2, 2)):
    """Lattice over [1.5, n - 2.5] per axis: a translation by up to one voxel
    keeps every vertex inside the image (no clamping by R1)."""
    xs = np.linspace(1.5, nx - 2.5, cells[0] + 1)
    ys = np.linspace(1.5, ny - 2.5, cells[1] + 1)
    zs = np.linspace(1.5, nz - 2.5, cells[2] + 1)
    return box_lattice(xs, ys, zs)


@pytest.mark.parametrize("t", [(1, 0, 0), (0, -1, 1), (0, 0, 0)])
def test_integer_translation_is_exact(oracle_lib, t):
    """A translation by whole voxels has map rows in {-1, 0, 1}: FP32
    evaluates it exactly, so the report leaves nothing open, and the labels
    are those at p + t."""
    nz, ny, nx = 8, 9, 10
    img_s, img_t = _two_level((nz, ny, nx), 4), _two_level((nz, ny, nx), 5)
    pts, tets = _inner_box(nx, ny, nz)
    tgt = (pts + np.array(t, np.float32)).astype(np.float32)
    o = oracle.Oracle(problem(img_s, img_t, pts, tets, h_mode=1, g_mode=2))
    o.set_perturbation(GAMMA_POS, GAMMA_VAL)
    r = o.eval(pts, tgt, with_tets=True)
    assert (r["tets"]["amb_n"] == 0).all() and (r["tets"]["amb_slack"] == 0).all()
    k, j, i = np.meshgrid(np.arange(2, nz - 2), np.arange(2, ny - 2), np.arange(2, nx - 2), indexing="ij")
    lab = (np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx) % 7).astype(np.uint8)
    w, cand = o.warp_labels(pts, tgt, 0, lab, candidates=True)
    np.testing.assert_array_equal(w[k, j, i], lab[k + t[2], j + t[1], i + t[0]])
    assert (cand == w[..., None]).all()


def test_doubling_map_closed_form(oracle_lib):
    """T(p) = 2 p (entries 2: not exact by the rule, so eps > 0): every
    mapped position is a grid point, the sample is the stored value there,
    and a voxel is open exactly when that value is 0 and a nonzero value
    lies in the 3x3x3 neighbourhood; the spread is |a^2 - 1| (a > 0) or 1
    (a = 0)."""
    n = 16
    img_s, img_t = _two_level((n, n, n), 4), _two_level((n, n, n), 5)
    pts, tets = box_lattice(*([np.linspace(1.5, 5.5, 3)] * 3))
    tgt = (2.0 * pts).astype(np.float32)
    o = oracle.Oracle(problem(img_s, img_t, pts, tets, h_mode=1, g_mode=2))
    o.set_perturbation(GAMMA_POS, GAMMA_VAL)
    r = o.eval(pts, tgt, with_tets=True)
    k, j, i = np.meshgrid(*([np.arange(2, 6)] * 3), indexing="ij")     # covered source voxels
    assert r["tets"]["n_vox"][:, 0].sum() == i.size
    b = img_t[2 * k, 2 * j, 2 * i].astype(np.float64)
    near = ndimage.maximum_filter((img_t != 0).astype(np.uint8), size=3, mode="constant")[2 * k, 2 * j, 2 * i] > 0
    amb = (b == 0) & near
    a = img_s[k, j, i].astype(np.float64)
    spread = np.where(a > 0, np.abs(a * a - 1.0), np.where(a == 0, 1.0, 0.0))
    assert amb.sum() > 0
    assert r["tets"]["amb_n"][:, 0].sum() == amb.sum()
    assert r["tets"]["amb_slack"][:, 0].sum() == pytest.approx(spread[amb].sum(), rel=1e-12)
    h = np.where((a > 0) & (b > 0), (a - b) ** 2, np.where((a == 0) & (b == 0), 0.0, 1.0))
    assert r["tets"]["e_img"][:, 0].sum() == pytest.approx(h.sum(), rel=1e-12)


def test_half_voxel_labels_closed_form(oracle_lib):
    """T(p) = 2 p + (1/2, 0, 0): x lands exactly on half-integers, where the
    exact tie goes to the even neighbour 2x and the report allows both 2x
    and 2x + 1; y and z land on grid points and stay fixed."""
    n = 16
    img = _two_level((n, n, n), 6)
    pts, tets = box_lattice(*([np.linspace(1.5, 5.5, 3)] * 3))
    tgt = (2.0 * pts + np.array([0.5, 0.0, 0.0])).astype(np.float32)
    o = oracle.Oracle(problem(img, img, pts, tets, g_mode=2))
    o.set_perturbation(GAMMA_POS, GAMMA_VAL)
    lab = np.random.default_rng(7).integers(0, 9, size=(n, n, n)).astype(np.uint8)
    w, cand = o.warp_labels(pts, tgt, 0, lab, candidates=True)
    k, j, i = np.meshgrid(*([np.arange(2, 6)] * 3), indexing="ij")
    np.testing.assert_array_equal(w[k, j, i], lab[2 * k, 2 * j, 2 * i])
    c = cand[k, j, i]                                  # slot bit 0 = the x choice
    assert (c[..., 0::2] == lab[2 * k, 2 * j, 2 * i][..., None]).all()
    assert (c[..., 1::2] == lab[2 * k, 2 * j, 2 * i + 1][..., None]).all()
    assert (w[:, :, :2] == 255).all() and (cand[:, :, :2] == 255).all()     # not covered


# ---------------------------------------------------------------------------
# soundness against an independent FP32 evaluation
# ---------------------------------------------------------------------------

def _trilinear(img, y, dt):
    """Trilinear sample of ``img`` at y (x, y, z) in dtype dt, reading R4's
    clamping and cells, lerps as v0 + f (v1 - v0) without fused operations."""
    n = np.array(img.shape[::-1])[:, None]
    c = np.minimum(np.maximum(y.astype(dt), dt(0)), (n - 1).astype(dt))
    i0 = np.minimum(np.floor(c).astype(np.int64), n - 2)
    f = (c - i0.astype(dt)).astype(dt)
    v = img.astype(dt)

    def g(dx, dy, dz):
        return v[i0[2] + dz, i0[1] + dy, i0[0] + dx]

    def lerp(a, b, t):
        return (a + t * (b - a)).astype(dt)

    c00 = lerp(g(0, 0, 0), g(1, 0, 0), f[0])
    c10 = lerp(g(0, 1, 0), g(1, 1, 0), f[0])
    c01 = lerp(g(0, 0, 1), g(1, 0, 1), f[0])
    c11 = lerp(g(0, 1, 1), g(1, 1, 1), f[0])
    return lerp(lerp(c00, c10, f[1]), lerp(c01, c11, f[1]), f[2])


def _exact_sample(img, own, oth, v, S):
    """Trilinear sample (R4) at the exact T(p) of voxel centre v, in
    rationals: lambda_i = D_i(p) / D, w_i = q_i / S - 1/2."""
    p = [v[0] * S + S // 2, v[1] * S + S // 2, v[2] * S + S // 2]
    D = oracle.orient(*own)
    y = [Fraction(-1, 2)] * 3
    for i in range(4):
        w = list(own)
        w[i] = p
        Di = oracle.orient(*w)
        for ax in range(3):
            y[ax] += Fraction(Di * int(oth[i][ax]), D * S)
    n = img.shape[::-1]
    i0, f = [], []
    for ax in range(3):
        c = min(max(y[ax], Fraction(0)), Fraction(n[ax] - 1))
        i = min(int(c.numerator // c.denominator), n[ax] - 2)
        i0.append(i)
        f.append(c - i)
    b = Fraction(0)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                wgt = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                if wgt:
                    b += wgt * Fraction(float(img[i0[2] + dz, i0[1] + dy, i0[0] + dx]))
    return b


def _case(a, b):
    return np.where((a > 0) & (b > 0), 2, np.where((a == 0) & (b == 0), 1, 0))


def _hval(a, b, case):
    return np.where(case == 2, (a - b) ** 2, np.where(case == 1, 0.0, 1.0))


def _soundness_case(seed, scale_map):
    rng = np.random.default_rng(seed)
    if scale_map:
        # one tet mapped by T(p) = t0 + M (p - s0), M = diag(-0.6, -0.6, 0.6):
        # every vertex is on the grid, so T(p) is exactly integer (or, with
        # the offset, exactly half-integer) in an axis whenever that axis of
        # p - s0 is a multiple of 5.  FP32 rounds 0.6 and the products, so
        # near |p - s0| ~ 45 it lands just off those values: the case of h
        # (zero stored values beside nonzero ones) and the nearest voxel move.
        n = 64
        img_s, img_t = _two_level((n, n, n), 31 + seed), _two_level((n, n, n), 41 + seed)
        s0 = np.array([58.0, 58.0, 2.0])
        src = np.array([s0, [8, 58, 2], [58, 8, 2], [58, 58, 12]], np.float64)
        t0 = np.array([3.0 + 0.5 * (seed % 2), 3.0, 2.0])
        tgt = t0 + (src - s0) * np.array([-0.6, -0.6, 0.6])
        prob = problem(img_s, img_t, src.astype(np.float32), np.array([[0, 1, 2, 3]], np.int32), h_mode=1,
                       g_mode=2)
        return prob, src.astype(np.float32), tgt.astype(np.float32)
    nz, ny, nx = 10, 9, 11
    img_s, img_t = _two_level((nz, ny, nx), 10 + seed), _two_level((nz, ny, nx), 20 + seed)
    pts, tets = _full_box(nx, ny, nz)
    interior = np.all((pts > -0.5) & (pts < np.array([nx, ny, nz]) - 0.5), axis=1)
    src = pts.copy()
    src[interior] += rng.uniform(-0.8, 0.8, size=(interior.sum(), 3))
    tgt = pts.copy()
    tgt[interior] += rng.uniform(-0.8, 0.8, size=(interior.sum(), 3))
    return problem(img_s, img_t, pts, tets, h_mode=1, g_mode=2), src.astype(np.float32), tgt.astype(np.float32)


@pytest.mark.parametrize("seed,scale_map", [(0, False), (1, False), (2, True), (3, True)])
def test_report_covers_an_fp32_evaluation(oracle_lib, seed, scale_map):
    prob, src, tgt = _soundness_case(seed, scale_map)
    o = oracle.Oracle(prob)
    o.set_perturbation(GAMMA_POS, GAMMA_VAL)
    r = o.eval(src, tgt, with_tets=True)
    tt = o.oriented_tets()
    S = 256
    q = {0: np.array([[oracle.snap1(float(x), n, 8) for x, n in zip(v, (prob.nx, prob.ny, prob.nz))] for v in src]),
         1: np.array([[oracle.snap1(float(x), n, 8) for x, n in zip(v, (prob.nx, prob.ny, prob.nz))] for v in tgt])}
    imgs = {0: prob.image_s, 1: prob.image_t}
    lab = np.random.default_rng(seed).integers(0, 5, size=prob.image_t.shape).astype(np.uint8)
    _, cand = o.warp_labels(src, tgt, 0, lab, candidates=True)
    n_xyz = np.array([prob.nx, prob.ny, prob.nz])
    mismatches = label_moves = 0
    for t in range(len(tt)):
        for side in (0, 1):
            own, oth = q[side][tt[t]], q[1 - side][tt[t]]
            if oracle.orient(*own) <= 0:
                continue
            ov, tv = own / S - 0.5, oth / S - 0.5             # voxel units
            E = (ov[1:] - ov[0]).T
            F = (tv[1:] - tv[0]).T
            M64 = F @ np.linalg.inv(E)
            M32 = M64.astype(np.float32)
            lo = np.maximum(np.ceil(ov.min(0)).astype(int), 0)
            hi = np.minimum(np.floor(ov.max(0)).astype(int), [prob.nx - 1, prob.ny - 1, prob.nz - 1])
            tet12 = own.reshape(12)
            vox = [(i, j, k) for k in range(lo[2], hi[2] + 1) for j in range(lo[1], hi[1] + 1)
                   for i in range(lo[0], hi[0] + 1)
                   if oracle.inside(tet12, [i * S + S // 2, j * S + S // 2, k * S + S // 2])]
            if not vox:
                continue
            p = np.array(vox, np.float64)
            y64 = tv[0] + (p - ov[0]) @ M64.T            # nearest voxel only; the sample is exact below
            d32 = (p - ov[0]).astype(np.float32)
            y32 = tv[0].astype(np.float32) + (d32[:, :, None] * M32.T[None]).astype(np.float32).sum(1, dtype=np.float32)
            a = imgs[side][p[:, 2].astype(int), p[:, 1].astype(int), p[:, 0].astype(int)].astype(np.float64)
            oth_img = imgs[1 - side]
            b32 = _trilinear(oth_img, y32.T.astype(np.float32), np.float32).astype(np.float64)
            if side == 0:                  # nearest voxel of the FP32 position (R15)
                m32 = np.clip(np.rint(y32), 0, n_xyz - 1).astype(int)
                m64 = np.clip(np.rint(y64), 0, n_xyz - 1).astype(int)
                label_moves += int((m32 != m64).any(1).sum())
                l32 = lab[m32[:, 2], m32[:, 1], m32[:, 0]]
                cv = cand[p[:, 2].astype(int), p[:, 1].astype(int), p[:, 0].astype(int)]
                assert (cv == l32[:, None]).any(1).all(), (t, "label outside the reported candidates")
            # the exact sample, in rationals: T(p) = sum_i D_i(p) w_i / D
            bx = np.array([_exact_sample(oth_img, own, oth, v, S) for v in vox], dtype=object)
            cx = np.array([2 if (ai > 0 and bi > 0) else 1 if (ai == 0 and bi == 0) else 0
                           for ai, bi in zip(a, bx)])
            bxf = bx.astype(np.float64)
            c32 = _case(a, b32)
            diff = int((cx != c32).sum())
            mismatches += diff
            rec = r["tets"][t]
            # the oracle's sum is the exact-decision one
            assert _hval(a, bxf, cx).sum() == pytest.approx(rec["e_img"][side], rel=1e-12, abs=1e-9)
            # an FP32 evaluation moves only reported decisions, by at most the reported spread
            assert diff <= rec["amb_n"][side], (t, side, diff, rec["amb_n"][side])
            e32 = _hval(a, bxf, c32).sum()
            assert abs(e32 - rec["e_img"][side]) <= rec["amb_slack"][side] + 1e-9 * (1 + abs(rec["e_img"][side]))
    print(f"case decisions moved by FP32: {mismatches}; nearest voxels moved: {label_moves}")
    if scale_map:                          # the constructed maps must exercise the report
        assert (label_moves if seed % 2 else mismatches) > 0
