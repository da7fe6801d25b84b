"""Pins of the surface-distance oracle (reading R17, the Hausdorff distance
and its 95th percentile of Sec. 5) and of the warped label image.

The directed distances are checked against scipy's exact Euclidean
distance transform (an independent library routine), the Hausdorff
distance against hand-derived values on boxes and single voxels, and the
nearest-rank percentile on a distance multiset built by hand."""

import math

import numpy as np
import pytest

import oracle
import synth
from oracle import surface as sd

ndimage = pytest.importorskip("scipy.ndimage")


def box(shape, lo, hi):
    m = np.zeros(shape, bool)
    m[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = True
    return m


def test_surface_of_a_box_is_its_shell():
    m = box((12, 12, 12), (2, 2, 2), (8, 8, 8))
    s = sd.surface(m)
    assert s.sum() == 7 ** 3 - 5 ** 3
    assert not s[3:8, 3:8, 3:8].any()


def test_mask_touching_the_border_keeps_its_border_face():
    m = np.ones((4, 5, 6), bool)
    s = sd.surface(m)
    assert s.sum() == 4 * 5 * 6 - 2 * 3 * 4


def test_directed_distances_equal_the_exact_edt():
    rng = np.random.default_rng(3)
    a = rng.random((20, 22, 24)) < 0.3
    b = ndimage.binary_opening(rng.random((20, 22, 24)) < 0.6)
    sa, sb = sd.surface(a), sd.surface(b)
    want = ndimage.distance_transform_edt(~sb) ** 2
    got = sd.directed_sq(np.argwhere(sa), np.argwhere(sb))
    np.testing.assert_array_equal(got, np.rint(want[sa]).astype(np.int64))


def test_nested_boxes():
    # A = [10, 20]^3 inside B = [8, 22]^3: every A surface voxel is 2 from B's
    # shell; B's corners are sqrt(12) from A's corners
    a = box((32, 32, 32), (10, 10, 10), (20, 20, 20)).astype(np.uint8)
    b = box((32, 32, 32), (8, 8, 8), (22, 22, 22)).astype(np.uint8)
    hd, hd95, na, nb = sd.hausdorff(a, b, 1)
    assert hd == math.sqrt(12.0)
    assert na == 11 ** 3 - 9 ** 3 and nb == 15 ** 3 - 13 ** 3
    dab = sd.directed_sq(np.argwhere(sd.surface(a == 1)), np.argwhere(sd.surface(b == 1)))
    assert (dab == 4).all()


def test_box_shifted_along_x():
    a = box((32, 32, 32), (10, 10, 10), (20, 20, 20)).astype(np.uint8)
    b = box((32, 32, 32), (13, 10, 10), (23, 20, 20)).astype(np.uint8)
    hd, _, _, _ = sd.hausdorff(a, b, 1)
    assert hd == 3.0


def test_single_voxels():
    a = np.zeros((9, 10, 11), np.uint8)
    b = np.zeros_like(a)
    a[1, 2, 3] = 4
    b[7, 9, 10] = 4
    hd, hd95, na, nb = sd.hausdorff(a, b, 4)
    assert (na, nb) == (1, 1)
    assert hd == hd95 == math.sqrt(36 + 49 + 49)


def test_nearest_rank_percentile_on_a_known_multiset():
    # 20 isolated voxels at x = 2, 4, ..., 40 and one voxel at the origin: the
    # directed squared distances of A are (2i)^2; the 19th smallest is 38^2
    a = np.zeros((1, 1, 41), np.uint8)
    a[0, 0, 2:41:2] = 1
    b = np.zeros_like(a)
    b[0, 0, 0] = 1
    hd, hd95, na, nb = sd.hausdorff(a, b, 1)
    assert (na, nb) == (20, 1)
    assert hd == 40.0 and hd95 == 38.0
    assert sd.nearest_rank(np.arange(1, 101), 95) == 95
    assert sd.nearest_rank(np.arange(1, 102), 95) == 96


def test_identity_symmetry_and_absent_label():
    la, lb = synth.label_pair((32, 32, 32), synth.phantom.C0_ELLIPSOIDS, 2.0)
    for l in (1, 2, 3):
        assert sd.hausdorff(la, la, l)[:2] == (0.0, 0.0)
        assert sd.hausdorff(la, lb, l)[:2] == sd.hausdorff(lb, la, l)[:2]
    hd, hd95, na, nb = sd.hausdorff(la, lb, 9)
    assert math.isnan(hd) and math.isnan(hd95) and na == nb == 0


def test_concentric_balls():
    n = 40
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    r2 = (x - 20) ** 2 + (y - 20) ** 2 + (z - 20) ** 2
    a = (r2 <= 36).astype(np.uint8)
    b = (r2 <= 100).astype(np.uint8)
    hd, _, _, _ = sd.hausdorff(a, b, 1)
    assert 3.0 <= hd <= 5.0


def test_warped_labels_of_the_identity_are_the_labels():
    # identical meshes on both sides: T is the identity, so the pulled-back
    # label is the other image's own label at every covered voxel
    p = synth.make_c0(n_sol=1)
    la, lb = synth.label_pair((32, 32, 32), synth.phantom.C0_ELLIPSOIDS, 2.0)
    orc = oracle.Oracle(p)
    ref = p.ref_points.astype(np.float32)
    w = orc.warp_labels(ref, ref, 0, lb)
    np.testing.assert_array_equal(w, lb)


def test_warped_labels_agree_with_the_overlap_counts():
    p = synth.make_c0(n_sol=2)
    la, lb = synth.label_pair((32, 32, 32), synth.phantom.C0_ELLIPSOIDS, 2.0)
    orc = oracle.Oracle(p)
    for side in (0, 1):
        own, oth = (la, lb) if side == 0 else (lb, la)
        w = orc.warp_labels(p.sol_src[1], p.sol_tgt[1], side, oth)
        _, counts = orc.dvf(p.sol_src[1], p.sol_tgt[1], side, own, oth, 4)
        cov = w != 255
        for l in range(4):
            assert counts[l, 1] == int(((w == l) & cov).sum())
            assert counts[l, 2] == int(((w == l) & (own == l) & cov).sum())
