"""GPU parity of the warped label image and of the surface distances
(reading R17, Hausdorff distance and its 95th percentile, Sec. 5) against
the oracle.  Warped labels equal the oracle's exact pull-back element by
element, except at voxels whose nearest voxel the FP32 error bound leaves
open, which must hold one of the labels it allows
(helpers.check_warped_labels).  HD / HD95 of the same label images are
square roots of integers, so they equal bit for bit."""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import check_warped_labels
from oracle import surface as sd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def gpu_hd(mo, a, b, label, work=None):
    out = mo.surface_distance(torch.as_tensor(a).cuda(), torch.as_tensor(b).cuda(), label, work=work)
    return out.cpu().numpy()


def check(mo, a, b, label, work=None):
    got = gpu_hd(mo, a, b, label, work)
    hd, hd95, na, nb = sd.hausdorff(a, b, label)
    assert (int(got[2]), int(got[3])) == (na, nb)
    if math.isnan(hd):
        assert np.isnan(got[0]) and np.isnan(got[1])
    else:
        assert got[0] == hd and got[1] == hd95, (got, hd, hd95)
    return got


@pytest.mark.parametrize("shape", [(24, 22, 20), (33, 45, 70), (5, 3, 37), (1, 1, 41), (40, 1, 1)])
@pytest.mark.parametrize("seed", [0, 1])
def test_random_masks(mo, shape, seed):
    rng = np.random.default_rng(seed)
    a = (rng.random(shape) < 0.35).astype(np.uint8) * 3
    b = (rng.random(shape) < 0.55).astype(np.uint8) * 3
    check(mo, a, b, 3)
    check(mo, b, a, 3)


@pytest.mark.parametrize("shape", [(2, 3, 1024), (2, 1024, 3), (1024, 2, 3)])
def test_maximum_line_lengths(mo, shape):
    """Lines of 1024 voxels along each axis: 32 chunks in the x pass, and
    128 KiB of staged column in the y and z passes."""
    rng = np.random.default_rng(sum(shape))
    a = (rng.random(shape) < 0.02).astype(np.uint8)
    b = (rng.random(shape) < 0.01).astype(np.uint8)
    check(mo, a, b, 1)
    check(mo, a, b, 0)


def test_hand_cases(mo):
    a = np.zeros((1, 1, 41), np.uint8)
    a[0, 0, 2:41:2] = 1
    b = np.zeros_like(a)
    b[0, 0, 0] = 1
    got = check(mo, a, b, 1)
    assert got[0] == 40.0 and got[1] == 38.0
    box = np.zeros((32, 32, 32), np.uint8)
    box[10:21, 10:21, 10:21] = 1
    big = np.zeros_like(box)
    big[8:23, 8:23, 8:23] = 1
    assert check(mo, box, big, 1)[0] == math.sqrt(12.0)


def test_identity_absent_label_and_full_image(mo):
    la, lb = synth.label_pair((32, 32, 32), synth.phantom.C0_ELLIPSOIDS, 2.0)
    assert list(check(mo, la, la, 1)[:2]) == [0.0, 0.0]
    check(mo, la, lb, 9)                       # absent: NaN
    full = np.ones((7, 9, 11), np.uint8)
    check(mo, full, full, 1)
    check(mo, full, np.zeros_like(full), 0)    # label 0 absent from the first


def test_phantom_organs_and_workspace_reuse(mo):
    la, lb = synth.label_pair((128, 128, 96), synth.phantom.C1_ELLIPSOIDS, 6.0)
    work = torch.empty(mo.surface_distance_workspace(128, 128, 96), dtype=torch.uint8, device="cuda")
    for label in range(1, 6):                  # the organs (the background's shell is the whole border)
        check(mo, la, lb, label, work=work)


@pytest.mark.parametrize("side", [0, 1])
def test_warped_labels_c0(mo, side):
    p = synth.make_c0(n_sol=3)
    la, lb = synth.label_pair((32, 32, 32), synth.phantom.C0_ELLIPSOIDS, 2.0)
    own, oth = (la, lb) if side == 0 else (lb, la)
    gp = mo.Problem(p, max_solutions=1)
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits)
    for i in range(3):
        w = gp.warp_labels(torch.as_tensor(p.sol_src[i]).cuda(), torch.as_tensor(p.sol_tgt[i]).cuda(), side,
                           torch.as_tensor(oth).cuda()).cpu().numpy()
        check_warped_labels(w, orc, p.sol_src[i], p.sol_tgt[i], side, oth)
        for label in (1, 2, 3):
            check(mo, own, w, label)


def test_partial_mesh_marks_uncovered(mo):
    from helpers import problem, random_image
    img = random_image((10, 10, 10), 1)
    pts = np.array([[1.0, 1.0, 1.0], [8.0, 1.0, 1.0], [1.0, 8.0, 1.0], [1.0, 1.0, 8.0]], np.float32)
    p = problem(img, img, pts, np.array([[0, 1, 2, 3]], np.int32), sol_src=pts[None], sol_tgt=pts[None])
    lab = np.random.default_rng(2).integers(0, 4, size=(10, 10, 10)).astype(np.uint8)
    gp = mo.Problem(p, max_solutions=1)
    tgt = (pts + 0.75).astype(np.float32)
    w = gp.warp_labels(torch.as_tensor(pts).cuda(), torch.as_tensor(tgt).cuda(), 0,
                       torch.as_tensor(lab).cuda()).cpu().numpy()
    check_warped_labels(w, oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits), pts, tgt, 0, lab)
    assert (w == mo.NO_LABEL).any() and (w != mo.NO_LABEL).any()


def test_full_size_registration_scores(mo):
    """128x128x96 problem: the warped organ labels of one solution and the
    HD / HD95 of every organ, GPU against oracle."""
    p = synth.make_c1(n_sol=2)
    la, lb = synth.label_pair((128, 128, 96), synth.phantom.C1_ELLIPSOIDS, 6.0)
    gp = mo.Problem(p, max_solutions=1)
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits)
    w = gp.warp_labels(torch.as_tensor(p.sol_src[1]).cuda(), torch.as_tensor(p.sol_tgt[1]).cuda(), 0,
                       torch.as_tensor(lb).cuda())
    w = w.cpu().numpy()
    check_warped_labels(w, orc, p.sol_src[1], p.sol_tgt[1], 0, lb)
    for label in range(1, 6):
        check(mo, la, w, label)
