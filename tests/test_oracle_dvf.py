"""Pins of the oracle's displacement field and label overlap (reading R15).

- The identity deformation gives a zero field over the whole image.
- A global affine deformation of a box-spanning mesh gives the closed-form
  field (A - I) p + b at every voxel, whatever the tetrahedralisation.
- With the identity, every voxel keeps its label (Dice 1); under an integer
  translation the pulled-back labels are the shifted label image, clamped
  at the border (numpy closed form).
- Voxels in no copy, or in a folded copy, are NaN; the covered count
  equals the voxel count of the objective."""

import numpy as np
import pytest

import oracle
from helpers import box_lattice, problem, random_image


def _box(nx=12, ny=10, nz=9, flip_x=False):
    pts, tets = box_lattice([-0.5, 4.0, 8.0, nx - 0.5], [-0.5, 5.0, ny - 0.5], [-0.5, 3.0, 6.0, nz - 0.5],
                            flip_x=flip_x)
    img = random_image((nz, ny, nx), 5)
    return pts, tets, img


def test_identity_field_is_zero_everywhere():
    pts, tets, img = _box()
    orc = oracle.Oracle(problem(img, img, pts, tets))
    dvf, _ = orc.dvf(pts, pts, 0)
    assert not np.isnan(dvf).any()
    np.testing.assert_allclose(dvf, 0.0, rtol=0, atol=1e-12)     # FP64 barycentric rounding only


@pytest.mark.parametrize("flip_x", [False, True])
@pytest.mark.parametrize("side", [0, 1])
def test_affine_deformation_gives_the_closed_form(flip_x, side):
    nx, ny, nz = 12, 10, 9
    pts, tets, img = _box(nx, ny, nz, flip_x)
    c = np.array([(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2])
    # a dyadic contraction with shear about the centre: every vertex stays inside the
    # image box, so no coordinate is clamped and the deformation is exactly affine
    A = np.array([[0.875, 0.0625, 0.0], [-0.03125, 0.9375, 0.0], [0.0, 0.015625, 0.75]])
    b = np.array([0.25, -0.0625, 0.0])
    tgt = ((pts - c) @ A.T + c + b).astype(np.float32)
    assert np.all(tgt >= -0.5) and np.all(tgt <= np.array([nx, ny, nz]) - 0.5)
    src = pts.astype(np.float32)
    orc = oracle.Oracle(problem(img, img, pts, tets, subvoxel_bits=8))
    dvf, _ = orc.dvf(src, tgt, side)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([x, y, z], -1).astype(np.float64)
    S = 256.0
    # snapped vertices are exact here (dyadic coordinates), so the map is exactly affine
    src_s = np.round((src.astype(np.float64) + 0.5) * S) / S - 0.5
    tgt_s = np.round((tgt.astype(np.float64) + 0.5) * S) / S - 0.5
    np.testing.assert_array_equal(src_s, src)
    np.testing.assert_array_equal(tgt_s, tgt)
    if side == 0:
        want = (P - c) @ A.T + c + b - P
    else:
        Ainv = np.linalg.inv(A)
        want = (P - c - b) @ Ainv.T + c - P
    covered = ~np.isnan(dvf[..., 0])
    assert covered.sum() > 0.4 * covered.size
    np.testing.assert_allclose(dvf[covered], want[covered], rtol=0, atol=1e-11)


def test_labels_identity_and_integer_translation():
    nx, ny, nz = 12, 10, 9
    pts, tets, img = _box(nx, ny, nz)
    rng = np.random.default_rng(2)
    lab_s = rng.integers(0, 4, size=(nz, ny, nx)).astype(np.uint8)
    lab_t = rng.integers(0, 4, size=(nz, ny, nx)).astype(np.uint8)
    orc = oracle.Oracle(problem(img, img, pts, tets))
    _, counts = orc.dvf(pts, pts, 0, lab_s, lab_s, 4)
    for l in range(4):
        nl = int((lab_s == l).sum())
        assert counts[l].tolist() == [nl, nl, nl]
    # a mesh over part of the box (x in [0.5, 8]) and its copy moved by 2 voxels in x:
    # nothing is clamped, T(p) = p + (2, 0, 0), and the pulled-back label is lab_t[.., x + 2]
    pts2, tets2 = box_lattice([0.5, 4.0, 8.0], [-0.5, 5.0, ny - 0.5], [-0.5, 3.0, 6.0, nz - 0.5])
    orc2 = oracle.Oracle(problem(img, img, pts2, tets2))
    tgt = (pts2 + np.array([2.0, 0.0, 0.0], np.float32)).astype(np.float32)
    dvf, counts = orc2.dvf(pts2, tgt, 0, lab_s, lab_t, 4)
    covered = ~np.isnan(dvf[..., 0])
    xs_cov = np.unique(np.nonzero(covered)[2])
    assert xs_cov.min() >= 1 and xs_cov.max() <= 8
    pulled = np.zeros_like(lab_t)
    pulled[:, :, :nx - 2] = lab_t[:, :, 2:]
    for l in range(4):
        a = (lab_s == l) & covered
        bb = (pulled == l) & covered
        assert counts[l].tolist() == [int(a.sum()), int(bb.sum()), int((a & bb).sum())]


def test_uncovered_and_folded_voxels_are_nan():
    img = random_image((10, 10, 10), 1)
    pts = np.array([[1.0, 1.0, 1.0], [8.0, 1.0, 1.0], [1.0, 8.0, 1.0], [1.0, 1.0, 8.0]], np.float32)
    tets = np.array([[0, 1, 2, 3]], np.int32)
    p = problem(img, img, pts, tets, sol_src=pts[None], sol_tgt=pts[None])
    orc = oracle.Oracle(p)
    dvf, _ = orc.dvf(pts, pts + 0.5, 0)
    covered = ~np.isnan(dvf[..., 0])
    rec = orc.eval(pts, pts + 0.5, with_tets=True)["tets"][0]
    assert covered.sum() == rec["n_vox"][0] > 0
    np.testing.assert_allclose(dvf[covered], 0.5, rtol=0, atol=1e-12)
    folded = pts.copy()
    folded[3, 2] = -0.4                                       # vertex through the opposite face
    dvf, _ = orc.dvf(folded, folded, 0)
    assert np.isnan(dvf).all()
