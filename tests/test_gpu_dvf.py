"""GPU parity of the displacement field and label overlap (reading R15)
against the oracle: the covered voxels (the NaN pattern) are exact;
displacements are the FP32 affine map against the FP64 barycentric map,
within 1e-4 voxel; the label counts agree with the oracle's exact pull-back
except at voxels whose nearest voxel the FP32 error bound leaves open
(helpers.check_warped_labels)."""

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import box_lattice, check_warped_labels, problem, random_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def compare(mo, p, src, tgt, side, n_labels=5, seed=0):
    rng = np.random.default_rng(seed)
    lab_own = rng.integers(0, n_labels + 1, size=(p.nz, p.ny, p.nx)).astype(np.uint8)   # includes an uncounted label
    lab_oth = rng.integers(0, n_labels + 1, size=(p.nz, p.ny, p.nx)).astype(np.uint8)
    gp = mo.Problem(p, max_solutions=1)
    dvf, counts = gp.displacement(torch.as_tensor(src).cuda(), torch.as_tensor(tgt).cuda(), side,
                                  torch.as_tensor(lab_own).cuda(), torch.as_tensor(lab_oth).cuda(), n_labels)
    torch.cuda.synchronize()
    dvf, counts = dvf.cpu().numpy(), counts.cpu().numpy()
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits)
    want, wc = orc.dvf(src, tgt, side, lab_own, lab_oth, n_labels)
    np.testing.assert_array_equal(np.isnan(dvf), np.isnan(want))
    cov = ~np.isnan(want)
    np.testing.assert_allclose(dvf[cov], want[cov], rtol=0, atol=1e-4)
    w = gp.warp_labels(torch.as_tensor(src).cuda(), torch.as_tensor(tgt).cuda(), side,
                       torch.as_tensor(lab_oth).cuda()).cpu().numpy()
    _, amb = check_warped_labels(w, orc, src, tgt, side, lab_oth, n_labels, counts, lab_own)
    if not amb.any():                 # then the oracle's own counts hold exactly
        np.testing.assert_array_equal(counts, wc)
    return dvf, counts


@pytest.mark.parametrize("side", [0, 1])
def test_c0_solutions(mo, side):
    p = synth.make_c0(n_sol=3)
    for i in range(3):
        compare(mo, p, p.sol_src[i], p.sol_tgt[i], side, seed=i)


@pytest.mark.parametrize("seed", range(4))
def test_random_small_meshes(mo, seed):
    from test_gpu_parity import _random_case
    p = _random_case(seed)
    compare(mo, p, p.sol_src[0], p.sol_tgt[0], seed % 2, seed=seed)


def test_partial_mesh_leaves_nan(mo):
    img = random_image((10, 10, 10), 1)
    pts = np.array([[1.0, 1.0, 1.0], [8.0, 1.0, 1.0], [1.0, 8.0, 1.0], [1.0, 1.0, 8.0]], np.float32)
    p = problem(img, img, pts, np.array([[0, 1, 2, 3]], np.int32), sol_src=pts[None], sol_tgt=pts[None])
    dvf, _ = compare(mo, p, pts, (pts + 0.75).astype(np.float32), 0)
    assert np.isnan(dvf).any() and (~np.isnan(dvf)).any()


def test_full_size_field(mo):
    p = synth.make_c1()
    compare(mo, p, p.sol_src[0], p.sol_tgt[0], 0, n_labels=6)
