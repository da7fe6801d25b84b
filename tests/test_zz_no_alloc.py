"""The allocation-free entry point against the handle-based evaluation.

morea_fold_magnitude_noalloc is for callers that cannot allocate device
memory -- code running inside another allocator or memory pool that must not
re-enter it, or environments that only hand out pre-sized buffers.  It keeps
its per-(solution, tet) intermediates in one fixed array inside the library.
The test calls it through the C ABI twice in a row on different inputs (the
second call reuses that array) and checks each result against
morea_eval_full of the same solutions: fold flags and severities exactly,
f_magnitude within the 1e-5 relative tolerance of the parity tests.  This file
is collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""

import ctypes

import numpy as np
import pytest
import torch

import synth
from helpers import box_lattice, problem, random_image

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(mo, p, subvoxel_bits, src, tgt, f_mag, folded, sev):
    tets = torch.as_tensor(np.ascontiguousarray(p.tets, np.int32)).cuda()
    ref = torch.as_tensor(np.ascontiguousarray(p.ref_points, np.float32)).cuda()
    cdelta = torch.as_tensor(np.asarray(p.tissue_factor, np.float64)[p.tet_label].astype(np.float32)).cuda()
    n, V = int(src.shape[0]), int(src.shape[1])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = mo.lib().morea_fold_magnitude_noalloc(
        n, V, int(tets.shape[0]), _ptr(tets), _ptr(ref), _ptr(cdelta), p.nx, p.ny, p.nz, subvoxel_bits,
        _ptr(src), _ptr(tgt), _ptr(f_mag), _ptr(folded), _ptr(sev), stream)
    torch.cuda.synchronize()
    return rc


def test_noalloc_matches_eval_full_on_two_calls_in_a_row():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea as mo

    # call 1: the 32^3 problem; call 2: larger jitter, so some meshes fold
    cases = [synth.make_c0(n_sol=8), synth.make_c0(n_sol=6, jitter=4.5)]
    assert cases[1].n_solutions == 6
    for call, p in enumerate(cases):
        n = p.n_solutions
        gp = mo.Problem(p, max_solutions=n)
        src = torch.as_tensor(p.sol_src).cuda()
        tgt = torch.as_tensor(p.sol_tgt).cuda()
        obj, folded_ref, sev_ref = gp.eval_full(src, tgt)
        f_mag = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        folded = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        sev = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        rc = _noalloc(mo, p, gp.subvoxel_bits, src, tgt, f_mag, folded, sev)
        assert rc == mo.OK, mo.status_string(rc)
        np.testing.assert_array_equal(folded.cpu().numpy(), folded_ref.cpu().numpy())
        np.testing.assert_array_equal(sev.cpu().numpy(), sev_ref.cpu().numpy())
        np.testing.assert_allclose(f_mag.cpu().numpy(), obj[:, 1].cpu().numpy(), rtol=1e-5, atol=0)
        if call == 1:
            assert folded_ref.cpu().numpy().any(), "the second call should contain folded meshes"
        gp.close()


def test_noalloc_rejects_batches_beyond_its_scratch():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea as mo
    p = synth.make_c0(n_sol=1)
    n = mo.NOALLOC_MAX_TET_EVALS // p.n_tets + 1
    src = torch.as_tensor(np.repeat(p.sol_src, n, axis=0)).cuda()
    out = (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda"),
           torch.empty(n, dtype=torch.float64, device="cuda"))
    rc = _noalloc(mo, p, 8, src, src, *out)
    assert rc == mo.EINVAL


def test_noalloc_chooses_the_grid_of_problem_creation():
    """subvoxel_bits = 0 picks the same grid as problem creation: on a
    512-voxel-long box both lower k from 8 to 7."""
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea as mo
    nx, ny, nz = 512, 6, 5
    pts, tets = box_lattice(np.linspace(-0.5, nx - 0.5, 9), [-0.5, 2.0, ny - 0.5], [-0.5, nz - 0.5])
    rng = np.random.default_rng(11)
    sols = np.repeat(pts[None], 4, axis=0).astype(np.float64)
    ix = (pts[:, 0] > -0.5) & (pts[:, 0] < nx - 0.5)          # off the x faces: move along x
    iy = pts[:, 1] == np.float32(2.0)                           # the inner y level: move along y
    sols[:, ix, 0] += rng.uniform(-3.0, 3.0, size=(4, int(ix.sum())))
    sols[:, iy, 1] += rng.uniform(-0.4, 0.4, size=(4, int(iy.sum())))
    img = random_image((nz, ny, nx), 3)
    p = problem(img, img, pts, tets, subvoxel_bits=0, sol_src=sols.astype(np.float32),
                sol_tgt=sols[::-1].copy().astype(np.float32))
    gp = mo.Problem(p, max_solutions=4)
    assert gp.subvoxel_bits == 7
    src, tgt = torch.as_tensor(p.sol_src).cuda(), torch.as_tensor(p.sol_tgt).cuda()
    obj, folded_ref, sev_ref = gp.eval_full(src, tgt)
    p.n_solutions = 4
    out = (torch.empty(4, dtype=torch.float64, device="cuda"), torch.empty(4, dtype=torch.uint8, device="cuda"),
           torch.empty(4, dtype=torch.float64, device="cuda"))
    assert _noalloc(mo, p, 0, src, tgt, *out) == mo.OK
    np.testing.assert_array_equal(out[1].cpu().numpy(), folded_ref.cpu().numpy())
    np.testing.assert_array_equal(out[2].cpu().numpy(), sev_ref.cpu().numpy())
    np.testing.assert_allclose(out[0].cpu().numpy(), obj[:, 1].cpu().numpy(), rtol=1e-5, atol=0)
    gp.close()


def test_noalloc_reports_a_zero_reference_volume():
    """A tet whose reference volume is zero (problem creation rejects it) is
    not evaluated: every solution reports f_magnitude NaN and folded."""
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea as mo
    p = synth.make_c0(n_sol=3)
    ref = p.ref_points.copy()
    t0 = p.tets[5]
    ref[t0[3]] = ref[t0[0]]                 # collapse the tet onto a triangle
    p.ref_points = ref
    src, tgt = torch.as_tensor(p.sol_src).cuda(), torch.as_tensor(p.sol_tgt).cuda()
    out = (torch.zeros(3, dtype=torch.float64, device="cuda"), torch.zeros(3, dtype=torch.uint8, device="cuda"),
           torch.zeros(3, dtype=torch.float64, device="cuda"))
    assert _noalloc(mo, p, 8, src, tgt, *out) == mo.OK
    assert np.isnan(out[0].cpu().numpy()).all()
    assert (out[1].cpu().numpy() == 1).all()
