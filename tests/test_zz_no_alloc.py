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
