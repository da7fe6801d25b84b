"""GPU parity of the tissue-overlap elasticity factor (App. A.1) against the
oracle: with a tissue mask the library sets each tet's c_delta from the
voxel centres of its reference copy; the per-tet magnitude terms (c_delta
times the edge sum) and f_magnitude must match the oracle's within the
FP32 tolerance of the magnitude term, and the other objectives are
unaffected."""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def _masked(p, shape, ellipsoids, amp, seed):
    la, _ = synth.label_pair(shape, ellipsoids, amp)
    L = int(la.max()) + 1
    p.tissue_mask = la
    p.tissue_factor = np.random.default_rng(seed).uniform(0.5, 4.0, L)
    return p


@pytest.mark.parametrize("case", ["c0", "c1"])
def test_mask_factors_match_oracle(mo, case):
    if case == "c0":
        p = _masked(synth.make_c0(n_sol=3), (32, 32, 32), synth.phantom.C0_ELLIPSOIDS, 2.0, 1)
    else:
        p = _masked(synth.make_c1(n_sol=2), (128, 128, 96), synth.phantom.C1_ELLIPSOIDS, 6.0, 2)
    n = p.sol_src.shape[0]
    gp = mo.Problem(p, max_solutions=n)
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits, trunc_radius=gp.trunc_radius)
    c = orc.cdelta()
    assert len(np.unique(np.round(c, 9))) > 2
    obj, _, _ = gp.eval_full(torch.as_tensor(p.sol_src).cuda(), torch.as_tensor(p.sol_tgt).cuda())
    obj = obj.cpu().numpy()
    recs = gp.read_records(n)
    for i in range(n):
        r = orc.eval(p.sol_src[i], p.sol_tgt[i], with_tets=True)
        np.testing.assert_allclose(recs[i]["e_mag"], r["tets"]["e_mag"], rtol=1e-4, atol=1e-9)
        np.testing.assert_allclose(obj[i], r["obj"], rtol=1e-5, atol=1e-10)
    # without the mask the same problem takes the per-label factors
    p2 = synth.make_c0(n_sol=1) if case == "c0" else synth.make_c1(n_sol=1)
    gp2 = mo.Problem(p2, max_solutions=1)
    o2 = gp2.eval_full(torch.as_tensor(p2.sol_src).cuda(), torch.as_tensor(p2.sol_tgt).cuda())[0].cpu().numpy()
    r2 = oracle.Oracle(p2, subvoxel_bits=gp2.subvoxel_bits, trunc_radius=gp2.trunc_radius).eval(
        p2.sol_src[0], p2.sol_tgt[0])
    np.testing.assert_allclose(o2[0], r2["obj"], rtol=1e-5, atol=1e-10)
