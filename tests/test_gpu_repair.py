"""GPU parity of the repair of folded solutions (Sec. 4.3.1, reading R14)
against the oracle: moved-point counts, the repaired coordinates and the
fold severity afterwards are bit-exact (the visit order, the trial scale
and the trial positions follow the same explicitly rounded FP64
arithmetic, and orientations are exact)."""

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import _random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def run_both(mo, p, src, tgt, max_points, scale, seed, fixed=None):
    n = src.shape[0]
    rng = np.random.default_rng(seed)
    noise = rng.normal(size=(n, max_points, 64, 3)).astype(np.float32)
    gp = mo.Problem(p, max_solutions=n)
    S = torch.as_tensor(np.ascontiguousarray(src, np.float32)).cuda()
    T = torch.as_tensor(np.ascontiguousarray(tgt, np.float32)).cuda()
    fx = None if fixed is None else torch.as_tensor(fixed).cuda()
    moved, sev = gp.repair_folds(S, T, torch.as_tensor(noise).cuda(), max_points, scale, fixed=fx)
    torch.cuda.synchronize()
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits)
    return S.cpu().numpy(), T.cpu().numpy(), moved.cpu().numpy(), sev.cpu().numpy(), orc, noise


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("scale", [1.0, 0.4])
def test_repair_matches_oracle_on_random_folded_meshes(mo, seed, scale):
    p = _random_case(60 + seed, fold=True)
    mp = 12
    S, T, moved, sev, orc, noise = run_both(mo, p, p.sol_src, p.sol_tgt, mp, scale, seed)
    for i in range(p.sol_src.shape[0]):
        s, t, m, sv = orc.repair(p.sol_src[i], p.sol_tgt[i], noise[i], mp, float(np.float32(scale)))
        assert moved[i] == m, i
        assert sev[i] == sv, i
        np.testing.assert_array_equal(S[i], s)
        np.testing.assert_array_equal(T[i], t)


@pytest.mark.parametrize("seed", range(3))
def test_repair_with_fixed_boundary_axes(mo, seed):
    p = _random_case(70 + seed, fold=True)
    f = p.fixed_axes.astype(np.uint8)
    fixed = (f[:, 0] | (f[:, 1] << 1) | (f[:, 2] << 2)).astype(np.uint8)
    mp = 12
    S, T, moved, sev, orc, noise = run_both(mo, p, p.sol_src, p.sol_tgt, mp, 1.0, seed, fixed=fixed)
    for i in range(p.sol_src.shape[0]):
        s, t, m, sv = orc.repair(p.sol_src[i], p.sol_tgt[i], noise[i], mp, 1.0, fixed=fixed)
        assert moved[i] == m and sev[i] == sv, i
        np.testing.assert_array_equal(S[i], s)
        np.testing.assert_array_equal(T[i], t)
        np.testing.assert_array_equal(S[i][p.fixed_axes], p.sol_src[i][p.fixed_axes])


def test_repair_on_the_full_size_mesh(mo):
    p = synth.make_c1()
    n = 8
    rng = np.random.default_rng(21)
    src = (p.sol_src[:n] + rng.normal(0, 6.0, p.sol_src[:n].shape)).astype(np.float32)   # many folds
    tgt = (p.sol_tgt[:n] + rng.normal(0, 6.0, p.sol_tgt[:n].shape)).astype(np.float32)
    S, T, moved, sev, orc, noise = run_both(mo, p, src, tgt, 40, 1.0, 3)
    assert moved.max() > 0
    for i in (0, 5):
        s, t, m, sv = orc.repair(src[i], tgt[i], noise[i], 40, 1.0)
        assert moved[i] == m and sev[i] == sv
        np.testing.assert_array_equal(S[i], s)
        np.testing.assert_array_equal(T[i], t)
    # the repair never increases the severity
    gp = mo.Problem(p, max_solutions=n)
    f0, s0 = gp.check_folds(torch.as_tensor(src).cuda(), torch.as_tensor(tgt).cuda())
    assert np.all(sev <= s0.cpu().numpy())


def test_unfolded_solutions_are_left_alone(mo):
    p = synth.make_c0(n_sol=4)
    S, T, moved, sev, orc, noise = run_both(mo, p, p.sol_src, p.sol_tgt, 8, 1.0, 0)
    assert np.all(moved == 0) and np.all(sev == 0.0)
    np.testing.assert_array_equal(S, p.sol_src)
    np.testing.assert_array_equal(T, p.sol_tgt)
