"""GPU parity of the initialisation noise (reading R18, Sec. 4.2.2): the
kept rounds and every coordinate equal the oracle bit for bit (both sides
evaluate the same explicitly rounded FP64 operations and decide folds on
exact orientations)."""

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


def fixed_bits(fixed_axes):
    f = fixed_axes.astype(np.uint8)
    return (f[:, 0] | (f[:, 1] << 1) | (f[:, 2] << 2)).astype(np.uint8)


def draw_kernels(rng, n, K, box, sigma=(4.0, 12.0), a=(0.02, 0.2)):
    c = rng.uniform(0, 1, size=(n, 2, K, 3)) * (np.asarray(box, np.float64) - 1)
    s = rng.uniform(*sigma, size=(n, 2, K, 1))
    w = rng.uniform(*a, size=(n, 2, K, 1))
    return np.concatenate([c, s, w], -1).astype(np.float32)


def compare(mo, p, start_s, start_t, ker, max_rounds, fixed):
    n = ker.shape[0]
    gp = mo.Problem(p, max_solutions=1)
    S = torch.as_tensor(start_s).cuda().contiguous()
    T = torch.as_tensor(start_t).cuda().contiguous()
    fx = None if fixed is None else torch.as_tensor(fixed).cuda()
    rounds = gp.init_noise(S, T, torch.as_tensor(ker).cuda(), max_rounds, fixed=fx).cpu().numpy()
    S, T = S.cpu().numpy(), T.cpu().numpy()
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits)
    for i in range(n):
        for m, (start, got) in enumerate(((start_s, S), (start_t, T))):
            want, r = orc.init_noise(start[i], ker[i, m], fixed, max_rounds)
            assert rounds[i, m] == r, (i, m, rounds[i, m], r)
            np.testing.assert_array_equal(got[i], want)
    return rounds, S, T


@pytest.mark.parametrize("seed", range(3))
def test_c0_population(mo, seed):
    p = synth.make_c0(n_sol=1)
    rng = np.random.default_rng(seed)
    n = 6
    ref = np.broadcast_to(p.ref_points.astype(np.float32), (n, p.n_points, 3)).copy()
    ker = draw_kernels(rng, n, 5, (32, 32, 32), sigma=(3.0, 9.0), a=(0.05, 0.3))
    rounds, S, T = compare(mo, p, ref, ref, ker, 25, fixed_bits(p.fixed_axes))
    assert rounds.min() >= 1


@pytest.mark.parametrize("seed", range(3))
def test_random_ragged_meshes(mo, seed):
    from test_gpu_parity import _random_case
    p = _random_case(seed)
    rng = np.random.default_rng(seed + 10)
    n = p.sol_src.shape[0]
    ker = draw_kernels(rng, n, 3, (p.nx, p.ny, p.nz), sigma=(1.0, 4.0), a=(0.05, 0.5))
    compare(mo, p, p.sol_src, p.sol_tgt, ker, 12, None)


def test_degenerate_inputs(mo):
    p = synth.make_c0(n_sol=2)
    n = 2
    fx = fixed_bits(p.fixed_axes)
    gp = mo.Problem(p, max_solutions=1)
    S = torch.as_tensor(p.sol_src).cuda()
    T = torch.as_tensor(p.sol_tgt).cuda()
    # no kernels: nothing moves, every round is kept
    r = gp.init_noise(S, T, torch.zeros((n, 2, 0, 5), dtype=torch.float32, device="cuda"), 4).cpu().numpy()
    assert (r == 4).all()
    np.testing.assert_array_equal(S.cpu().numpy(), p.sol_src)
    # no rounds
    ker = torch.as_tensor(draw_kernels(np.random.default_rng(0), n, 2, (32, 32, 32))).cuda()
    r = gp.init_noise(S, T, ker, 0).cpu().numpy()
    assert (r == 0).all()
    np.testing.assert_array_equal(T.cpu().numpy(), p.sol_tgt)
    # a collapsing kernel: the first round folds and is rejected
    col = np.tile(np.array([16.0, 16.0, 16.0, 1e6, 1.0], np.float32), (n, 2, 1, 1))
    compare(mo, p, p.sol_src, p.sol_tgt, col, 3, fx)


def test_full_size_population(mo):
    """The 128x128x96 mesh (567 points, 2304 tets), 32 solutions, 8 kernels per
    mesh, up to 50 rounds: the benchmark's configuration on a quarter of its
    population."""
    p = synth.make_c1(n_sol=1)
    rng = np.random.default_rng(7)
    n = 32
    ref = np.broadcast_to(p.ref_points.astype(np.float32), (n, p.n_points, 3)).copy()
    ker = draw_kernels(rng, n, 8, (128, 128, 96), sigma=(8.0, 24.0), a=(0.02, 0.15))
    rounds, S, T = compare(mo, p, ref, ref, ker, 50, fixed_bits(p.fixed_axes))
    assert rounds.mean() > 5
