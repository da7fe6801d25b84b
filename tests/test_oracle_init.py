"""Pins of the initialisation-noise oracle (reading R18, Sec. 4.2.2 and
App. A.5: Gaussian kernels attract the mesh points in rounds while the
mesh stays unfolded).

The own exp is checked against the library exp, a single round against
the printed attraction written with numpy's exp, and the round logic by
its invariants: zero strength keeps the mesh, a collapsing round is
rejected, results are never folded, fixed axes stay, and the process is
memoryless (r rounds then R - r rounds equal R rounds)."""

import math

import numpy as np
import pytest

import oracle
import synth


def test_gexp_against_the_library_exp():
    # the reduction r = t - n ln2 uses ln2 rounded to double (error <= 2^-54),
    # so |n| <= 93 costs up to ~1e-14 relative; near 0 (n <= 1) a few ulp
    for t in np.linspace(-64.0, 0.0, 4001):
        want = math.exp(t)
        got = oracle.gexp(float(t))
        assert abs(got - want) <= 1e-13 * want, (t, got, want)
        if t >= -1.0:
            assert abs(got - want) <= 4 * math.ulp(want), (t, got, want)
    assert oracle.gexp(0.0) == 1.0
    assert oracle.gexp(-64.5) == 0.0
    assert oracle.gexp(-1e300) == 0.0


@pytest.fixture(scope="module")
def c0():
    p = synth.make_c0(n_sol=1)
    return p, oracle.Oracle(p)


def fixed_bits(p):
    f = p.fixed_axes.astype(np.uint8)
    return (f[:, 0] | (f[:, 1] << 1) | (f[:, 2] << 2)).astype(np.uint8)


def test_one_round_is_the_printed_attraction(c0):
    p, orc = c0
    X = p.ref_points.astype(np.float32)
    ker = np.array([[12.0, 15.0, 17.0, 6.0, 0.3], [25.0, 8.0, 20.0, 4.0, 0.2]], np.float32)
    fx = fixed_bits(p)
    Y, r = orc.init_noise(X, ker, fx, max_rounds=1)
    assert r == 1
    x = X.astype(np.float64)
    d = np.zeros_like(x)
    for cx, cy, cz, sig, a in ker.astype(np.float64):
        c = np.array([cx, cy, cz])
        g = np.exp(-((c - x) ** 2).sum(1) / (2 * sig * sig))
        d += (a * g)[:, None] * (c - x)
    want = (x + d).astype(np.float32)
    want[p.fixed_axes] = X[p.fixed_axes]
    ulp = np.spacing(np.abs(want).astype(np.float32) + np.float32(1))
    assert np.all(np.abs(Y - want) <= ulp)
    moved = np.abs(Y - X) > 0
    assert moved.any() and not moved[p.fixed_axes].any()


def test_zero_strength_keeps_the_mesh(c0):
    p, orc = c0
    X = p.sol_src[0]
    ker = np.array([[10.0, 10.0, 10.0, 5.0, 0.0]], np.float32)
    Y, r = orc.init_noise(X, ker, None, max_rounds=7)
    assert r == 7
    np.testing.assert_array_equal(Y, X)


def test_collapsing_round_is_rejected(c0):
    p, orc = c0
    X = p.ref_points.astype(np.float32)
    # g ~ 1 everywhere and a = 1: every point moves onto the centre, every tet
    # becomes degenerate (zero volume counts as folded)
    ker = np.array([[16.0, 16.0, 16.0, 1e6, 1.0]], np.float32)
    Y, r = orc.init_noise(X, ker, None, max_rounds=5)
    assert r == 0
    np.testing.assert_array_equal(Y, X)


def test_point_at_a_centre_does_not_move(c0):
    p, orc = c0
    X = p.ref_points.astype(np.float32)
    v = 31
    ker = np.array([list(X[v]) + [3.0, 0.5]], np.float32)
    Y, r = orc.init_noise(X, ker, None, max_rounds=1)
    assert r == 1
    np.testing.assert_array_equal(Y[v], X[v])


@pytest.mark.parametrize("seed", range(4))
def test_results_unfolded_fixed_axes_kept_and_memoryless(c0, seed):
    p, orc = c0
    rng = np.random.default_rng(seed)
    K = 6
    ker = np.concatenate([rng.uniform(0, 31, (K, 3)), rng.uniform(3, 10, (K, 1)), rng.uniform(0.05, 0.4, (K, 1))],
                         1).astype(np.float32)
    fx = fixed_bits(p)
    X0 = p.ref_points.astype(np.float32)
    Y, r = orc.init_noise(X0, ker, fx, max_rounds=30)
    assert 0 <= r <= 30
    assert orc.eval(Y, Y)["folded"] == 0
    np.testing.assert_array_equal(Y[p.fixed_axes], X0[p.fixed_axes])
    if r >= 2:
        Z, r1 = orc.init_noise(X0, ker, fx, max_rounds=r // 2)
        Z, r2 = orc.init_noise(Z, ker, fx, max_rounds=30 - r // 2)
        assert r1 == r // 2 and r1 + r2 == r
        np.testing.assert_array_equal(Z, Y)
    if r < 30:                                   # the next round folds
        _, more = orc.init_noise(Y, ker, fx, max_rounds=1)
        assert more == 0
