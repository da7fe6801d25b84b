"""Pins of the oracle's repair method (reading R14, Sec. 4.3.1).

Hand-built single-tet cases fix each rule: the trial scale is the distance
from the point to the plane of its opposite face (a closed form); a trial
that carries the point back through that plane removes the fold and is the
one kept (the lowest index among equal best trials); when every trial makes
the fold worse the repair stops with the solution unchanged; and on random
folded meshes the severity never grows and unfolded solutions are left
alone."""

import numpy as np
import pytest

import oracle
import synth
from test_oracle_sampling import _one_tet

BASE = np.array([6.0, 6.0, 6.0], np.float32)
CORNER = np.array([[0, 0, 0], [8, 0, 0], [0, 8, 0], [0, 0, 8]], np.float32) + BASE


def _orc(verts):
    img = np.zeros((24, 24, 24))
    return oracle.Oracle(_one_tet(img, img, CORNER, verts))


def test_sigma_is_the_distance_to_the_opposite_plane():
    orc = _orc(CORNER)
    # vertex 0 sits at the corner; its opposite face lies in x + y + z = 8 (relative)
    assert orc.repair_sigma(CORNER, 0, 1.0) == pytest.approx(8.0 / np.sqrt(3.0), rel=1e-14)
    assert orc.repair_sigma(CORNER, 0, 0.25) == pytest.approx(2.0 / np.sqrt(3.0), rel=1e-14)
    # vertex 3: the opposite face is z = 0, 8 voxels away
    assert orc.repair_sigma(CORNER, 3, 1.0) == pytest.approx(8.0, rel=1e-14)


def test_a_trial_through_the_plane_removes_the_fold():
    folded = CORNER.copy()
    folded[0] = BASE + np.array([4.0, 4.0, 4.0], np.float32)     # past x + y + z = 8: inverted
    orc = _orc(folded)
    before = orc.eval(folded, CORNER)
    assert before["folded"] == 1 and before["severity"] > 0
    sigma = orc.repair_sigma(folded, 0, 1.0)
    want = np.array([-3.0, -3.0, -3.0])                          # back to BASE + (1, 1, 1): unfolded
    noise = np.zeros((2, 64, 3), np.float32)
    noise[0, 9] = want / sigma
    noise[0, 5] = want / sigma                                   # an equally good earlier trial
    noise[0, 7] = np.array([0.5, 0.0, 0.0]) / sigma              # keeps the fold (worse or equal)
    s, t, moved, sev = orc.repair(folded, CORNER, noise, max_points=2)
    assert moved == 1 and sev == 0.0
    step = np.float64(sigma) * noise[0, 5].astype(np.float64)
    np.testing.assert_array_equal(s[0], (folded[0].astype(np.float64) + step).astype(np.float32))
    np.testing.assert_array_equal(s[1:], folded[1:])
    np.testing.assert_array_equal(t, CORNER)
    assert orc.eval(s, t)["folded"] == 0


def test_repair_stops_when_every_trial_deteriorates():
    folded = CORNER.copy()
    folded[0] = BASE + np.array([4.0, 4.0, 4.0], np.float32)
    orc = _orc(folded)
    sev0 = orc.eval(folded, CORNER)["severity"]
    sigma = orc.repair_sigma(folded, 0, 1.0)
    noise = np.tile(np.array([1.0, 1.0, 1.0], np.float32) / np.float32(sigma), (3, 64, 1))  # deeper
    s, t, moved, sev = orc.repair(folded, CORNER, noise, max_points=3)
    assert moved == 0
    np.testing.assert_array_equal(s, folded)
    assert sev == sev0


@pytest.mark.parametrize("seed", range(5))
def test_random_meshes_never_get_worse(seed):
    from test_gpu_parity import _random_case
    p = _random_case(60 + seed, fold=True)
    orc = oracle.Oracle(p)
    rng = np.random.default_rng(seed)
    for i in range(p.sol_src.shape[0]):
        s0, t0 = p.sol_src[i], p.sol_tgt[i]
        before = orc.eval(s0, t0)
        noise = rng.normal(size=(16, 64, 3)).astype(np.float32)
        s, t, moved, sev = orc.repair(s0, t0, noise, max_points=16)
        assert sev <= before["severity"] + 1e-15
        assert 0 <= moved <= 16
        after = orc.eval(s, t)
        assert after["severity"] == pytest.approx(sev, rel=1e-15, abs=1e-15)
        if not before["folded"]:
            assert moved == 0
            np.testing.assert_array_equal(s, s0)


def test_fixed_axes_stay_in_every_trial():
    # the same inversion as above; with x and z of vertex 0 fixed, the kept
    # trial moves only y: the best trial is the one whose y step undoes the
    # fold, whatever its x and z draws are
    folded = CORNER.copy()
    folded[0] = BASE + np.array([1.0, 10.0, 1.0], np.float32)    # x + y + z = 12 > 8: inverted
    orc = _orc(folded)
    sigma = orc.repair_sigma(folded, 0, 1.0)
    noise = np.zeros((2, 64, 3), np.float32)
    noise[0, 3] = np.array([-40.0, -9.0, -40.0]) / sigma         # y back to 1; x, z would leave the box
    fixed = np.zeros(4, np.uint8)
    fixed[0] = 1 | 4                                             # x and z of vertex 0
    s, t, moved, sev = orc.repair(folded, CORNER, noise, max_points=2, fixed=fixed)
    assert moved == 1 and sev == 0.0
    y = (np.float64(folded[0, 1]) + np.float64(sigma) * np.float64(noise[0, 3, 1])).astype(np.float32)
    np.testing.assert_array_equal(s[0], [folded[0, 0], y, folded[0, 2]])
    # without the fixed axes the same draw moves x and z as well
    s2, _, _, _ = orc.repair(folded, CORNER, noise, max_points=2)
    assert s2[0, 0] != folded[0, 0] and s2[0, 2] != folded[0, 2]


@pytest.mark.parametrize("seed", range(3))
def test_fixed_boundary_axes_on_random_meshes(seed):
    from test_gpu_parity import _random_case
    p = _random_case(70 + seed, fold=True)
    orc = oracle.Oracle(p)
    f = p.fixed_axes.astype(np.uint8)
    fixed = (f[:, 0] | (f[:, 1] << 1) | (f[:, 2] << 2)).astype(np.uint8)
    rng = np.random.default_rng(seed)
    for i in range(p.sol_src.shape[0]):
        s0, t0 = p.sol_src[i], p.sol_tgt[i]
        noise = rng.normal(size=(16, 64, 3)).astype(np.float32)
        s, t, moved, sev = orc.repair(s0, t0, noise, max_points=16, fixed=fixed)
        np.testing.assert_array_equal(s[p.fixed_axes], s0[p.fixed_axes])
        np.testing.assert_array_equal(t[p.fixed_axes], t0[p.fixed_axes])
        assert sev <= orc.eval(s0, t0)["severity"] + 1e-15
