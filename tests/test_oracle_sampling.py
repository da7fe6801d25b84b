"""Pins of the oracle's sampled estimator (reading R13, App. A.2).

Each building block is checked against something other than itself:
- the Sobol generator against SciPy's unscrambled Sobol sequence, which uses
  the same published direction numbers;
- the coordinate hash and the shift mixer against their published test
  vectors;
- the barycentric samples against the moments of the uniform distribution on
  a simplex, which are closed forms;
- the whole estimator against closed forms: the sample count of a tet of
  known volume, a linear image under a translation (every sample gives the
  same h), and the mean of x^2 over a tet.
"""

import dataclasses

import numpy as np
import pytest

import oracle
import synth

S8 = 256          # 2^k for subvoxel_bits = 8


def test_sobol_matches_scipy_unscrambled():
    qmc = pytest.importorskip("scipy.stats.qmc")
    n = 1 << 13
    ref = (qmc.Sobol(d=4, scramble=False, bits=32).random(n) * 2.0 ** 32).astype(np.uint64)
    mine = np.array([[oracle.sobol(j, d) for d in range(4)] for j in range(n)], np.uint64)
    np.testing.assert_array_equal(mine, ref)


def test_hash_and_mixer_published_vectors():
    # FNV-1a 64-bit test vectors
    assert oracle.fnv1a64(b"") == 0xCBF29CE484222325
    assert oracle.fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert oracle.fnv1a64(b"foobar") == 0x85944171F73967E8
    # splitmix64 outputs for the states 0 and 1234567
    assert oracle.splitmix64_outputs(0, 1) == [0xE220A8397B1DCDAF]
    assert oracle.splitmix64_outputs(1234567, 5) == [6457827717110365317, 3203168211198807973,
                                                     9817491932198370423, 4593380528125082431,
                                                     16408922859458223821]


def test_shifts_follow_the_coordinates():
    tet = np.array([[0, 0, 0], [8, 0, 0], [0, 8, 0], [0, 0, 8]], np.int64) * S8 + 128
    a = oracle.copy_shifts(tet)
    np.testing.assert_array_equal(a, oracle.copy_shifts(tet.copy()))
    moved = tet + np.array([1, 0, 0])
    assert not np.array_equal(a, oracle.copy_shifts(moved))
    # the shifts are the splitmix64 outputs from the FNV-1a hash of the
    # coordinates as little-endian int32 words
    h = oracle.fnv1a64(tet.astype("<i4").tobytes())
    want = [x >> 32 for x in oracle.splitmix64_outputs(h, 4)]
    np.testing.assert_array_equal(a, np.array(want, np.uint32))


def test_barycentric_samples_have_the_uniform_simplex_moments():
    shift = np.array([0x12345678, 0x9ABCDEF0, 0x0F1E2D3C, 0x4B5A6978], np.uint32)
    n = 1 << 14
    lam = np.array([oracle.sample_lambda(shift, j) for j in range(n)])
    assert np.all(lam >= 0.0)
    np.testing.assert_allclose(lam.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    # uniform on the simplex = Dirichlet(1, 1, 1, 1):
    # E[l_i] = 1/4, E[l_i^2] = 1/10, E[l_i l_j] = 1/20
    np.testing.assert_allclose(lam.mean(axis=0), 0.25, atol=2e-4)
    second = lam.T @ lam / n
    want = np.full((4, 4), 1 / 20) + np.eye(4) * (1 / 10 - 1 / 20)
    np.testing.assert_allclose(second, want, atol=2e-4)


def _one_tet(img_s, img_t, verts_s, verts_t, rate=1.0):
    nz, ny, nx = img_s.shape
    tets = np.array([[0, 1, 2, 3]], np.int32)
    return synth.Problem(
        name="one-tet", nx=nx, ny=ny, nz=nz, dtype="f32",
        image_s=img_s.astype(np.float32), image_t=img_t.astype(np.float32),
        ref_points=np.asarray(verts_s, np.float32), tets=tets,
        tet_label=np.zeros(1, np.int32), tissue_factor=np.ones(1), guid_s=np.zeros((0, 3), np.float32),
        guid_t=np.zeros((0, 3), np.float32), guid_group=np.zeros(0, np.int32), trunc_radius=2.0,
        sol_src=np.asarray(verts_s, np.float32)[None], sol_tgt=np.asarray(verts_t, np.float32)[None],
        fixed_axes=np.zeros((4, 3), bool), g_mode=synth.phantom.G_OFF, estimator=1, sampling_rate=rate)


def _grid(n=24):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


@pytest.mark.parametrize("rate", [1.0, 0.5, 2.75])
def test_sample_count_is_the_rounded_volume(rate):
    x, _, _ = _grid()
    v = np.array([[4, 4, 4], [12, 4, 4], [4, 12, 4], [4, 4, 12]], np.float32)   # volume 512 / 6
    p = _one_tet(x, x, v, v, rate)
    rec = oracle.Oracle(p).eval(p.sol_src[0], p.sol_tgt[0], with_tets=True)["tets"][0]
    want = int(np.floor(np.float64(np.float32(rate)) * (512.0 / 6.0) + 0.5))
    assert rec["n_vox"][0] == want and rec["n_vox"][1] == want


def test_linear_image_under_translation_gives_the_closed_form():
    x, y, z = _grid()
    a = np.array([1.5, -2.0, 0.75])
    img = a[0] * x + a[1] * y + a[2] * z + 3.0
    vs = np.array([[5, 5, 5], [13, 6, 5], [6, 14, 7], [7, 6, 15]], np.float32)
    t = np.array([1.25, -0.5, 0.75], np.float32)              # dyadic: exact on the snap grid
    p = _one_tet(img, img, vs, vs + t)
    r = oracle.Oracle(p).eval(p.sol_src[0], p.sol_tgt[0])
    # every sample: a - b = a . (p - T(p)) = -a . t on side 0 and +a . t on side 1
    assert r["obj"][0] == pytest.approx(float(a @ t) ** 2, rel=1e-12)
    assert r["obj"][1] == pytest.approx(0.0, abs=1e-12)


def test_mean_of_x_squared_over_a_tet():
    x, _, _ = _grid(32)
    vs = np.array([[3, 4, 5], [27, 6, 4], [5, 26, 8], [9, 7, 28]], np.float32)
    p = _one_tet(x, np.zeros_like(x), vs, vs, rate=1.0)
    rec = oracle.Oracle(p).eval(p.sol_src[0], p.sol_tgt[0], with_tets=True)["tets"][0]
    # side 0: h = (x - 0)^2 at uniform points of the tet; E[x^2] for the uniform
    # distribution on a simplex is (sum_i x_i^2 + (sum_i x_i)^2) / 20
    xs = vs[:, 0].astype(np.float64)
    want = (np.sum(xs ** 2) + np.sum(xs) ** 2) / 20.0
    got = rec["e_img"][0] / rec["n_vox"][0]
    assert rec["n_vox"][0] > 1000
    assert got == pytest.approx(want, rel=2e-3)
    # side 1 samples the target copy (same coordinates, its own seed = same
    # shifts) and compares I_t = 0 there with I_s at the same point
    assert rec["e_img"][1] == pytest.approx(rec["e_img"][0], rel=1e-12)


def test_voxel_mode_is_unchanged_by_the_new_fields():
    p = synth.make_c0(n_sol=2)
    a = oracle.Oracle(p).eval(p.sol_src[0], p.sol_tgt[0])
    b = oracle.Oracle(dataclasses.replace(p, sampling_rate=3.0)).eval(p.sol_src[0], p.sol_tgt[0])
    np.testing.assert_array_equal(a["obj"], b["obj"])
    assert a["n_vox"] == b["n_vox"]


def test_sampled_partial_equals_fresh_full():
    p = dataclasses.replace(synth.make_c0(n_sol=2), estimator=1, sampling_rate=0.5)
    orc = oracle.Oracle(p)
    s0, t0 = p.sol_src[0], p.sol_tgt[0]
    full0 = orc.eval(s0, t0)
    s1, t1 = s0.copy(), t0.copy()
    chg = np.array([31, 32, 56], np.int32)
    rng = np.random.default_rng(3)
    s1[chg] += rng.normal(0, 0.7, (3, 3)).astype(np.float32)
    t1[chg] += rng.normal(0, 0.7, (3, 3)).astype(np.float32)
    part = orc.eval_partial(s0, t0, s1, t1, chg, full0)
    fresh = orc.eval(s1, t1)
    assert part["n_vox"] == fresh["n_vox"]
    np.testing.assert_allclose(part["obj"], fresh["obj"], rtol=1e-12)
