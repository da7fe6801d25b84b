"""Small hand-built problems shared by the oracle pins and the GPU parity tests."""

from types import SimpleNamespace

import numpy as np

import synth

# FP32 error model of the kernels' decisions (R9: the case of h; R15: the
# nearest voxel of T(p)), used to certify them against the FP64 oracle.
# A kernel evaluates T(p) = t0 + M (p - s0) with M = F adj(E) / D rounded
# once to FP32 (relative error 2^-24) and at most three rounded operations
# per coordinate (p - s0 is exact on the 2^-k grid); its error per axis is
# at most 4 * 2^-24 (|t0| + sum |M_ab| |p_b - s0_b|).  GAMMA_POS doubles
# that.  Its trilinear sample of exactly stored values takes three levels
# of (difference, fused lerp), at most 9 * 2^-24 times the largest stored
# value of the cell; GAMMA_VAL = 16 * 2^-24.  The oracle turns these into a
# per-voxel position radius and sample radius (``Oracle.set_perturbation``).
GAMMA_POS = 2.0 ** -21
GAMMA_VAL = 2.0 ** -20
# Largest fraction of covered voxels whose decision the model leaves open.
MAX_AMBIGUOUS = 0.02


def problem(img_s, img_t, ref, tets, *, label=None, tissue=None, guid_s=None, guid_t=None,
            guid_group=None, trunc_radius=4.0, h_mode=0, g_mode=0, subvoxel_bits=8,
            sol_src=None, sol_tgt=None, dtype=None):
    img_s = np.asarray(img_s)
    img_t = np.asarray(img_t)
    nz, ny, nx = img_s.shape
    ref = np.asarray(ref, np.float32)
    tets = np.asarray(tets, np.int32)
    if guid_s is None:
        guid_s = np.zeros((0, 3), np.float32)
        guid_t = np.zeros((0, 3), np.float32)
        guid_group = np.zeros((0,), np.int32)
    if guid_group is None:
        guid_group = np.zeros(len(guid_s), np.int32)
    if dtype is None:
        dtype = "f16" if img_s.dtype == np.float16 else "f32"
    return SimpleNamespace(
        name="handmade", nx=nx, ny=ny, nz=nz, dtype=dtype,
        image_s=img_s, image_t=img_t, ref_points=ref, tets=tets,
        tet_label=np.zeros(len(tets), np.int32) if label is None else np.asarray(label, np.int32),
        tissue_factor=np.ones(1) if tissue is None else np.asarray(tissue, np.float64),
        guid_s=np.asarray(guid_s, np.float32), guid_t=np.asarray(guid_t, np.float32),
        guid_group=np.asarray(guid_group, np.int32), trunc_radius=float(trunc_radius),
        h_mode=h_mode, g_mode=g_mode, subvoxel_bits=subvoxel_bits,
        sol_src=sol_src, sol_tgt=sol_tgt, n_points=len(ref), n_tets=len(tets),
        fixed_axes=np.zeros(ref.shape, bool))


def box_lattice(xs, ys, zs, flip_x=False):
    pts = synth.lattice_points(xs, ys, zs)
    tets = synth.kuhn_lattice(len(xs), len(ys), len(zs), flip_x=flip_x)
    return pts, tets


def random_image(shape_zyx, seed, scale=100.0, dtype=np.float32):
    rng = np.random.default_rng(seed)
    return (rng.normal(0.0, scale, size=shape_zyx)).astype(dtype)


def check_warped_labels(got, orc, src, tgt, side, lab_oth, n_labels=None, counts=None, lab_own=None):
    """Warped label image ``got`` (and optionally the per-label counts) of a
    GPU run against the oracle's exact pull-back (R15).  Voxels whose nearest
    voxel is the same over the whole FP32 error range must agree exactly; the
    others (ambiguous) must hold one of the labels that range allows, and
    stay below MAX_AMBIGUOUS of the covered voxels.  Counts: the own-label
    column exactly, the other two within the ambiguous voxels that allow
    the label."""
    orc.set_perturbation(GAMMA_POS, GAMMA_VAL)
    want, cand = orc.warp_labels(src, tgt, side, lab_oth, candidates=True)
    got = np.asarray(got)
    uniform = (cand == want[..., None]).all(-1)
    np.testing.assert_array_equal(got[uniform], want[uniform])
    amb = ~uniform
    covered = int((want != 255).sum())
    assert amb.sum() <= MAX_AMBIGUOUS * max(1, covered), "too many ambiguous voxels"
    if amb.any():
        assert (cand[amb] == got[amb][:, None]).any(-1).all(), "label outside the allowed range"
    if counts is not None:
        cov = want != 255
        lo = np.asarray(lab_own)
        want_counts = np.zeros((n_labels, 3), np.int64)
        for l in range(n_labels):
            want_counts[l, 0] = np.sum(cov & (lo == l))
            want_counts[l, 1] = np.sum(cov & (want == l))
            want_counts[l, 2] = np.sum(cov & (want == l) & (lo == l))
            allow = int(np.sum((cand[amb] == l).any(-1)))
            assert counts[l, 0] == want_counts[l, 0]
            assert abs(int(counts[l, 1]) - int(want_counts[l, 1])) <= allow
            assert abs(int(counts[l, 2]) - int(want_counts[l, 2])) <= allow
    return want, amb
