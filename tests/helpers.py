"""Small hand-built problems shared by the oracle pins and the GPU parity tests."""

from types import SimpleNamespace

import numpy as np

import synth


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
