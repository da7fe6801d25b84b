"""Seeded synthetic registration problems shaped like MOREA's workloads.

The paper registers abdominal CT pairs (1.5 mm isotropic voxels, organs that
deform strongly, contour point sets as guidance, meshes of ~600 points; paper
Sec. 5.1-5.2).  Those scans are private, so these generators stand in for them
with analytic phantoms: ellipsoid "organs" on a background, a second image
that is the first warped by a smooth sinusoidal displacement, contour points
sampled on the ellipsoid surfaces (paired with their warped positions), a
lattice mesh split into tetrahedra, and a population of jittered meshes.

Conventions shared with the evaluator:
  * images are ``[nz][ny][nx]`` arrays, x fastest;
  * coordinates are voxel-index units, voxel (i, j, k) has its centre at
    (x, y, z) = (i, j, k) and the image box is [-0.5, n - 0.5] per axis;
  * points are ``(x, y, z)`` rows of float32.

Nothing here evaluates an objective; it only draws inputs.
"""

from __future__ import annotations

import dataclasses
import itertools
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

H_PLAIN_SSD = 0
H_MOREA_FG = 1
G_CONTINUOUS = 0
G_PAIR_TRANSFER = 1
G_OFF = 2


@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    nz: int
    dtype: str                      # "f32" or "f16" (storage type of both images)
    image_s: np.ndarray             # source image [nz][ny][nx]
    image_t: np.ndarray             # target image [nz][ny][nx]
    ref_points: np.ndarray          # [V][3] float32, reference (initial) mesh
    tets: np.ndarray                # [T][4] int32 shared topology
    tet_label: np.ndarray           # [T] int32 tissue label per tet
    tissue_factor: np.ndarray       # [L] float64 elasticity factor per label
    guid_s: np.ndarray              # [n][3] float32 contour points on the source image
    guid_t: np.ndarray              # [n][3] float32 corresponding points on the target
    guid_group: np.ndarray          # [n] int32 contour group id
    trunc_radius: float             # guidance truncation radius r (voxels)
    sol_src: np.ndarray             # [P][V][3] float32 source-mesh points per solution
    sol_tgt: np.ndarray             # [P][V][3] float32 target-mesh points per solution
    fixed_axes: np.ndarray          # [V][3] bool, coordinate pinned to the box face
    h_mode: int = H_PLAIN_SSD
    g_mode: int = G_CONTINUOUS
    subvoxel_bits: int = 8
    lattice: Tuple[int, int, int] = (0, 0, 0)
    estimator: int = 0              # 0: voxel association, 1: sampled points
    sampling_rate: float = 1.0      # sampled estimator: points per voxel^3 of tet volume

    @property
    def n_points(self) -> int:
        return int(self.ref_points.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_solutions(self) -> int:
        return int(self.sol_src.shape[0])

    def voxels(self) -> int:
        return self.nx * self.ny * self.nz


# ---------------------------------------------------------------------------
# images
# ---------------------------------------------------------------------------

def _displacement(x, y, z, shape_xyz, amp):
    """Smooth sinusoidal displacement field u(x) with amplitude ``amp``."""
    nx, ny, nz = shape_xyz
    sx = np.sin(2.0 * np.pi * x / nx)
    sy = np.sin(2.0 * np.pi * y / ny)
    sz = np.sin(2.0 * np.pi * z / nz)
    return amp * sy * sz, amp * sz * sx, amp * sx * sy


def _paint(x, y, z, background, ellipsoids):
    """Piecewise-constant phantom: the last ellipsoid containing a point wins."""
    out = np.full(np.broadcast(x, y, z).shape, background, dtype=np.float64)
    for (cx, cy, cz, rx, ry, rz, val) in ellipsoids:
        inside = ((x - cx) / rx) ** 2 + ((y - cy) / ry) ** 2 + ((z - cz) / rz) ** 2 <= 1.0
        out[inside] = val
    return out


def phantom_pair(shape_xyz, ellipsoids, background, amp, noise_sigma,
                 seed_s, seed_t, dtype):
    nx, ny, nz = shape_xyz
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    img_s = _paint(x, y, z, background, ellipsoids)
    ux, uy, uz = _displacement(x, y, z, shape_xyz, amp)
    img_t = _paint(x + ux, y + uy, z + uz, background, ellipsoids)
    if noise_sigma > 0:
        img_s = img_s + np.random.default_rng(seed_s).normal(0.0, noise_sigma, img_s.shape)
        img_t = img_t + np.random.default_rng(seed_t).normal(0.0, noise_sigma, img_t.shape)
    np_dtype = np.float32 if dtype == "f32" else np.float16
    return img_s.astype(np_dtype), img_t.astype(np_dtype)


def label_pair(shape_xyz, ellipsoids, amp):
    """Organ masks of a phantom pair: uint8 label images [nz][ny][nx] of the
    source and of the target (warped by the same displacement as the images),
    0 for background and i + 1 inside ellipsoid i (the last one wins)."""
    nx, ny, nz = shape_xyz
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    ids = [e[:6] + (float(i + 1),) for i, e in enumerate(ellipsoids)]
    lab_s = _paint(x, y, z, 0.0, ids)
    ux, uy, uz = _displacement(x, y, z, shape_xyz, amp)
    lab_t = _paint(x + ux, y + uy, z + uz, 0.0, ids)
    return lab_s.astype(np.uint8), lab_t.astype(np.uint8)


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------

def lattice_points(xs: Sequence[float], ys: Sequence[float], zs: Sequence[float]) -> np.ndarray:
    """Points of a rectilinear lattice, vertex id = (k * len(ys) + j) * len(xs) + i."""
    zz, yy, xx = np.meshgrid(np.asarray(zs, np.float64), np.asarray(ys, np.float64),
                             np.asarray(xs, np.float64), indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1).astype(np.float32)


def kuhn_lattice(nxp: int, nyp: int, nzp: int, flip_x: bool = False) -> np.ndarray:
    """Kuhn (Freudenthal) split of every lattice cube into 6 tetrahedra.

    Each tetrahedron follows a monotone path from one cube corner to the
    opposite one, one axis at a time, so all cubes share faces consistently.
    ``flip_x`` mirrors every cube in x, which gives a second conforming
    tetrahedralisation of the same lattice (diagonals along (-1, 1, 1)).
    The vertex order is left as it falls; the evaluator orients tets itself.
    """
    tets = []
    def vid(i, j, k):
        return (k * nyp + j) * nxp + i
    for k in range(nzp - 1):
        for j in range(nyp - 1):
            for i in range(nxp - 1):
                for perm in itertools.permutations(range(3)):
                    c = [0, 0, 0]
                    path = [tuple(c)]
                    for a in perm:
                        c[a] = 1
                        path.append(tuple(c))
                    tet = []
                    for (bx, by, bz) in path:
                        if flip_x:
                            bx = 1 - bx
                        tet.append(vid(i + bx, j + by, k + bz))
                    tets.append(tet)
    return np.asarray(tets, dtype=np.int32)


def vertex_adjacency(tets: np.ndarray, n_points: int) -> List[List[int]]:
    """Mesh edges as adjacency lists (used only to draw connected point subsets)."""
    adj = [set() for _ in range(n_points)]
    for t in tets:
        for a in range(4):
            for b in range(4):
                if a != b:
                    adj[int(t[a])].add(int(t[b]))
    return [sorted(s) for s in adj]


def _fixed_axes(points: np.ndarray, shape_xyz) -> np.ndarray:
    lo = -0.5
    fixed = np.zeros(points.shape, dtype=bool)
    for a in range(3):
        hi = shape_xyz[a] - 0.5
        fixed[:, a] = (points[:, a] == np.float32(lo)) | (points[:, a] == np.float32(hi))
    return fixed


def jitter_population(ref_points: np.ndarray, fixed_axes: np.ndarray, n_sol: int,
                      amplitude, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """Each solution = reference mesh + uniform(-a, a) jitter on both meshes.

    Coordinates pinned to a box face keep their boundary-normal component, so
    every mesh still spans the image box.  ``amplitude`` is a scalar or a
    per-vertex array.
    """
    rng = np.random.default_rng(seed)
    amp = np.broadcast_to(np.asarray(amplitude, np.float64).reshape(-1, 1)
                          if np.ndim(amplitude) else np.float64(amplitude),
                          ref_points.shape)
    out = []
    for _ in range(2):
        j = rng.uniform(-1.0, 1.0, size=(n_sol,) + ref_points.shape) * amp
        j[:, fixed_axes] = 0.0
        out.append((ref_points[None].astype(np.float64) + j).astype(np.float32))
    return out[0], out[1]


def partial_requests(prob: Problem, adjacency: List[List[int]], n_subsets: int,
                     min_pts: int, max_pts: int, sigma: float, seed: int,
                     slots: Optional[np.ndarray] = None):
    """Linkage subsets for GOMEA-style partial re-evaluation.

    For each slot and each of ``n_subsets`` subsets: a breadth-first connected
    neighbourhood of ``min_pts..max_pts`` mesh points around a random seed
    point, moved by N(0, sigma^2) on both meshes (pinned axes stay put).
    Returns a list (one entry per subset round) of dicts with
    ``slot [R]``, ``chg_off [R+1]``, ``chg_pts [C]``, ``chg_src [C][3]``,
    ``chg_tgt [C][3]`` where the new coordinates are absolute (parent + move)
    relative to ``prob.sol_src/sol_tgt`` as given.
    """
    rng = np.random.default_rng(seed)
    if slots is None:
        slots = np.arange(prob.n_solutions, dtype=np.int32)
    rounds = []
    for _ in range(n_subsets):
        offs = [0]
        pts, src, tgt = [], [], []
        for s in slots:
            m = int(rng.integers(min_pts, max_pts + 1))
            start = int(rng.integers(0, prob.n_points))
            seen = [start]
            mark = {start}
            head = 0
            while len(seen) < m and head < len(seen):
                for nb in adjacency[seen[head]]:
                    if nb not in mark and len(seen) < m:
                        mark.add(nb)
                        seen.append(nb)
                head += 1
            ids = np.asarray(sorted(seen), dtype=np.int32)
            mv_s = rng.normal(0.0, sigma, size=(len(ids), 3))
            mv_t = rng.normal(0.0, sigma, size=(len(ids), 3))
            fx = prob.fixed_axes[ids]
            mv_s[fx] = 0.0
            mv_t[fx] = 0.0
            pts.append(ids)
            src.append((prob.sol_src[s, ids].astype(np.float64) + mv_s).astype(np.float32))
            tgt.append((prob.sol_tgt[s, ids].astype(np.float64) + mv_t).astype(np.float32))
            offs.append(offs[-1] + len(ids))
        rounds.append(dict(
            slot=np.asarray(slots, dtype=np.int32),
            chg_off=np.asarray(offs, dtype=np.int32),
            chg_pts=np.concatenate(pts).astype(np.int32),
            chg_src=np.concatenate(src).astype(np.float32).reshape(-1, 3),
            chg_tgt=np.concatenate(tgt).astype(np.float32).reshape(-1, 3),
        ))
    return rounds


# ---------------------------------------------------------------------------
# guidance contours
# ---------------------------------------------------------------------------

def _surface_points(ellipsoids, n, rng):
    pts, grp = [], []
    for m in range(n):
        g = m % len(ellipsoids)
        cx, cy, cz, rx, ry, rz, _ = ellipsoids[g]
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        pts.append((cx + rx * d[0], cy + ry * d[1], cz + rz * d[2]))
        grp.append(g)
    return np.asarray(pts, np.float64), np.asarray(grp, np.int32)


def _invert_displacement(c, shape_xyz, amp, iters=200):
    """Solve y + u(y) = c by fixed-point iteration (u is a contraction here)."""
    y = c.copy()
    for _ in range(iters):
        ux, uy, uz = _displacement(y[:, 0], y[:, 1], y[:, 2], shape_xyz, amp)
        y = c - np.stack([ux, uy, uz], axis=1)
    return y


def _labels(ref_points, tets, ellipsoids):
    cen = ref_points[tets].astype(np.float64).mean(axis=1)
    lab = np.zeros(len(tets), np.int32)
    for e, (cx, cy, cz, rx, ry, rz, _) in enumerate(ellipsoids):
        inside = (((cen[:, 0] - cx) / rx) ** 2 + ((cen[:, 1] - cy) / ry) ** 2
                  + ((cen[:, 2] - cz) / rz) ** 2) <= 1.0
        lab[inside] = e + 1
    return lab


# ---------------------------------------------------------------------------
# assembled problems
# ---------------------------------------------------------------------------

def make_problem(name, shape_xyz, ellipsoids, background, amp, noise_sigma, dtype,
                 xs, ys, zs, n_guid, n_sol, jitter, tissue, seeds,
                 groups=None, flip_x=False, trunc_radius=None,
                 h_mode=H_PLAIN_SSD, g_mode=G_CONTINUOUS, subvoxel_bits=8) -> Problem:
    nx, ny, nz = shape_xyz
    img_s, img_t = phantom_pair(shape_xyz, ellipsoids, background, amp, noise_sigma,
                                seeds[0], seeds[1], dtype)
    ref = lattice_points(xs, ys, zs)
    tets = kuhn_lattice(len(xs), len(ys), len(zs), flip_x=flip_x)
    fixed = _fixed_axes(ref, shape_xyz)
    if callable(jitter):
        jitter = jitter(ref)
    sol_src, sol_tgt = jitter_population(ref, fixed, n_sol, jitter, seeds[2])
    grng = np.random.default_rng(seeds[0] + 1000)
    gell = ellipsoids if groups is None else [ellipsoids[g] for g in groups]
    gs, grp = _surface_points(gell, n_guid, grng)
    gt = _invert_displacement(gs, shape_xyz, amp)
    if trunc_radius is None:
        trunc_radius = 0.025 * nx                 # 2.5% of the image width (App. A.3)
    return Problem(
        name=name, nx=nx, ny=ny, nz=nz, dtype=dtype,
        image_s=img_s, image_t=img_t, ref_points=ref, tets=tets,
        tet_label=_labels(ref, tets, ellipsoids),
        tissue_factor=np.asarray(tissue, np.float64),
        guid_s=gs.astype(np.float32), guid_t=gt.astype(np.float32),
        guid_group=grp, trunc_radius=float(trunc_radius),
        sol_src=sol_src, sol_tgt=sol_tgt, fixed_axes=fixed,
        h_mode=h_mode, g_mode=g_mode, subvoxel_bits=subvoxel_bits,
        lattice=(len(xs), len(ys), len(zs)))


def _even_axis(n, cells):
    return np.linspace(-0.5, n - 0.5, cells + 1)


C0_ELLIPSOIDS = [
    (10.0, 12.0, 16.0, 6.0, 5.0, 7.0, 40.0),
    (21.0, 18.0, 14.0, 5.0, 7.0, 6.0, 80.0),
    (16.0, 22.0, 22.0, 4.0, 4.0, 5.0, 120.0),
]


def make_c0(n_sol: int = 8, **kw) -> Problem:
    """32^3 float32, three ellipsoids 40/80/120, sigma 5 noise, warp amplitude 2,
    5x5x5 lattice (384 tets), 100 guidance pairs, 8 jittered solutions."""
    args = dict(name="c0_32cube_f32", shape_xyz=(32, 32, 32), ellipsoids=C0_ELLIPSOIDS,
                background=0.0, amp=2.0, noise_sigma=5.0, dtype="f32",
                xs=_even_axis(32, 4), ys=_even_axis(32, 4), zs=_even_axis(32, 4),
                n_guid=100, n_sol=n_sol, jitter=1.0,
                tissue=[1.0, 0.5, 2.0, 4.0], seeds=(0, 1, 2))
    args.update(kw)
    return make_problem(**args)


C1_ELLIPSOIDS = [
    (40.0, 44.0, 40.0, 22.0, 18.0, 16.0, 40.0),
    (84.0, 50.0, 52.0, 18.0, 22.0, 18.0, 80.0),
    (62.0, 88.0, 46.0, 16.0, 14.0, 20.0, 120.0),
    (92.0, 92.0, 30.0, 14.0, 12.0, 10.0, 160.0),
    (50.0, 80.0, 70.0, 12.0, 16.0, 12.0, 200.0),
]


def make_c1(n_sol: int = 128, **kw) -> Problem:
    """128x128x96 float32, five ellipsoids, warp amplitude 6, 9x9x7 lattice
    (567 points, 2304 tets), 1000 guidance pairs, population 128."""
    args = dict(name="c1_128x128x96_f32", shape_xyz=(128, 128, 96), ellipsoids=C1_ELLIPSOIDS,
                background=0.0, amp=6.0, noise_sigma=5.0, dtype="f32",
                xs=_even_axis(128, 8), ys=_even_axis(128, 8), zs=_even_axis(96, 6),
                n_guid=1000, n_sol=n_sol, jitter=2.0,
                tissue=[1.0, 0.5, 2.0, 4.0, 1.5, 8.0], seeds=(0, 1, 2))
    args.update(kw)
    return make_problem(**args)


def _graded_axis(n, cells, ratio, flip):
    w = ratio ** np.arange(cells, dtype=np.float64)
    if flip:
        w = w[::-1]
    edges = np.concatenate([[0.0], np.cumsum(w)])
    edges = edges / edges[-1] * n - 0.5
    edges[0], edges[-1] = -0.5, n - 0.5
    # keep lattice coordinates exactly representable on the 1/256-voxel grid
    return np.round(edges * 256.0) / 256.0


C2_ELLIPSOIDS = [
    (128.0, 128.0, 80.0, 118.0, 100.0, 76.0, 40.0),     # body: soft tissue
    (128.0, 110.0, 70.0, 34.0, 28.0, 26.0, 10.0),       # bladder (fluid)
    (128.0, 168.0, 64.0, 18.0, 16.0, 30.0, 30.0),       # rectum
    (90.0, 80.0, 96.0, 26.0, 22.0, 24.0, 60.0),         # bowel
    (70.0, 150.0, 60.0, 16.0, 20.0, 40.0, 700.0),       # left pelvic bone
    (186.0, 150.0, 60.0, 16.0, 20.0, 40.0, 1200.0),     # right pelvic bone
    (128.0, 196.0, 80.0, 12.0, 12.0, 60.0, 1500.0),     # spine
]


def make_c2(n_sol: int = 256, **kw) -> Problem:
    """256x256x160 float16 HU-like volumes (air -1000, soft tissue 0-80, bone
    700-1500), warp amplitude 6, graded 13x13x9 lattice (1521 points,
    6912 tets, cell volumes spanning ~3 orders of magnitude), 300 guidance
    pairs on six organ/bone contours, population 256."""
    rng = np.random.default_rng(4)
    flips = rng.integers(0, 2, size=3).astype(bool)
    xs = _graded_axis(256, 12, 1.25, flips[0])
    ys = _graded_axis(256, 12, 1.25, flips[1])
    zs = _graded_axis(160, 8, 1.25, flips[2])

    def jit(ref):
        # 10% of the smallest neighbouring cell width per vertex
        amp = np.empty(len(ref))
        def local(axis_vals, v):
            k = int(np.argmin(np.abs(axis_vals - v)))
            ws = []
            if k > 0:
                ws.append(axis_vals[k] - axis_vals[k - 1])
            if k + 1 < len(axis_vals):
                ws.append(axis_vals[k + 1] - axis_vals[k])
            return min(ws)
        for m, p in enumerate(ref):
            amp[m] = 0.1 * min(local(xs, p[0]), local(ys, p[1]), local(zs, p[2]))
        return amp

    args = dict(name="c2_256x256x160_f16", shape_xyz=(256, 256, 160), ellipsoids=C2_ELLIPSOIDS,
                background=-1000.0, amp=6.0, noise_sigma=10.0, dtype="f16",
                xs=xs, ys=ys, zs=zs, n_guid=300, n_sol=n_sol, jitter=jit,
                tissue=[1.0, 1.0, 0.2, 0.8, 1.0, 10.0, 10.0, 10.0], seeds=(10, 11, 12),
                groups=[1, 2, 3, 4, 5, 6])
    args.update(kw)
    return make_problem(**args)


def make_c4(seed: int = 5, max_problems: int = 16) -> List[Problem]:
    """16 problems of uneven sizes: extents log-uniform between 64^3 and
    192x192x128 (FP16), lattices of ~200-1500 points, populations 32-256."""
    rng = np.random.default_rng(seed)
    probs = []
    for m in range(max_problems):
        t = rng.uniform(0.0, 1.0)
        nx = int(round(64 * (192 / 64) ** t))
        ny = int(round(64 * (192 / 64) ** rng.uniform(0.0, 1.0)))
        nz = int(round(64 * (128 / 64) ** rng.uniform(0.0, 1.0)))
        target_pts = int(round(200 * (1500 / 200) ** rng.uniform(0.0, 1.0)))
        # lattice dims roughly proportional to the extents
        scale = (target_pts / (nx * ny * nz)) ** (1.0 / 3.0)
        lx = max(3, int(round(nx * scale)))
        ly = max(3, int(round(ny * scale)))
        lz = max(3, int(round(nz * scale)))
        pop = int(2 ** rng.integers(5, 9))         # 32..256
        ell = []
        for e in range(4):
            c = rng.uniform(0.3, 0.7, size=3) * np.array([nx, ny, nz])
            r = rng.uniform(0.08, 0.2, size=3) * np.array([nx, ny, nz])
            ell.append((c[0], c[1], c[2], r[0], r[1], r[2], float(40 * (e + 1))))
        spacing = min(nx / (lx - 1), ny / (ly - 1), nz / (lz - 1))
        probs.append(make_problem(
            name=f"c4_p{m:02d}_{nx}x{ny}x{nz}_f16", shape_xyz=(nx, ny, nz), ellipsoids=ell,
            background=0.0, amp=4.0, noise_sigma=5.0, dtype="f16",
            xs=np.round(_even_axis(nx, lx - 1) * 256) / 256,
            ys=np.round(_even_axis(ny, ly - 1) * 256) / 256,
            zs=np.round(_even_axis(nz, lz - 1) * 256) / 256,
            n_guid=400, n_sol=pop, jitter=0.1 * spacing,
            tissue=[1.0, 0.5, 2.0, 4.0, 8.0], seeds=(100 + 3 * m, 101 + 3 * m, 102 + 3 * m)))
    return probs


CONFIGS = {
    "c0": make_c0,
    "c1": make_c1,
    "c2": make_c2,
}
