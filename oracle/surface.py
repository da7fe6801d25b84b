"""Surface distances between two label masks: the Hausdorff distance and
its 95th percentile, the evaluation metrics of Sec. 5 (reading R17).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy: the
surfaces by explicit neighbour tests, every directed distance by brute
force over all surface pairs in exact int64, percentiles by sorting.

Reading R17 (the paper defines the Hausdorff distance as the largest
minimal distance between the points of two object surfaces, and also
reports its 95th percentile; it does not fix the discretisation):
  - The surface of a mask M (voxels with label l) is the set of voxels of
    M with at least one of their six face neighbours outside M; a
    neighbour beyond the image border is outside M.
  - Distances are Euclidean between voxel centres, in voxel units.
  - d(a, S) = min over s in S of |a - s|; the directed distances of S_A
    are d(a, S_B) for every a in S_A, and those of S_B likewise.
  - HD = the largest directed distance of either surface.
  - HD95 = the larger of the two directed 95th percentiles, each by
    nearest rank: the ceil(0.95 n)-th smallest of the n directed
    distances of that surface.
  - An empty surface (the label is absent from a mask) gives NaN.
"""

from __future__ import annotations

import numpy as np


def surface(mask: np.ndarray) -> np.ndarray:
    """Boolean surface of a boolean [nz][ny][nx] mask (R17)."""
    m = np.asarray(mask, bool)
    p = np.pad(m, 1, constant_values=False)
    inner = m.copy()
    nz, ny, nx = m.shape
    for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        inner &= p[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return m & ~inner


def directed_sq(a_pts: np.ndarray, b_pts: np.ndarray, chunk: int = 512) -> np.ndarray:
    """Squared distance from every point of a_pts [n][3] to its nearest point
    of b_pts [m][3], exact in int64, by brute force."""
    a = np.asarray(a_pts, np.int64)
    b = np.asarray(b_pts, np.int64)
    out = np.empty(len(a), np.int64)
    for s in range(0, len(a), chunk):
        d = a[s:s + chunk, None, :] - b[None, :, :]
        out[s:s + chunk] = (d * d).sum(-1).min(1)
    return out


def nearest_rank(d_sq: np.ndarray, q_percent: int = 95) -> int:
    """The ceil(q n / 100)-th smallest value (1-based nearest rank)."""
    n = len(d_sq)
    r = (q_percent * n + 99) // 100
    return int(np.sort(d_sq)[max(r, 1) - 1])


def hausdorff(labels_a: np.ndarray, labels_b: np.ndarray, label: int):
    """(HD, HD95, |S_A|, |S_B|) of label ``label`` in two label images."""
    sa = np.argwhere(surface(np.asarray(labels_a) == label))
    sb = np.argwhere(surface(np.asarray(labels_b) == label))
    if len(sa) == 0 or len(sb) == 0:
        return float("nan"), float("nan"), len(sa), len(sb)
    dab = directed_sq(sa, sb)
    dba = directed_sq(sb, sa)
    hd_sq = max(int(dab.max()), int(dba.max()))
    p95_sq = max(nearest_rank(dab), nearest_rank(dba))
    return float(np.sqrt(float(hd_sq))), float(np.sqrt(float(p95_sq))), len(sa), len(sb)
