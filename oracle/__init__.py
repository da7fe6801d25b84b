"""ctypes wrapper around the plain FP64 MOREA oracle (``morea_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2303_04873_gb300``) never imports it, and it never imports the
product.  ``build()`` compiles the C oracle with the host compiler into
``oracle/_build/`` (plain C99 + libm, so it builds the same on x86-64 and
aarch64).

Parity status of each oracle function (what pins it) is listed in
``tests/test_oracle_pins.py``; every function here is pinned there.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmorea_oracle.so")
_SRC = os.path.join(_HERE, "morea_oracle.c")

TET_DTYPE = np.dtype([
    ("e_img", "<f8", (2,)), ("e_guid", "<f8", (2,)),
    ("n_vox", "<i8", (2,)), ("n_gp", "<i8", (2,)),
    ("e_mag", "<f8"), ("sev", "<u8"), ("folded", "<i4"), ("pad", "<i4"),
    ("amb_n", "<i8", (2,)), ("amb_slack", "<f8", (2,)),
])


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("img_s", ctypes.c_void_p), ("img_t", ctypes.c_void_p),
        ("n_points", ctypes.c_int32), ("n_tets", ctypes.c_int32),
        ("tets", ctypes.c_void_p), ("ref_points", ctypes.c_void_p),
        ("tet_label", ctypes.c_void_p), ("tissue_factor", ctypes.c_void_p),
        ("n_labels", ctypes.c_int32), ("n_guid", ctypes.c_int32),
        ("guid_s", ctypes.c_void_p), ("guid_t", ctypes.c_void_p), ("guid_group", ctypes.c_void_p),
        ("trunc_radius", ctypes.c_double),
        ("h_mode", ctypes.c_int32), ("g_mode", ctypes.c_int32),
        ("subvoxel_bits", ctypes.c_int32), ("estimator", ctypes.c_int32),
        ("sampling_rate", ctypes.c_double), ("tissue_mask", ctypes.c_void_p),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("obj", ctypes.c_double * 3), ("severity", ctypes.c_double),
        ("s_img", ctypes.c_double), ("s_guid", ctypes.c_double), ("s_mag", ctypes.c_double),
        ("n_vox", ctypes.c_int64), ("n_gp", ctypes.c_int64), ("n_folded", ctypes.c_int64),
        ("sev_raw", ctypes.c_uint64), ("folded", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]

    def as_dict(self):
        return dict(obj=np.array(self.obj[:], np.float64), severity=self.severity,
                    s_img=self.s_img, s_guid=self.s_guid, s_mag=self.s_mag,
                    n_vox=int(self.n_vox), n_gp=int(self.n_gp), n_folded=int(self.n_folded),
                    sev_raw=int(self.sev_raw), folded=int(self.folded))


_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no vendor code)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.orc_setup.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(ctypes.c_void_p)]
        L.orc_setup.restype = ctypes.c_int
        L.orc_free.argtypes = [ctypes.c_void_p]
        L.orc_eval.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.POINTER(_Result)]
        L.orc_eval.restype = ctypes.c_int
        L.orc_eval_tet.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_void_p]
        L.orc_eval_partial.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [
            ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(_Result), ctypes.POINTER(_Result),
            ctypes.POINTER(ctypes.c_int32)]
        L.orc_eval_partial.restype = ctypes.c_int
        L.orc_n_groups.argtypes = [ctypes.c_void_p]
        L.orc_radius.argtypes = [ctypes.c_void_p]
        L.orc_radius.restype = ctypes.c_double
        L.orc_oriented_tets.argtypes = [ctypes.c_void_p]
        L.orc_oriented_tets.restype = ctypes.c_void_p
        L.orc_distance.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.orc_distance.restype = ctypes.c_void_p
        L.orc_snap1.argtypes = [ctypes.c_float, ctypes.c_int, ctypes.c_int]
        L.orc_snap1.restype = ctypes.c_int64
        L.orc_orient.argtypes = [ctypes.c_void_p] * 4
        L.orc_orient.restype = ctypes.c_int64
        L.orc_inside.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_inside.restype = ctypes.c_int
        L.orc_trilinear.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p]
        L.orc_trilinear.restype = ctypes.c_double
        L.orc_h.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_h.restype = ctypes.c_double
        L.orc_sobol.argtypes = [ctypes.c_uint64, ctypes.c_int]
        L.orc_sobol.restype = ctypes.c_uint32
        L.orc_fnv1a64.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
        L.orc_fnv1a64.restype = ctypes.c_uint64
        L.orc_splitmix64.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_copy_shifts.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_sample_lambda.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        L.orc_repair.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.c_double, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
        L.orc_repair.restype = ctypes.c_int
        L.orc_repair_sigma.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        L.orc_repair_sigma.restype = ctypes.c_double
        L.orc_dvf.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p]
        L.orc_set_perturbation.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.orc_cdelta.argtypes = [ctypes.c_void_p]
        L.orc_cdelta.restype = ctypes.c_void_p
        L.orc_dvf.restype = ctypes.c_int
        L.orc_gexp.argtypes = [ctypes.c_double]
        L.orc_gexp.restype = ctypes.c_double
        L.orc_init_noise.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int]
        L.orc_init_noise.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def getattr_default(g, name, default):
    try:
        return g(name)
    except AttributeError:
        return default


class Oracle:
    """One registration problem set up in the oracle.

    ``prob`` is any object with the attributes of ``synth.Problem`` (images,
    topology, reference points, labels, tissue factors, guidance pairs,
    modes).  Keyword overrides replace single attributes.
    """

    def __init__(self, prob, **override):
        g = lambda name: override.get(name, getattr(prob, name))
        L = lib()
        self._keep = []

        def arr(x, dt):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x), dtype=dt)
            self._keep.append(a)
            return a

        img_s = arr(np.asarray(g("image_s")).astype(np.float64), np.float64)
        img_t = arr(np.asarray(g("image_t")).astype(np.float64), np.float64)
        nz, ny, nx = img_s.shape
        tets = arr(g("tets"), np.int32)
        ref = arr(g("ref_points"), np.float32)
        lab = arr(g("tet_label"), np.int32)
        tis = arr(g("tissue_factor"), np.float64)
        gs = arr(g("guid_s"), np.float32)
        gt = arr(g("guid_t"), np.float32)
        gg = arr(g("guid_group"), np.int32)
        n_guid = 0 if gs is None else int(gs.shape[0])
        P = _Problem(nx=nx, ny=ny, nz=nz, pad0=0, img_s=_ptr(img_s), img_t=_ptr(img_t),
                     n_points=int(ref.shape[0]), n_tets=int(tets.shape[0]),
                     tets=_ptr(tets), ref_points=_ptr(ref), tet_label=_ptr(lab),
                     tissue_factor=_ptr(tis), n_labels=0 if tis is None else int(tis.shape[0]),
                     n_guid=n_guid, guid_s=_ptr(gs), guid_t=_ptr(gt), guid_group=_ptr(gg),
                     trunc_radius=float(g("trunc_radius")), h_mode=int(g("h_mode")),
                     g_mode=int(g("g_mode")), subvoxel_bits=int(g("subvoxel_bits")),
                     estimator=int(getattr_default(g, "estimator", 0)),
                     sampling_rate=float(np.float32(getattr_default(g, "sampling_rate", 1.0))),
                     tissue_mask=_ptr(arr(getattr_default(g, "tissue_mask", None), np.uint8)))
        self._P = P
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n_points = int(ref.shape[0])
        self.n_tets = int(tets.shape[0])
        h = ctypes.c_void_p()
        rc = L.orc_setup(ctypes.byref(P), ctypes.byref(h))
        if rc != 0:
            raise OracleError(f"oracle set-up rejected the problem (code {rc})")
        self._h = h
        self._L = L

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_free(h)
            self._h = None

    # -- queries ---------------------------------------------------------
    @property
    def n_groups(self) -> int:
        return int(self._L.orc_n_groups(self._h))

    @property
    def radius(self) -> float:
        return float(self._L.orc_radius(self._h))

    def oriented_tets(self) -> np.ndarray:
        p = self._L.orc_oriented_tets(self._h)
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_int32)),
                                     shape=(self.n_tets, 4)).copy()

    def cdelta(self) -> np.ndarray:
        """Elasticity factor c_delta of every tet (App. A.1)."""
        p = self._L.orc_cdelta(self._h)
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_double)), shape=(self.n_tets,)).copy()

    def distance_map(self, side: int, group: int) -> np.ndarray:
        p = self._L.orc_distance(self._h, side, group)
        if not p:
            raise OracleError("no distance map for that side/group")
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_double)),
                                     shape=(self.nz, self.ny, self.nx)).copy()

    # -- evaluation ------------------------------------------------------
    def eval(self, src, tgt, with_tets: bool = False):
        src = np.ascontiguousarray(src, dtype=np.float32)
        tgt = np.ascontiguousarray(tgt, dtype=np.float32)
        recs = np.zeros(self.n_tets, TET_DTYPE) if with_tets else None
        res = _Result()
        rc = self._L.orc_eval(self._h, _ptr(src), _ptr(tgt), _ptr(recs), ctypes.byref(res))
        if rc != 0:
            raise OracleError(f"oracle eval failed ({rc})")
        out = res.as_dict()
        out["_raw"] = res
        if with_tets:
            out["tets"] = recs
        return out

    def eval_tet(self, src, tgt, t: int):
        src = np.ascontiguousarray(src, dtype=np.float32)
        tgt = np.ascontiguousarray(tgt, dtype=np.float32)
        rec = np.zeros(1, TET_DTYPE)
        self._L.orc_eval_tet(self._h, _ptr(src), _ptr(tgt), int(t), _ptr(rec))
        return rec[0]

    def repair(self, src, tgt, noise, max_points: int, scale: float = 1.0, fixed=None):
        """Repair (R14) of one solution; returns (src, tgt, moved, severity).
        fixed: optional [V] uint8 axis bits of coordinates that stay."""
        s = np.array(src, dtype=np.float32, copy=True, order="C")
        t = np.array(tgt, dtype=np.float32, copy=True, order="C")
        z = np.ascontiguousarray(noise, dtype=np.float32)
        assert z.size >= max_points * 64 * 3
        fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        sev = ctypes.c_uint64(0)
        moved = self._L.orc_repair(self._h, _ptr(s), _ptr(t), _ptr(z), int(max_points), float(scale),
                                   ctypes.byref(sev), _ptr(fx))
        if moved < 0:
            raise OracleError("oracle repair failed")
        S = float(1 << int(self._P.subvoxel_bits))
        return s, t, int(moved), sev.value / (6.0 * S * S * S)

    def dvf(self, src, tgt, side: int, labels_own=None, labels_other=None, n_labels: int = 0):
        """R15: displacement field [nz][ny][nx][3] (NaN outside) and, with
        labels, the per-label counts [n_labels][3] (own, pulled back, both)."""
        s = np.ascontiguousarray(src, dtype=np.float32)
        t = np.ascontiguousarray(tgt, dtype=np.float32)
        out = np.zeros((self.nz, self.ny, self.nx, 3), np.float64)
        counts = None
        lo = lt = None
        if labels_own is not None:
            lo = np.ascontiguousarray(labels_own, dtype=np.uint8)
            lt = np.ascontiguousarray(labels_other, dtype=np.uint8)
            counts = np.zeros((n_labels, 3), np.int64)
        rc = self._L.orc_dvf(self._h, _ptr(s), _ptr(t), int(side), _ptr(out), _ptr(lo), _ptr(lt), int(n_labels),
                             _ptr(counts), None, None)
        if rc != 0:
            raise OracleError("oracle dvf failed")
        return out, counts

    def warp_labels(self, src, tgt, side: int, labels_other, candidates: bool = False):
        """R15/R17: the other image's label at the voxel nearest to T(p) for
        every voxel centre p covered by an unfolded copy of mesh ``side``;
        255 where no copy covers p.  With ``candidates``, also the [nz][ny][nx][8]
        labels the perturbation report allows per voxel (``set_perturbation``)."""
        s = np.ascontiguousarray(src, dtype=np.float32)
        t = np.ascontiguousarray(tgt, dtype=np.float32)
        lt = np.ascontiguousarray(labels_other, dtype=np.uint8)
        warped = np.zeros((self.nz, self.ny, self.nx), np.uint8)
        cand = np.zeros((self.nz, self.ny, self.nx, 8), np.uint8) if candidates else None
        rc = self._L.orc_dvf(self._h, _ptr(s), _ptr(t), int(side), None, None, _ptr(lt), 0, None, _ptr(warped),
                             _ptr(cand))
        if rc != 0:
            raise OracleError("oracle warp_labels failed")
        return (warped, cand) if candidates else warped

    def set_perturbation(self, gamma_pos: float, gamma_val: float):
        """Turn on (radii > 0) or off the perturbation report: per voxel the
        decisions of R9 (case of h) and R15 (nearest voxel) that change when
        the mapped position moves by gamma_pos (|t0| + |M||p - s0| + 1) per
        axis and the sample by the matching radius plus gamma_val times the
        largest stored value.  Returned values never change."""
        self._L.orc_set_perturbation(self._h, float(gamma_pos), float(gamma_val))

    def init_noise(self, X, kernels, fixed=None, max_rounds: int = 20):
        """R18: one mesh X [V][3] after the attraction rounds of the kernels
        [K][5] = (cx, cy, cz, sigma, a); returns (X', rounds kept)."""
        x = np.array(X, dtype=np.float32, copy=True, order="C")
        k = np.ascontiguousarray(kernels, dtype=np.float32).reshape(-1, 5)
        f = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        r = self._L.orc_init_noise(self._h, _ptr(x), _ptr(k), int(k.shape[0]), _ptr(f), int(max_rounds))
        if r < 0:
            raise OracleError("oracle init_noise failed")
        return x, int(r)

    def repair_sigma(self, X, v: int, scale: float = 1.0) -> float:
        x = np.ascontiguousarray(X, dtype=np.float32)
        return float(self._L.orc_repair_sigma(self._h, _ptr(x), int(v), float(scale)))

    def eval_partial(self, old_src, old_tgt, new_src, new_tgt, changed, old_result):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (old_src, old_tgt, new_src, new_tgt)]
        chg = np.ascontiguousarray(changed, dtype=np.int32)
        res = _Result()
        na = ctypes.c_int32(0)
        rc = self._L.orc_eval_partial(self._h, *[_ptr(a) for a in arrs], int(chg.size), _ptr(chg),
                                      ctypes.byref(old_result["_raw"]), ctypes.byref(res),
                                      ctypes.byref(na))
        if rc != 0:
            raise OracleError(f"oracle partial eval failed ({rc})")
        out = res.as_dict()
        out["_raw"] = res
        out["n_affected"] = int(na.value)
        return out


# -- building blocks, exposed for the pins -----------------------------------

def gexp(t: float) -> float:
    """R18's exp for t <= 0 (range reduction by ln 2 + Taylor series)."""
    return float(lib().orc_gexp(float(t)))


def snap1(x: float, n: int, k: int) -> int:
    return int(lib().orc_snap1(ctypes.c_float(x), n, k))


def orient(a, b, c, d) -> int:
    arrs = [np.ascontiguousarray(v, dtype=np.int64) for v in (a, b, c, d)]
    return int(lib().orc_orient(*[_ptr(v) for v in arrs]))


def inside(tet12, p) -> bool:
    t = np.ascontiguousarray(tet12, dtype=np.int64).reshape(12)
    q = np.ascontiguousarray(p, dtype=np.int64).reshape(3)
    return bool(lib().orc_inside(_ptr(t), _ptr(q)))


def trilinear(img: np.ndarray, y) -> float:
    a = np.ascontiguousarray(img, dtype=np.float64)
    nz, ny, nx = a.shape
    yy = np.ascontiguousarray(y, dtype=np.float64).reshape(3)
    return float(lib().orc_trilinear(_ptr(a), nx, ny, nz, _ptr(yy)))


def h(mode: int, a: float, b: float) -> float:
    return float(lib().orc_h(mode, a, b))


# -- the sampled estimator (R13) ---------------------------------------------

def sobol(j: int, d: int) -> int:
    """Coordinate d (0..3) of the unshifted Sobol point with Gray-code index j, as uint32."""
    return int(lib().orc_sobol(j, d))


def fnv1a64(data: bytes) -> int:
    buf = ctypes.create_string_buffer(data, len(data))
    return int(lib().orc_fnv1a64(ctypes.cast(buf, ctypes.c_void_p), len(data)))


def splitmix64_outputs(state: int, n: int):
    s = ctypes.c_uint64(state)
    return [int(lib().orc_splitmix64(ctypes.byref(s))) for _ in range(n)]


def copy_shifts(tet12) -> np.ndarray:
    t = np.ascontiguousarray(tet12, dtype=np.int64).reshape(12)
    out = np.zeros(4, np.uint32)
    lib().orc_copy_shifts(_ptr(t), _ptr(out))
    return out


def sample_lambda(shift, j: int) -> np.ndarray:
    sh = np.ascontiguousarray(shift, dtype=np.uint32).reshape(4)
    out = np.zeros(4, np.float64)
    lib().orc_sample_lambda(_ptr(sh), int(j), _ptr(out))
    return out
