"""ctypes binding of libmorea (include/morea.h): argument marshalling only.

Every step of the evaluation runs in the library's CUDA kernels; this module
checks tensor shapes, dtypes and devices, passes raw pointers and the current
torch CUDA stream, and turns status codes into exceptions.  PyTorch supplies
device memory and streams.  There is no CPU path: if ``libmorea.so`` is not
built, importing this module fails.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmorea.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTIMPL, EDEVICE = range(7)
F32, F16 = 0, 1
H_PLAIN_SSD, H_MOREA_FG = 0, 1
G_CONTINUOUS, G_PAIR_TRANSFER, G_OFF = 0, 1, 2

DEV_BAD_POINT = 0x1
DEV_TOO_MANY = 0x2
DEV_DUPLICATE = 0x4
DEV_OVERFLOW = 0x8
DEV_BAD_SLOT = 0x10
DEV_TIMEOUT = 0x20

# exported entry points, in header order (checked by the tests against include/morea.h)
ENTRY_POINTS = (
    "morea_create_problem", "morea_destroy_problem", "morea_eval_full", "morea_eval_partial",
    "morea_commit_partial", "morea_check_folds", "morea_read_records", "morea_read_totals",
    "morea_partial_features", "morea_mlp_create", "morea_mlp_destroy", "morea_mlp_info",
    "morea_mlp_set_params", "morea_mlp_get_params", "morea_mlp_forward", "morea_mlp_gradients",
    "morea_mlp_train_step", "morea_mlp_device_status", "morea_repair_folds", "morea_displacement",
    "morea_parallel_groups", "morea_init_noise", "morea_warp_labels", "morea_cluster", "morea_slot_objectives",
    "morea_sample_elements_workspace", "morea_sample_elements", "morea_surface_distance_workspace", "morea_surface_distance",
    "morea_device_status", "morea_problem_info", "morea_batch_create", "morea_batch_destroy",
    "morea_batch_eval_full", "morea_batch_capture", "morea_batch_replay", "morea_batch_latency", "morea_set_launch",
    "morea_batch_set_launch", "morea_profile", "morea_profile_read", "morea_fold_magnitude_noalloc",
    "morea_status_string",
)
MAX_BATCH = 64
NOALLOC_MAX_TET_EVALS = 524288

TET_RECORD_DTYPE = np.dtype([
    ("e_img", "<f4", (2,)), ("e_guid", "<f4", (2,)), ("n_vox", "<i4", (2,)), ("n_gp", "<i4", (2,)),
    ("e_mag", "<f4"), ("folded", "<u4"), ("sev", "<u8"),
])
TOTALS_DTYPE = np.dtype([
    ("s_img", "<f8"), ("s_guid", "<f8"), ("s_mag", "<f8"), ("n_vox", "<i8"), ("n_gp", "<i8"),
    ("n_folded", "<i8"), ("sev", "<u8"), ("reserved", "<i8"),
])


class MoreaError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


class ProblemDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("dtype", ctypes.c_int32),
        ("image_s", ctypes.c_void_p), ("image_t", ctypes.c_void_p),
        ("n_points", ctypes.c_int32), ("n_tets", ctypes.c_int32),
        ("tets", ctypes.c_void_p), ("ref_points", ctypes.c_void_p), ("tet_label", ctypes.c_void_p),
        ("tissue_factor", ctypes.c_void_p), ("n_labels", ctypes.c_int32), ("n_guid", ctypes.c_int32),
        ("guid_s", ctypes.c_void_p), ("guid_t", ctypes.c_void_p), ("guid_group", ctypes.c_void_p),
        ("trunc_radius", ctypes.c_double), ("h_mode", ctypes.c_int32), ("g_mode", ctypes.c_int32),
        ("subvoxel_bits", ctypes.c_int32), ("max_solutions", ctypes.c_int32),
        ("max_requests", ctypes.c_int32), ("max_changed", ctypes.c_int32),
        ("estimator", ctypes.c_int32), ("sampling_rate", ctypes.c_float),
        ("tissue_mask", ctypes.c_void_p),
    ]


_lib = None


def lib():
    """Load libmorea.so (built in-tree by ``paper_2303_04873_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmorea.so is not built ({LIB_PATH}); run paper_2303_04873_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u8p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p
    L.morea_create_problem.argtypes = [ctypes.POINTER(ProblemDesc), vp, ctypes.POINTER(vp)]
    L.morea_destroy_problem.argtypes = [vp]
    L.morea_eval_full.argtypes = [vp, i32, vp, vp, vp, vp, u8p, vp, vp]
    L.morea_eval_partial.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, u8p, vp, u8p, vp]
    L.morea_commit_partial.argtypes = [vp, i32, u8p, vp]
    L.morea_check_folds.argtypes = [vp, i32, vp, vp, u8p, vp, vp]
    L.morea_repair_folds.argtypes = [vp, i32, vp, vp, vp, i32, ctypes.c_float, vp, vp, vp, vp]
    L.morea_displacement.argtypes = [vp, vp, vp, i32, vp, vp, vp, i32, vp, vp]
    L.morea_parallel_groups.argtypes = [i32, i32, vp, i32, vp, vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.morea_warp_labels.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.morea_init_noise.argtypes = [vp, i32, vp, vp, vp, i32, vp, i32, vp, vp]
    L.morea_cluster.argtypes = [i32, vp, ctypes.c_double, i32, i32, ctypes.POINTER(i32), vp, ctypes.POINTER(i32),
                                vp, vp]
    L.morea_slot_objectives.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.morea_sample_elements_workspace.argtypes = [i32, i32]
    L.morea_sample_elements.argtypes = [vp, i32, vp, vp, i32, i32, vp, i32, vp, vp, vp, i32, vp, vp, vp, vp, vp,
                                        ctypes.c_size_t, vp, vp, vp]
    L.morea_surface_distance_workspace.argtypes = [i32, i32, i32]
    L.morea_surface_distance.argtypes = [i32, i32, i32, vp, vp, i32, vp, ctypes.c_size_t, vp, vp]
    L.morea_read_records.argtypes = [vp, i32, vp, vp, vp]
    L.morea_read_totals.argtypes = [vp, i32, vp, vp, vp]
    L.morea_device_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint32)]
    L.morea_problem_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
    L.morea_partial_features.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
    L.morea_mlp_create.argtypes = [i32, i32, i32, i32, i32, ctypes.POINTER(vp)]
    L.morea_mlp_destroy.argtypes = [vp]
    L.morea_mlp_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i32)]
    L.morea_mlp_set_params.argtypes = [vp, vp, vp]
    L.morea_mlp_get_params.argtypes = [vp, vp, vp]
    L.morea_mlp_forward.argtypes = [vp, i32, vp, vp, vp]
    L.morea_mlp_gradients.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.morea_mlp_train_step.argtypes = [vp, i32, vp, vp, ctypes.c_float, vp, vp]
    L.morea_mlp_device_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), vp]
    pa = ctypes.POINTER(ctypes.c_void_p)
    L.morea_batch_create.argtypes = [pa, i32, ctypes.POINTER(vp)]
    L.morea_batch_destroy.argtypes = [vp]
    L.morea_batch_eval_full.argtypes = [vp, ctypes.POINTER(i32), pa, pa, pa, pa, pa, vp]
    L.morea_batch_capture.argtypes = [vp, ctypes.POINTER(i32), pa, pa, pa, pa, pa, vp]
    L.morea_batch_replay.argtypes = [vp, vp]
    L.morea_batch_latency.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.morea_set_launch.argtypes = [vp, i32, i32]
    L.morea_batch_set_launch.argtypes = [vp, i32, i32]
    L.morea_profile.argtypes = [vp, ctypes.c_uint32]
    L.morea_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64)]
    L.morea_fold_magnitude_noalloc.argtypes = [i32, i32, i32, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, u8p,
                                               vp, vp]
    L.morea_status_string.argtypes = [i32]
    L.morea_status_string.restype = ctypes.c_char_p
    for name in ENTRY_POINTS:
        if name not in ("morea_status_string", "morea_surface_distance_workspace",
                        "morea_sample_elements_workspace"):
            getattr(L, name).restype = ctypes.c_int
    L.morea_surface_distance_workspace.restype = ctypes.c_size_t
    L.morea_sample_elements_workspace.restype = ctypes.c_size_t
    _lib = L
    return L


def parallel_groups(n_points: int, tets):
    """Edge FOS elements [m][2] and their parallel group ids [m] (Sec. 4.2.1; host call)."""
    t = np.ascontiguousarray(tets, dtype=np.int32)
    cap = max(1, int(n_points))
    el = np.zeros((cap, 2), np.int32)
    grp = np.zeros(cap, np.int32)
    m, g = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().morea_parallel_groups(int(n_points), int(t.shape[0]), t.ctypes.data_as(ctypes.c_void_p), cap,
                                       el.ctypes.data_as(ctypes.c_void_p), grp.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(m), ctypes.byref(g)), "morea_parallel_groups")
    return el[:m.value].copy(), grp[:m.value].copy()


NO_LABEL = 255


def sample_elements_workspace(n_clusters: int, n_elements: int) -> int:
    """Device bytes Problem.sample_elements needs for its models."""
    n = int(lib().morea_sample_elements_workspace(int(n_clusters), int(n_elements)))
    if n == 0:
        raise MoreaError(EINVAL, "morea_sample_elements_workspace")
    return n


def cluster(obj, tau: float = 0.35, k: int = 10, iters: int = 10):
    """Selection and balanced clustering of MO-RV-GOMEA (Sec. 3; host call).
    Returns (selected indices, members [k][c] population indices, cluster of
    every population member)."""
    o = np.ascontiguousarray(obj, dtype=np.float64)
    n = int(o.shape[0])
    sel = np.zeros(n, np.int32)
    mem = np.zeros((int(k), n), np.int32)
    pc = np.zeros(n, np.int32)
    ns, c = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().morea_cluster(n, o.ctypes.data_as(ctypes.c_void_p), float(tau), int(k), int(iters), ctypes.byref(ns),
                               sel.ctypes.data_as(ctypes.c_void_p), ctypes.byref(c), mem.ctypes.data_as(ctypes.c_void_p),
                               pc.ctypes.data_as(ctypes.c_void_p)), "morea_cluster")
    return sel[:ns.value].copy(), mem[:, :c.value].copy(), pc


def surface_distance_workspace(nx: int, ny: int, nz: int) -> int:
    """Device bytes surface_distance needs for an nx x ny x nz image."""
    n = int(lib().morea_surface_distance_workspace(int(nx), int(ny), int(nz)))
    if n == 0:
        raise MoreaError(EINVAL, "morea_surface_distance_workspace")
    return n


def surface_distance(a: torch.Tensor, b: torch.Tensor, label: int, work: Optional[torch.Tensor] = None,
                     out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Hausdorff distance, its 95th percentile (voxel units) and the two
    surface sizes of label ``label`` in two device uint8 label images
    [nz][ny][nx] (Sec. 5): a device float64 tensor [4] (``out`` if given,
    contiguous).  ``work`` may be a reused device uint8 buffer of
    surface_distance_workspace() bytes."""
    nz, ny, nx = (int(x) for x in a.shape)
    need = surface_distance_workspace(nx, ny, nz)
    if work is None:
        work = torch.empty((need,), dtype=torch.uint8, device=a.device)
    if out is None:
        out = torch.empty((4,), dtype=torch.float64, device=a.device)
    _check(lib().morea_surface_distance(
        nx, ny, nz, _dev(a, torch.uint8, (nz, ny, nx), "a"), _dev(b, torch.uint8, (nz, ny, nx), "b"), int(label),
        _dev(work, torch.uint8, None, "work"), ctypes.c_size_t(work.numel()), _dev(out, torch.float64, (4,), "out"),
        _stream(stream)), "morea_surface_distance")
    return out


def status_string(code: int) -> str:
    return lib().morea_status_string(int(code)).decode()


def _check(code: int, what: str):
    if code != OK:
        raise MoreaError(code, what)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t: Optional[torch.Tensor], dtype, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


class Problem:
    """A registration problem resident on the current CUDA device.

    ``prob`` is any object with the attributes of ``synth.Problem`` (images,
    topology, reference points, labels, tissue factors, guidance pairs,
    modes).  Keyword overrides replace single attributes.
    """

    def __init__(self, prob, max_solutions: Optional[int] = None, max_requests: int = 0,
                 max_changed: int = 64, stream=None, **override):
        g = lambda name: override.get(name, getattr(prob, name))
        g_opt = lambda name, default: override.get(name, getattr(prob, name, default))
        L = lib()
        keep = []

        def host(x, dt):
            if x is None:
                return None
            a = _host(x, dt)
            keep.append(a)
            return a

        img_s = np.ascontiguousarray(np.asarray(g("image_s")))
        img_t = np.ascontiguousarray(np.asarray(g("image_t")))
        if img_s.dtype == np.float16:
            dtype = F16
        else:
            img_s = img_s.astype(np.float32)
            img_t = img_t.astype(np.float32)
            dtype = F32
        img_t = img_t.astype(img_s.dtype)
        keep += [img_s, img_t]
        nz, ny, nx = img_s.shape
        tets = host(g("tets"), np.int32)
        ref = host(g("ref_points"), np.float32)
        lab = host(g("tet_label"), np.int32)
        tis = host(g("tissue_factor"), np.float64)
        gs = host(g("guid_s"), np.float32)
        gt = host(g("guid_t"), np.float32)
        gg = host(g("guid_group"), np.int32)
        n_guid = 0 if gs is None else int(gs.shape[0])
        if max_solutions is None:
            sol = override.get("sol_src", getattr(prob, "sol_src", None))
            max_solutions = int(sol.shape[0]) if sol is not None else 1
        ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        desc = ProblemDesc(
            nx=nx, ny=ny, nz=nz, dtype=dtype, image_s=ptr(img_s), image_t=ptr(img_t),
            n_points=int(ref.shape[0]), n_tets=int(tets.shape[0]), tets=ptr(tets), ref_points=ptr(ref),
            tet_label=ptr(lab), tissue_factor=ptr(tis), n_labels=0 if tis is None else int(tis.shape[0]),
            n_guid=n_guid, guid_s=ptr(gs), guid_t=ptr(gt), guid_group=ptr(gg),
            trunc_radius=float(g("trunc_radius")), h_mode=int(g("h_mode")), g_mode=int(g("g_mode")),
            subvoxel_bits=int(g("subvoxel_bits")), max_solutions=int(max_solutions),
            max_requests=int(max_requests), max_changed=int(max_changed),
            estimator=int(g_opt("estimator", 0)), sampling_rate=float(g_opt("sampling_rate", 1.0)),
            tissue_mask=ptr(host(g_opt("tissue_mask", None), np.uint8)))
        h = ctypes.c_void_p()
        _check(L.morea_create_problem(ctypes.byref(desc), _stream(stream), ctypes.byref(h)),
               "morea_create_problem")
        self._h = h
        self._L = L
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dtype = dtype
        nv, nt, ng, kb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        rr = ctypes.c_double()
        _check(L.morea_problem_info(h, ctypes.byref(nv), ctypes.byref(nt), ctypes.byref(ng), ctypes.byref(rr),
                                    ctypes.byref(kb)), "morea_problem_info")
        self.n_points, self.n_tets, self.n_groups = nv.value, nt.value, ng.value
        self.trunc_radius, self.subvoxel_bits = rr.value, kb.value
        self.max_solutions = int(max_solutions)
        self.max_requests = int(max_requests) if max_requests else int(max_solutions)
        self.max_changed = int(max_changed)
        self.h_mode, self.g_mode = int(g("h_mode")), int(g("g_mode"))
        self.estimator = int(g_opt("estimator", 0))

    # -- lifetime -----------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _check(self._L.morea_destroy_problem(h), "morea_destroy_problem")
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- evaluation ---------------------------------------------------------
    def eval_full(self, src: torch.Tensor, tgt: torch.Tensor, slots: Optional[torch.Tensor] = None,
                  out=None, stream=None):
        """Full evaluation; returns (obj [n,3] f64, folded [n] u8, severity [n] f64) on the device."""
        n = int(src.shape[0])
        V = self.n_points
        dev = src.device
        obj, folded, sev = out if out is not None else (
            torch.empty((n, 3), dtype=torch.float64, device=dev),
            torch.empty((n,), dtype=torch.uint8, device=dev),
            torch.empty((n,), dtype=torch.float64, device=dev))
        _check(self._L.morea_eval_full(
            self._h, n, _dev(slots, torch.int32, (n,), "slots"),
            _dev(src, torch.float32, (n, V, 3), "src"), _dev(tgt, torch.float32, (n, V, 3), "tgt"),
            _dev(obj, torch.float64, (n, 3), "obj"), _dev(folded, torch.uint8, (n,), "folded"),
            _dev(sev, torch.float64, (n,), "severity"), _stream(stream)), "morea_eval_full")
        return obj, folded, sev

    def eval_partial(self, slots: torch.Tensor, chg_off: torch.Tensor, chg_pts: torch.Tensor,
                     chg_src: torch.Tensor, chg_tgt: torch.Tensor, commit: Optional[torch.Tensor] = None,
                     out=None, stream=None):
        """Partial evaluation of ``len(slots)`` requests; returns (obj, folded, severity)."""
        n = int(slots.shape[0])
        c = int(chg_pts.shape[0])
        dev = slots.device
        obj, folded, sev = out if out is not None else (
            torch.empty((n, 3), dtype=torch.float64, device=dev),
            torch.empty((n,), dtype=torch.uint8, device=dev),
            torch.empty((n,), dtype=torch.float64, device=dev))
        _check(self._L.morea_eval_partial(
            self._h, n, _dev(slots, torch.int32, (n,), "slots"), _dev(chg_off, torch.int32, (n + 1,), "chg_off"),
            _dev(chg_pts, torch.int32, (c,), "chg_pts"), _dev(chg_src, torch.float32, (c, 3), "chg_src"),
            _dev(chg_tgt, torch.float32, (c, 3), "chg_tgt"), _dev(obj, torch.float64, (n, 3), "obj"),
            _dev(folded, torch.uint8, (n,), "folded"), _dev(sev, torch.float64, (n,), "severity"),
            _dev(commit, torch.uint8, (n,), "commit"), _stream(stream)), "morea_eval_partial")
        return obj, folded, sev

    def commit_partial(self, accept: torch.Tensor, stream=None):
        n = int(accept.shape[0])
        _check(self._L.morea_commit_partial(self._h, n, _dev(accept, torch.uint8, (n,), "accept"),
                                            _stream(stream)), "morea_commit_partial")

    def repair_folds(self, src: torch.Tensor, tgt: torch.Tensor, noise: torch.Tensor, max_points: int,
                     scale: float = 1.0, fixed: Optional[torch.Tensor] = None, stream=None):
        """Repair (Sec. 4.3.1) of src/tgt [n][V][3] in place; noise [n][max_points][64][3] N(0,1);
        fixed [V] uint8 axis bits of coordinates that stay.  Returns (moved [n] int32,
        severity [n] f64) on the device."""
        n = int(src.shape[0])
        V = self.n_points
        moved = torch.empty((n,), dtype=torch.int32, device=src.device)
        sev = torch.empty((n,), dtype=torch.float64, device=src.device)
        _check(self._L.morea_repair_folds(
            self._h, n, _dev(src, torch.float32, (n, V, 3), "src"), _dev(tgt, torch.float32, (n, V, 3), "tgt"),
            _dev(noise, torch.float32, (n, int(max_points), 64, 3), "noise"), int(max_points), float(scale),
            _dev(fixed, torch.uint8, (V,), "fixed"),
            _dev(moved, torch.int32, (n,), "moved"), _dev(sev, torch.float64, (n,), "severity"),
            _stream(stream)), "morea_repair_folds")
        return moved, sev

    def displacement(self, src: torch.Tensor, tgt: torch.Tensor, side: int = 0, labels_own=None,
                     labels_other=None, n_labels: int = 0, stream=None):
        """Displacement field [nz][ny][nx][3] of one solution (src, tgt [V][3]) on
        image ``side`` (NaN outside the mesh) and, with label images, the per-label
        counts [n_labels][3] (own, pulled back, both).  Device tensors."""
        V = self.n_points
        dev = src.device
        dvf = torch.empty((self.nz, self.ny, self.nx, 3), dtype=torch.float32, device=dev)
        counts = None
        lo = lt = None
        if labels_own is not None:
            counts = torch.empty((int(n_labels), 3), dtype=torch.int64, device=dev)
            lo = _dev(labels_own, torch.uint8, (self.nz, self.ny, self.nx), "labels_own")
            lt = _dev(labels_other, torch.uint8, (self.nz, self.ny, self.nx), "labels_other")
        _check(self._L.morea_displacement(
            self._h, _dev(src, torch.float32, (V, 3), "src"), _dev(tgt, torch.float32, (V, 3), "tgt"), int(side),
            _dev(dvf, torch.float32, None, "dvf"), lo, lt, int(n_labels),
            None if counts is None else _dev(counts, torch.int64, None, "overlap"), _stream(stream)),
            "morea_displacement")
        return dvf, counts

    def slot_objectives(self, n: int, slots: Optional[torch.Tensor] = None, stream=None):
        """(obj [n][3], folded [n], severity [n]) of committed slots (device)."""
        dev = torch.device("cuda")
        obj = torch.empty((n, 3), dtype=torch.float64, device=dev)
        folded = torch.empty((n,), dtype=torch.uint8, device=dev)
        sev = torch.empty((n,), dtype=torch.float64, device=dev)
        _check(self._L.morea_slot_objectives(
            self._h, int(n), _dev(slots, torch.int32, (n,), "slots"), _dev(obj, torch.float64, (n, 3), "obj"),
            _dev(folded, torch.uint8, (n,), "folded"), _dev(sev, torch.float64, (n,), "severity"), _stream(stream)),
            "morea_slot_objectives")
        return obj, folded, sev

    def sample_elements(self, src: torch.Tensor, tgt: torch.Tensor, members: torch.Tensor, elements: torch.Tensor,
                        cmult: torch.Tensor, req_sol: torch.Tensor, req_cluster: torch.Tensor,
                        req_element: torch.Tensor, z: torch.Tensor, fixed: Optional[torch.Tensor] = None,
                        work: Optional[torch.Tensor] = None, stream=None):
        """New coordinates (new_src, new_tgt [n_req*2][3]) of the two points of
        each requested FOS element, drawn from its cluster's distribution
        (Sec. 3).  src, tgt [n_pop][V][3]; members [k][c]; elements [m][2]."""
        n_pop, V = int(src.shape[0]), self.n_points
        k, c = (int(x) for x in members.shape)
        m = int(elements.shape[0])
        n_req = int(req_sol.shape[0])
        if work is None:
            work = torch.empty((sample_elements_workspace(k, m),), dtype=torch.uint8, device=src.device)
        new_s = torch.empty((2 * n_req, 3), dtype=torch.float32, device=src.device)
        new_t = torch.empty((2 * n_req, 3), dtype=torch.float32, device=src.device)
        _check(self._L.morea_sample_elements(
            self._h, n_pop, _dev(src, torch.float32, (n_pop, V, 3), "src"),
            _dev(tgt, torch.float32, (n_pop, V, 3), "tgt"), k, c, _dev(members, torch.int32, (k, c), "members"), m,
            _dev(elements, torch.int32, (m, 2), "elements"), _dev(fixed, torch.uint8, (V,), "fixed"),
            _dev(cmult, torch.float32, (k,), "cmult"), n_req, _dev(req_sol, torch.int32, (n_req,), "req_sol"),
            _dev(req_cluster, torch.int32, (n_req,), "req_cluster"),
            _dev(req_element, torch.int32, (n_req,), "req_element"), _dev(z, torch.float32, (n_req, 12), "z"),
            _dev(work, torch.uint8, None, "work"), ctypes.c_size_t(work.numel()),
            _dev(new_s, torch.float32, None, "new_src"), _dev(new_t, torch.float32, None, "new_tgt"),
            _stream(stream)), "morea_sample_elements")
        return new_s, new_t

    def init_noise(self, src: torch.Tensor, tgt: torch.Tensor, kernels: torch.Tensor, max_rounds: int,
                   fixed: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Gaussian-attraction initialisation noise (Sec. 4.2.2), in place on
        src, tgt [n][V][3]; kernels [n][2][K][5] = (cx, cy, cz, sigma, a);
        fixed [V] uint8 axis bits.  Returns the rounds kept, [n][2] int32."""
        n = int(src.shape[0])
        V = self.n_points
        K = int(kernels.shape[2])
        rounds = torch.empty((n, 2), dtype=torch.int32, device=src.device)
        _check(self._L.morea_init_noise(
            self._h, n, _dev(src, torch.float32, (n, V, 3), "src"), _dev(tgt, torch.float32, (n, V, 3), "tgt"),
            _dev(fixed, torch.uint8, (V,), "fixed"), K, _dev(kernels, torch.float32, (n, 2, K, 5), "kernels"),
            int(max_rounds), _dev(rounds, torch.int32, (n, 2), "rounds"), _stream(stream)), "morea_init_noise")
        return rounds

    def warp_labels(self, src: torch.Tensor, tgt: torch.Tensor, side: int, labels_other: torch.Tensor,
                    stream=None) -> torch.Tensor:
        """Warped label image [nz][ny][nx] uint8 of one solution on image
        ``side``: the other image's label at the voxel nearest to T(p);
        NO_LABEL where no copy covers p."""
        V = self.n_points
        warped = torch.empty((self.nz, self.ny, self.nx), dtype=torch.uint8, device=src.device)
        _check(self._L.morea_warp_labels(
            self._h, _dev(src, torch.float32, (V, 3), "src"), _dev(tgt, torch.float32, (V, 3), "tgt"), int(side),
            _dev(labels_other, torch.uint8, (self.nz, self.ny, self.nx), "labels_other"),
            _dev(warped, torch.uint8, None, "warped"), _stream(stream)), "morea_warp_labels")
        return warped

    def check_folds(self, src: torch.Tensor, tgt: torch.Tensor, stream=None):
        n = int(src.shape[0])
        V = self.n_points
        folded = torch.empty((n,), dtype=torch.uint8, device=src.device)
        sev = torch.empty((n,), dtype=torch.float64, device=src.device)
        _check(self._L.morea_check_folds(
            self._h, n, _dev(src, torch.float32, (n, V, 3), "src"), _dev(tgt, torch.float32, (n, V, 3), "tgt"),
            _dev(folded, torch.uint8, (n,), "folded"), _dev(sev, torch.float64, (n,), "severity"),
            _stream(stream)), "morea_check_folds")
        return folded, sev

    def read_records(self, n: int, slots: Optional[torch.Tensor] = None, stream=None) -> np.ndarray:
        """Per-(slot, tet) cached records as a numpy structured array [n][T]."""
        buf = torch.empty((n, self.n_tets, TET_RECORD_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        _check(self._L.morea_read_records(self._h, n, _dev(slots, torch.int32, (n,), "slots"),
                                          ctypes.c_void_p(buf.data_ptr()), _stream(stream)),
               "morea_read_records")
        return buf.cpu().numpy().view(TET_RECORD_DTYPE).reshape(n, self.n_tets)

    def read_totals(self, n: int, slots: Optional[torch.Tensor] = None, stream=None) -> np.ndarray:
        buf = torch.empty((n, TOTALS_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        _check(self._L.morea_read_totals(self._h, n, _dev(slots, torch.int32, (n,), "slots"),
                                         ctypes.c_void_p(buf.data_ptr()), _stream(stream)),
               "morea_read_totals")
        return buf.cpu().numpy().view(TOTALS_DTYPE).reshape(n)

    def device_status(self, stream=None) -> int:
        bits = ctypes.c_uint32(0)
        rc = self._L.morea_device_status(self._h, _stream(stream), ctypes.byref(bits))
        if rc not in (OK, EDEVICE):
            _check(rc, "morea_device_status")
        return int(bits.value)

    def partial_features(self, slots: torch.Tensor, chg_off: torch.Tensor, chg_pts: torch.Tensor,
                         chg_src: torch.Tensor, chg_tgt: torch.Tensor, out: Optional[torch.Tensor] = None,
                         stream=None) -> torch.Tensor:
        """Displacement features [n][V*3] of the candidates of a partial-request list."""
        n = int(slots.shape[0])
        c = int(chg_pts.shape[0])
        if out is None:
            out = torch.empty((n, self.n_points * 3), dtype=torch.float32, device=slots.device)
        _check(self._L.morea_partial_features(
            self._h, n, _dev(slots, torch.int32, (n,), "slots"), _dev(chg_off, torch.int32, (n + 1,), "chg_off"),
            _dev(chg_pts, torch.int32, (c,), "chg_pts"), _dev(chg_src, torch.float32, (c, 3), "chg_src"),
            _dev(chg_tgt, torch.float32, (c, 3), "chg_tgt"), _dev(out, torch.float32, (n, self.n_points * 3), "out"),
            _stream(stream)), "morea_partial_features")
        return out

    def set_launch(self, blocks_per_sm: int, chunk: int):
        """Launch shape of the image/guidance passes (see morea_set_launch)."""
        _check(self._L.morea_set_launch(self._h, int(blocks_per_sm), int(chunk)), "morea_set_launch")

    # -- instrumentation ----------------------------------------------------
    def profile(self, flags: int):
        """bit 0: time every launch of the hot kernel with CUDA events; bit 1: count voxel visits."""
        _check(self._L.morea_profile(self._h, int(flags)), "morea_profile")

    def profile_read(self):
        ms, n, v = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check(self._L.morea_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(v)),
               "morea_profile_read")
        return ms.value, n.value, v.value


class Batch:
    """Several problems evaluated with one launch per kernel (morea_batch_*).

    ``problems`` are :class:`Problem` objects with the same storage type and
    modes; they must stay open while the batch lives.
    """

    def __init__(self, problems: Sequence[Problem]):
        self.problems = list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[p.handle.value for p in self.problems])
        h = ctypes.c_void_p()
        _check(lib().morea_batch_create(arr, len(self.problems), ctypes.byref(h)), "morea_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().morea_batch_destroy(self._h), "morea_batch_destroy")
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _args(self, srcs, tgts, outs):
        n = len(self.problems)
        if len(srcs) != n or len(tgts) != n or len(outs) != n:
            raise ValueError("one (src, tgt, out) per problem")
        n_sol = (ctypes.c_int32 * n)(*[int(x.shape[0]) for x in srcs])
        ptrs = lambda ts, dt, shp: (ctypes.c_void_p * n)(*[_dev(t, dt, shp(i), "batch tensor").value
                                                        for i, t in enumerate(ts)])
        V = [p.n_points for p in self.problems]
        src_p = ptrs(srcs, torch.float32, lambda i: (n_sol[i], V[i], 3))
        tgt_p = ptrs(tgts, torch.float32, lambda i: (n_sol[i], V[i], 3))
        obj_p = ptrs([o[0] for o in outs], torch.float64, lambda i: (n_sol[i], 3))
        fol_p = ptrs([o[1] for o in outs], torch.uint8, lambda i: (n_sol[i],))
        sev_p = ptrs([o[2] for o in outs], torch.float64, lambda i: (n_sol[i],))
        self._keep = (n_sol, src_p, tgt_p, obj_p, fol_p, sev_p)
        return n_sol, src_p, tgt_p, obj_p, fol_p, sev_p

    @staticmethod
    def outputs(srcs):
        return [(torch.empty((int(s.shape[0]), 3), dtype=torch.float64, device=s.device),
                 torch.empty(int(s.shape[0]), dtype=torch.uint8, device=s.device),
                 torch.empty(int(s.shape[0]), dtype=torch.float64, device=s.device)) for s in srcs]

    def eval_full(self, srcs, tgts, outs=None, stream=None):
        outs = outs if outs is not None else self.outputs(srcs)
        _check(lib().morea_batch_eval_full(self._h, *self._args(srcs, tgts, outs), _stream(stream)),
               "morea_batch_eval_full")
        return outs

    def capture(self, srcs, tgts, outs, stream):
        """Record one batched evaluation of these (fixed) buffers into a CUDA graph."""
        _check(lib().morea_batch_capture(self._h, *self._args(srcs, tgts, outs), _stream(stream)),
               "morea_batch_capture")

    def replay(self, stream=None):
        _check(lib().morea_batch_replay(self._h, _stream(stream)), "morea_batch_replay")

    def latency(self):
        """Per-problem completion of the last evaluation, ms after it started:
        (records complete, objectives written), as numpy arrays (-1: not
        complete).  Synchronises the device."""
        n = len(self.problems)
        rec, obj = (ctypes.c_double * n)(), (ctypes.c_double * n)()
        _check(lib().morea_batch_latency(self._h, rec, obj), "morea_batch_latency")
        return np.array(rec[:]), np.array(obj[:])

    def set_launch(self, blocks_per_sm: int, chunk: int):
        _check(lib().morea_batch_set_launch(self._h, int(blocks_per_sm), int(chunk)), "morea_batch_set_launch")


class Mlp:
    """The surrogate network n_in -> h1 -> h2 -> n_out (morea_mlp_*)."""

    def __init__(self, n_in: int, h1: int = 512, h2: int = 256, n_out: int = 3, max_batch: int = 1024,
                 seed: Optional[int] = 0):
        self.n_in, self.h1, self.h2, self.n_out, self.max_batch = n_in, h1, h2, n_out, max_batch
        h = ctypes.c_void_p()
        _check(lib().morea_mlp_create(n_in, h1, h2, n_out, max_batch, ctypes.byref(h)), "morea_mlp_create")
        self._h = h
        npar, kin = ctypes.c_int64(), ctypes.c_int32()
        _check(lib().morea_mlp_info(h, ctypes.byref(npar), ctypes.byref(kin)), "morea_mlp_info")
        self.n_params, self.kin = npar.value, kin.value
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        if seed is not None:
            self.set_params(self.init_params(seed))

    def init_params(self, seed: int) -> np.ndarray:
        """He-uniform weights, zero biases, in the library's parameter layout."""
        rng = np.random.default_rng(seed)
        def he(rows, cols):
            b = np.sqrt(6.0 / cols)
            return rng.uniform(-b, b, size=(rows, cols))
        W1 = np.zeros((self.h1, self.kin))
        W1[:, :self.n_in] = he(self.h1, self.n_in)
        parts = [W1.ravel(), np.zeros(self.h1), he(self.h2, self.h1).ravel(), np.zeros(self.h2),
                 he(self.n_out, self.h2).ravel(), np.zeros(self.n_out)]
        return np.concatenate(parts).astype(np.float32)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().morea_mlp_destroy(self._h), "morea_mlp_destroy")
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self) -> int:
        """Read and clear the network's device status bits (0: all waits completed)."""
        bits = ctypes.c_uint32()
        _check(lib().morea_mlp_device_status(self._h, ctypes.byref(bits), _stream(None)), "morea_mlp_device_status")
        return bits.value

    def set_params(self, params):
        if isinstance(params, torch.Tensor):
            t = params.to(torch.float32).contiguous()
            _check(lib().morea_mlp_set_params(self._h, ctypes.c_void_p(t.data_ptr()), _stream(None)),
                   "morea_mlp_set_params")
            torch.cuda.current_stream().synchronize()
            return
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check(lib().morea_mlp_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p), _stream(None)),
               "morea_mlp_set_params")
        torch.cuda.current_stream().synchronize()

    def get_params(self) -> np.ndarray:
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(lib().morea_mlp_get_params(self._h, ctypes.c_void_p(out.data_ptr()), _stream(None)),
               "morea_mlp_get_params")
        return out.cpu().numpy()

    def forward(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Predictions for x [n][n_in] (n may exceed max_batch; processed in chunks)."""
        n = int(x.shape[0])
        if out is None:
            out = torch.empty((n, self.n_out), dtype=torch.float32, device=x.device)
        _dev(x, torch.float32, (n, self.n_in), "x")
        for a in range(0, n, self.max_batch):
            b = min(n, a + self.max_batch)
            _check(lib().morea_mlp_forward(self._h, b - a, ctypes.c_void_p(x[a:b].data_ptr()),
                                           ctypes.c_void_p(out[a:b].data_ptr()), _stream(stream)),
                   "morea_mlp_forward")
        return out

    def gradients(self, x: torch.Tensor, t: torch.Tensor, stream=None):
        n = int(x.shape[0])
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        _check(lib().morea_mlp_gradients(self._h, n, _dev(x, torch.float32, (n, self.n_in), "x"),
                                         _dev(t, torch.float32, (n, self.n_out), "t"), ctypes.c_void_p(g.data_ptr()),
                                         ctypes.c_void_p(self._loss.data_ptr()), _stream(stream)),
               "morea_mlp_gradients")
        return g, self._loss

    def train_step(self, x: torch.Tensor, t: torch.Tensor, lr: float, stream=None) -> torch.Tensor:
        n = int(x.shape[0])
        _check(lib().morea_mlp_train_step(self._h, n, _dev(x, torch.float32, (n, self.n_in), "x"),
                                          _dev(t, torch.float32, (n, self.n_out), "t"), float(lr),
                                          ctypes.c_void_p(self._loss.data_ptr()), _stream(stream)),
               "morea_mlp_train_step")
        return self._loss


def fold_magnitude_noalloc(tets: torch.Tensor, ref_points: torch.Tensor, cdelta: torch.Tensor, shape_xyz,
                           subvoxel_bits: int, src: torch.Tensor, tgt: torch.Tensor, out=None, stream=None):
    """Fold constraint and f_magnitude without a problem handle and without
    any allocation inside the library (for callers that cannot allocate
    device memory; see morea_fold_magnitude_noalloc in include/morea.h).
    ``out`` = (f_mag [n] f64, folded [n] u8, severity [n] f64), preallocated
    by the caller; when omitted this wrapper allocates them with torch."""
    n, V = int(src.shape[0]), int(src.shape[1])
    T = int(tets.shape[0])
    if out is None:
        out = (torch.empty(n, dtype=torch.float64, device=src.device),
               torch.empty(n, dtype=torch.uint8, device=src.device),
               torch.empty(n, dtype=torch.float64, device=src.device))
    f_mag, folded, sev = out
    nx, ny, nz = shape_xyz
    _check(lib().morea_fold_magnitude_noalloc(
        n, V, T, _dev(tets, torch.int32, (T, 4), "tets"), _dev(ref_points, torch.float32, (V, 3), "ref_points"),
        _dev(cdelta, torch.float32, (T,), "cdelta"), int(nx), int(ny), int(nz), int(subvoxel_bits),
        _dev(src, torch.float32, (n, V, 3), "src"), _dev(tgt, torch.float32, (n, V, 3), "tgt"),
        _dev(f_mag, torch.float64, (n,), "f_mag"), _dev(folded, torch.uint8, (n,), "folded"),
        _dev(sev, torch.float64, (n,), "severity"), _stream(stream)), "morea_fold_magnitude_noalloc")
    return f_mag, folded, sev


def requests_to_device(rd, device="cuda"):
    """Move one round of partial requests (numpy dict) to device tensors."""
    return {k: torch.as_tensor(np.ascontiguousarray(v)).to(device) for k, v in rd.items()}
