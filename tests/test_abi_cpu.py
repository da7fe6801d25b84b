"""CPU-only checks of the C ABI: the library builds and loads, exports every
entry point that include/morea.h declares, the binding's struct layouts match
the header (checked by compiling the header with the host C compiler), and
invalid problem descriptions are rejected on the host with MOREA_EINVAL
before any CUDA call."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "morea.h")


@pytest.fixture(scope="module")
def built():
    from paper_2303_04873_gb300 import build
    return build.build()


@pytest.fixture(scope="module")
def mo(built):
    from paper_2303_04873_gb300 import morea
    return morea


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(morea_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_entry_points(mo):
    assert declared_functions() == sorted(mo.ENTRY_POINTS)


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (morea_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    L = ctypes.CDLL(built)
    for f in declared_functions():
        assert getattr(L, f) is not None


def test_struct_layouts_match_header(mo, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "morea.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("desc %zu rec %zu tot %zu\n", sizeof(morea_problem_desc), sizeof(morea_tet_record), sizeof(morea_totals));
  P(morea_problem_desc, image_s) P(morea_problem_desc, n_points) P(morea_problem_desc, tets)
  P(morea_problem_desc, n_labels) P(morea_problem_desc, guid_s) P(morea_problem_desc, trunc_radius)
  P(morea_problem_desc, h_mode) P(morea_problem_desc, max_changed)
  P(morea_problem_desc, estimator) P(morea_problem_desc, sampling_rate) P(morea_problem_desc, tissue_mask)
  P(morea_tet_record, n_vox) P(morea_tet_record, e_mag) P(morea_tet_record, sev)
  P(morea_totals, n_vox) P(morea_totals, sev)
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = dict(zip(["desc", "rec", "tot"], map(int, out[0].split()[1::2])))
    assert sizes["desc"] == ctypes.sizeof(mo.ProblemDesc)
    assert sizes["rec"] == mo.TET_RECORD_DTYPE.itemsize
    assert sizes["tot"] == mo.TOTALS_DTYPE.itemsize
    offs = {line.split()[0]: int(line.split()[1]) for line in out[1:] if line.strip()}
    for key, off in offs.items():
        struct, field = key.split(".")
        if struct == "morea_problem_desc":
            assert getattr(mo.ProblemDesc, field).offset == off, key
        elif struct == "morea_tet_record":
            assert mo.TET_RECORD_DTYPE.fields[field][1] == off, key
        else:
            assert mo.TOTALS_DTYPE.fields[field][1] == off, key


def _desc(mo, **kw):
    import synth
    p = synth.make_c0(n_sol=1)
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p)

    d = dict(nx=32, ny=32, nz=32, dtype=0, image_s=arr(p.image_s, np.float32), image_t=arr(p.image_t, np.float32),
             n_points=p.n_points, n_tets=p.n_tets, tets=arr(p.tets, np.int32), ref_points=arr(p.ref_points, np.float32),
             tet_label=arr(p.tet_label, np.int32), tissue_factor=arr(p.tissue_factor, np.float64), n_labels=4,
             n_guid=len(p.guid_s), guid_s=arr(p.guid_s, np.float32), guid_t=arr(p.guid_t, np.float32),
             guid_group=arr(p.guid_group, np.int32), trunc_radius=0.8, h_mode=0, g_mode=0, subvoxel_bits=8,
             max_solutions=8, max_requests=0, max_changed=64)
    d.update(kw)
    return mo.ProblemDesc(**d), keep


@pytest.mark.parametrize("bad", [
    dict(nx=1), dict(dtype=7), dict(n_points=3), dict(h_mode=5), dict(g_mode=9), dict(subvoxel_bits=12),
    dict(subvoxel_bits=1), dict(max_solutions=0), dict(max_changed=5000), dict(n_labels=0),
    dict(trunc_radius=float("nan")), dict(image_s=None),
    dict(estimator=2), dict(estimator=1, h_mode=1), dict(estimator=1, g_mode=1),
    dict(estimator=1, sampling_rate=float("nan")), dict(estimator=1, sampling_rate=1e9),
])
def test_invalid_descriptions_rejected_on_host(mo, bad):
    d, keep = _desc(mo, **bad)
    h = ctypes.c_void_p(123)
    rc = mo.lib().morea_create_problem(ctypes.byref(d), None, ctypes.byref(h))
    assert rc == mo.EINVAL
    assert not h.value


def test_tissue_mask_checked_on_host(mo):
    """A tissue mask needs tissue factors, at most 64 labels and every voxel
    label below n_labels; each violation is rejected before any device work."""
    bad_label = np.zeros((32, 32, 32), np.uint8)
    bad_label[3, 4, 5] = 4                     # n_labels is 4
    ok = np.zeros((32, 32, 32), np.uint8)
    for mask, kw in ((bad_label, {}), (ok, dict(tissue_factor=None)), (ok, dict(n_labels=65))):
        d, keep = _desc(mo, tissue_mask=mask.ctypes.data_as(ctypes.c_void_p), **kw)
        h = ctypes.c_void_p(123)
        assert mo.lib().morea_create_problem(ctypes.byref(d), None, ctypes.byref(h)) == mo.EINVAL
        assert not h.value


def test_degenerate_or_out_of_range_topology_rejected(mo):
    for tets in (np.array([[0, 1, 2, 2]], np.int32), np.array([[0, 1, 2, 999]], np.int32)):
        keep_t = np.ascontiguousarray(tets)
        d, keep = _desc(mo, n_tets=1, tets=keep_t.ctypes.data_as(ctypes.c_void_p),
                        tet_label=None, tissue_factor=None, n_labels=0)
        h = ctypes.c_void_p()
        assert mo.lib().morea_create_problem(ctypes.byref(d), None, ctypes.byref(h)) == mo.EINVAL


def test_bad_label_and_group_rejected(mo):
    lab = np.full(384, 9, np.int32)
    d, keep = _desc(mo, tet_label=lab.ctypes.data_as(ctypes.c_void_p))
    h = ctypes.c_void_p()
    assert mo.lib().morea_create_problem(ctypes.byref(d), None, ctypes.byref(h)) == mo.EINVAL
    grp = np.full(100, 8, np.int32)
    d, keep = _desc(mo, guid_group=grp.ctypes.data_as(ctypes.c_void_p))
    assert mo.lib().morea_create_problem(ctypes.byref(d), None, ctypes.byref(h)) == mo.EINVAL


def test_null_handles_and_status_strings(mo):
    L = mo.lib()
    assert L.morea_destroy_problem(None) == mo.OK
    assert L.morea_eval_full(None, 1, None, None, None, None, None, None, None) == mo.EINVAL
    assert L.morea_eval_partial(None, 1, *([None] * 10)) == mo.EINVAL
    assert L.morea_commit_partial(None, 1, None, None) == mo.EINVAL
    assert L.morea_check_folds(None, 1, None, None, None, None, None) == mo.EINVAL
    assert L.morea_device_status(None, None, None) == mo.EINVAL
    for code in range(7):
        assert mo.status_string(code) != "unknown status"
    assert mo.status_string(99) == "unknown status"


def test_surface_distance_arguments_checked_on_host(mo):
    L = mo.lib()
    need = mo.surface_distance_workspace(128, 128, 96)
    N = 128 * 128 * 96
    bins = 127 ** 2 + 127 ** 2 + 95 ** 2 + 1
    assert need >= N + 16 * N + 8 * bins
    assert need % 256 == 0
    assert L.morea_surface_distance_workspace(0, 4, 4) == 0
    assert L.morea_surface_distance_workspace(1025, 4, 4) == 0
    assert L.morea_surface_distance_workspace(1, 1, 1) > 0
    fake = ctypes.c_void_p(256)        # never dereferenced: every call below fails its host checks
    ok = (8, 8, 8, fake, fake, 1, fake, mo.surface_distance_workspace(8, 8, 8), fake, None)
    for i, bad in ((0, 0), (1, 2000), (3, None), (4, None), (5, -1), (5, 256), (6, None), (8, None)):
        args = list(ok)
        args[i] = bad
        assert L.morea_surface_distance(*args) == mo.EINVAL
    args = list(ok)
    args[7] = ok[7] - 1                # workspace one byte short
    assert L.morea_surface_distance(*args) == mo.EINVAL
    args = list(ok)
    args[6] = ctypes.c_void_p(256 + 16)   # workspace not 256-byte aligned
    assert L.morea_surface_distance(*args) == mo.EINVAL
    assert L.morea_warp_labels(None, fake, fake, 0, fake, fake, None) == mo.EINVAL


def test_noalloc_grid_checked_on_host(mo):
    """morea_fold_magnitude_noalloc applies problem creation's grid bounds
    before touching the GPU: an explicit k whose exact 64-bit severity sum
    could overflow (4 T N 8^k >= 2^63) or whose box exceeds 2^16 snapped
    units is rejected."""
    L = mo.lib()
    fake = ctypes.c_void_p(256)        # never dereferenced: the host checks fail first
    T = mo.NOALLOC_MAX_TET_EVALS

    def call(n_tets, box, k):
        return L.morea_fold_magnitude_noalloc(1, 4, n_tets, fake, fake, fake, *box, k, fake, fake, fake, fake,
                                              None, None)

    assert call(T, (256, 256, 160), 8) == mo.EINVAL          # 4 T N 8^8 ~ 2^68
    assert call(16, (512, 8, 8), 8) == mo.EINVAL             # 512 * 2^8 > 2^16
    assert call(16, (8, 8, 8), 15) == mo.EINVAL
    assert call(T + 1, (8, 8, 8), 0) == mo.EINVAL            # beyond the scratch
