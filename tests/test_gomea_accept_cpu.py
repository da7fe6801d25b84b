"""The generation driver's vectorised acceptance (Sec. 3: unfolded, and
either dominating the parent or not weakly dominated by the elitist
archive; Sec. 4.3.2: f_guidance within the steering bound) equals the rule
applied candidate by candidate with the scalar helpers."""

import numpy as np

from paper_2303_04873_gb300 import gomea
from paper_2303_04873_gb300.ea import Archive, dominates


def stub(archive_pts, obj):
    g = gomea.Gomea.__new__(gomea.Gomea)        # host logic only: no problem, no GPU
    g.archive = Archive(2000)
    for o in archive_pts:
        g.archive.add(o)
    g.obj = obj
    return g


def test_vectorised_acceptance_equals_the_rule():
    rng = np.random.default_rng(0)
    for trial in range(20):
        obj = rng.integers(0, 6, size=(12, 3)).astype(float)
        arch = rng.integers(0, 6, size=(25, 3)).astype(float)
        g = stub(arch, obj)
        n = 200
        o = rng.integers(0, 6, size=(n, 3)).astype(float)
        o[rng.random(n) < 0.05] = np.nan
        f = rng.random(n) < 0.2
        sol = rng.integers(0, 12, n)
        hi = np.inf if trial % 2 else 3.5
        got = g._accept(o, f, sol, hi)
        for r in range(n):
            ok = (not f[r]) and np.all(np.isfinite(o[r])) and o[r, 2] <= hi
            want = ok and (dominates(o[r], obj[sol[r]]) or g.archive.accepts(o[r]))
            assert got[r] == want, (trial, r)


def test_archive_check_in_chunks():
    rng = np.random.default_rng(1)
    arch = rng.random((300, 3))
    g = stub(arch, np.zeros((1, 3)))
    o = rng.random((5000, 3))
    got = g._archive_accepts(o, chunk=777)
    want = np.array([g.archive.accepts(x) for x in o])
    np.testing.assert_array_equal(got, want)
