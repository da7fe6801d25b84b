"""The library's host selection and clustering (morea_cluster, reading R19)
equals the oracle exactly: selected indices, cluster members and the
cluster of every population member, on random objective sets with ties,
duplicates and degenerate ranges."""

import numpy as np
import pytest

from oracle import gomea as gm


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def check(mo, obj, tau, k, iters=10):
    sel, mem, pc = mo.cluster(obj, tau, k, iters)
    wsel, wmem, wpc = gm.clusters(obj, tau, k, iters)
    np.testing.assert_array_equal(sel, wsel)
    np.testing.assert_array_equal(mem, np.array(wmem, np.int32))
    np.testing.assert_array_equal(pc, wpc)


@pytest.mark.parametrize("seed", range(6))
def test_random_populations(mo, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 120))
    obj = rng.random((n, 3)) * [3.0, 0.1, 50.0]
    check(mo, obj, 0.35, int(rng.integers(1, 12)))


def test_ties_duplicates_and_flat_objectives(mo):
    rng = np.random.default_rng(9)
    obj = rng.integers(0, 4, size=(60, 3)).astype(float)
    obj[:, 1] = 2.0                                       # a zero range
    obj[10:20] = obj[0]                                   # duplicates
    for k in (1, 3, 10, 40):
        check(mo, obj, 0.35, k)
    check(mo, obj, 1.0, 7, iters=1)


def test_more_clusters_than_selected(mo):
    obj = np.random.default_rng(3).random((8, 3))
    check(mo, obj, 0.35, 10)


def test_rejections(mo):
    obj = np.random.default_rng(0).random((5, 3))
    for tau, k, it in ((0.0, 2, 5), (1.5, 2, 5), (0.5, 0, 5), (0.5, 2, 0)):
        with pytest.raises(mo.MoreaError):
            mo.cluster(obj, tau, k, it)
    bad = obj.copy()
    bad[2, 1] = np.nan
    with pytest.raises(mo.MoreaError):
        mo.cluster(bad, 0.5, 2)
