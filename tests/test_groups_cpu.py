"""The library's linkage model and parallel groups (a host call, no GPU)
against the oracle's plain restatement (reading R16): identical elements
and group ids on the benchmark meshes and on random lattices."""

import numpy as np
import pytest

import synth
from oracle import fos


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


@pytest.mark.parametrize("make", [synth.make_c0, synth.make_c1])
def test_groups_equal_the_oracle_on_benchmark_meshes(mo, make):
    p = make(n_sol=1)
    el, grp = mo.parallel_groups(p.n_points, p.tets)
    want_el, want_grp = fos.parallel_groups(p.n_points, p.tets)
    np.testing.assert_array_equal(el, want_el)
    np.testing.assert_array_equal(grp, want_grp)


@pytest.mark.parametrize("seed", range(6))
def test_groups_equal_the_oracle_on_random_lattices(mo, seed):
    rng = np.random.default_rng(seed)
    dims = [int(v) for v in rng.integers(2, 6, size=3)]
    tets = synth.kuhn_lattice(*dims, flip_x=bool(seed % 2))
    n_points = int(np.prod(dims))
    perm = rng.permutation(n_points).astype(np.int32)       # relabel the points
    tets = perm[tets]
    el, grp = mo.parallel_groups(n_points, tets)
    want_el, want_grp = fos.parallel_groups(n_points, tets)
    np.testing.assert_array_equal(el, want_el)
    np.testing.assert_array_equal(grp, want_grp)


def test_bad_topology_is_rejected(mo):
    with pytest.raises(mo.MoreaError):
        mo.parallel_groups(4, np.array([[0, 1, 2, 9]], np.int32))
    with pytest.raises(mo.MoreaError):
        mo.parallel_groups(6, np.array([[0, 1, 2, 3]], np.int32))    # points 4, 5 in no tet
