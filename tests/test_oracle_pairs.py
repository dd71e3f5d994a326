"""Pins of the oracle's fixed-radius neighbour search (Sec. 3: every pair
with ||x_i - x_j|| <= psi, found with a K-D tree).  Brute force is pinned to
lattices whose neighbour sets are known by construction; the K-D tree is
pinned to brute force."""
import itertools

import numpy as np
import pytest

import oracle as O


def _lattice(dim, m, spacing=1.0):
    axes = [np.arange(m, dtype=np.float64) * spacing] * dim
    grid = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in grid])


def _expected_lattice_pairs(pos, offsets):
    dim, n = pos.shape
    index = {tuple(pos[:, i]): i for i in range(n)}
    out = set()
    for i in range(n):
        for off in offsets:
            q = tuple(pos[:, i] + np.array(off, dtype=np.float64))
            if q in index:
                out.add((i, index[q]))
    return out


@pytest.mark.parametrize("method", ["brute", "kdtree"])
@pytest.mark.parametrize("dim,psi2,shells", [
    (1, 1.0, 1), (1, 0.99, 0), (1, 4.0, 2),
    (2, 1.0, 1), (2, 2.0, 2), (2, 0.999, 0),
    (3, 1.0, 1), (3, 2.0, 2), (3, 3.0, 3),
])
def test_lattice_neighbour_sets(method, dim, psi2, shells):
    pos = _lattice(dim, 6 if dim > 1 else 12)
    # offsets with integer squared length <= psi2 (exact: integer coordinates)
    rng = range(-2, 3)
    offsets = [o for o in itertools.product(rng, repeat=dim)
               if 0 < sum(c * c for c in o) <= psi2]
    i, j = O.pairs(pos, psi2, method)
    got = set(zip(i.tolist(), j.tolist()))
    assert got == _expected_lattice_pairs(pos, offsets)
    if shells == 0:
        assert len(got) == 0


@pytest.mark.parametrize("method", ["brute", "kdtree"])
def test_cutoff_is_inclusive_on_exact_ties(method):
    # 0.75^2 + 1^2 = 1.5625 = 1.25^2 exactly in binary64
    pos = np.array([[0.0, 0.75, 10.0], [0.0, 1.0, 10.0]])
    i, j = O.pairs(pos, 1.5625, method)
    assert set(zip(i.tolist(), j.tolist())) == {(0, 1), (1, 0)}
    i, j = O.pairs(pos, np.nextafter(1.5625, 0.0), method)
    assert len(i) == 0


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kdtree_equals_brute_force(dim):
    rng = np.random.default_rng(dim)
    n = 1500
    L = {1: 300.0, 2: 40.0, 3: 12.0}[dim]
    pos = rng.uniform(0, L, size=(dim, n))
    pos[:, :50] = np.round(pos[:, :50])          # exact grid points and duplicates
    pos[:, 50:60] = pos[:, 60:70]                 # coincident particles
    pos[0, 70:80] = 0.0                           # on the wall
    for psi2 in (1.8, 0.25, 4.0):
        bi, bj = O.pairs(pos, psi2, "brute")
        ki, kj = O.pairs(pos, psi2, "kdtree")
        assert np.array_equal(bi, ki) and np.array_equal(bj, kj)
        # the relation is symmetric and irreflexive
        s = set(zip(bi.tolist(), bj.tolist()))
        assert all((b, a) in s for a, b in s)
        assert all(a != b for a, b in s)


def test_empty_and_single():
    i, j = O.pairs(np.zeros((2, 0)), 1.0, "kdtree")
    assert i.size == 0
    i, j = O.pairs(np.zeros((2, 1)), 1.0, "kdtree")
    assert i.size == 0
