"""Pins of the oracle's branch decomposition (CPU only).

By the elder rule (Section 2.1) a point of the merge tree at height f(u),
the component C of u in {w : w <= u}, lies on the branch of C's deepest
vertex: a vertex that is itself the deepest of its component is a minimum
heading its own branch. These tests compute that assignment by breadth-first
search over sublevel sets (brute.py, no sweep, no union-find) and check the
grouping against Python's own tuple sort."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from brute import _component, _neighbours


def _brute_branch(f):
    nz, ny, nx = f.shape
    flat = [float(x) for x in f.ravel()]
    order = sorted(range(f.size), key=lambda i: (flat[i], i))
    rank = [0] * f.size
    for r, i in enumerate(order):
        rank[i] = r
    nb = _neighbours(nx, ny, nz)
    out = np.empty(f.size, dtype=np.uint32)
    for u in range(f.size):
        comp = _component(nb, rank, u, rank[u])
        out[u] = min(comp, key=lambda w: rank[w])
    return out


@pytest.mark.parametrize("ties", [False, True])
def test_branch_of_is_the_deepest_vertex_below(ties):
    rng = np.random.default_rng(31 + ties)
    for _ in range(120):
        shape = tuple(int(x) for x in rng.integers(1, 6, size=3))
        f = (rng.integers(0, 5, size=shape).astype(np.float32) if ties else rng.random(shape, dtype=np.float32))
        W = oracle.merge_tree(f)
        assert np.array_equal(oracle.branch_of(W), _brute_branch(f))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_grouping_by_tuple_sort(seed):
    rng = np.random.default_rng(seed)
    f = rng.integers(0, 9, size=(6, 7, 9)).astype(np.float32)
    W = oracle.merge_tree(f)
    order, offsets = oracle.branches(f, W)
    b = oracle.branch_of(W)
    flat = [float(x) for x in f.ravel()]
    # reference grouping by Python's tuple sort
    ref = sorted(range(f.size), key=lambda i: (int(b[i]), flat[i], i))
    assert [int(x) for x in order] == ref
    p, roots = oracle.pairs(W)
    assert len(offsets) - 1 == len(p) + len(roots)  # one branch per minimum
    for i in range(len(offsets) - 1):
        grp = order[offsets[i]:offsets[i + 1]]
        assert grp[0] == b[grp[0]]  # starts with its minimum
        assert np.all(b[grp] == grp[0])
