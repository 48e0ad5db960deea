"""Pins of the oracle's persistence simplification (CPU only).

The reading under test: simplifying by eps fills every branch whose
persistence f(s) - f(u) (float32) is below eps up to its saddle s -- every
vertex of the branch's pit, u's component of {w : w < s}, is raised to f(s).
These tests build that filled field explicitly from the brute-force tree of
``brute.py`` (breadth-first searches over sublevel sets, no sort-sweep and no
union-find) and check the oracle against it:
  * G_t of the filled field is exactly the set the oracle keeps, split into
    the same components, each labelled with its deepest vertex of f;
  * the filled field's own diagram, without its zero-persistence pairs, is
    the oracle's simplified diagram (distinct values, where saddles are
    unambiguous).
"""

from __future__ import annotations

from collections import deque

import numpy as np
import pytest

import oracle
from brute import _component, _neighbours, brute_merge_tree

FFFF = np.uint32(0xFFFFFFFF)


def _rank(flat):
    order = sorted(range(len(flat)), key=lambda i: (flat[i], i))
    rank = [0] * len(flat)
    for r, i in enumerate(order):
        rank[i] = r
    return rank


def _filled(f: np.ndarray, W: np.ndarray, eps: float) -> np.ndarray:
    """The field with every branch of persistence < eps filled up to its saddle."""
    nz, ny, nx = f.shape
    flat = [float(x) for x in f.ravel()]
    rank = _rank(flat)
    nb = _neighbours(nx, ny, nz)
    g = f.ravel().copy()
    for u in range(f.size):
        s = int(W[u] >> np.uint64(32))
        if s == u:
            continue
        if np.float32(f.ravel()[s]) - np.float32(f.ravel()[u]) >= np.float32(eps):
            continue
        for w in _component(nb, rank, u, rank[s] - 1):
            g[w] = max(g[w], f.ravel()[s])
    return g.reshape(f.shape)


def _components_bfs(mask: np.ndarray, nb):
    """Component id per vertex of the mask (-1 outside), by breadth-first search."""
    comp = np.full(mask.size, -1, dtype=np.int64)
    c = 0
    for u in range(mask.size):
        if not mask[u] or comp[u] >= 0:
            continue
        comp[u] = c
        q = deque([u])
        while q:
            x = q.popleft()
            for w in nb[x]:
                if mask[w] and comp[w] < 0:
                    comp[w] = c
                    q.append(w)
        c += 1
    return comp


def _cases(count, seed, ties):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        shape = tuple(int(x) for x in rng.integers(1, 6, size=3))
        if ties:
            f = rng.integers(0, 6, size=shape).astype(np.float32)
        else:
            f = rng.random(shape, dtype=np.float32)
        lo, hi = float(f.min()), float(f.max())
        t = np.float32(rng.uniform(lo, hi))
        eps = np.float32(rng.uniform(0.0, (hi - lo) * 0.8 + 1e-3))
        yield f, float(t), float(eps)


@pytest.mark.parametrize("ties", [False, True])
def test_simplified_labels_equal_filled_field(ties):
    checked = 0
    for f, t, eps in _cases(150, 11 + ties, ties):
        W = oracle.merge_tree(f)
        assert np.array_equal(W, brute_merge_tree(f))
        g = _filled(f, brute_merge_tree(f), eps)
        lab = oracle.simplified_components(f, W, t, eps)
        nz, ny, nx = f.shape
        nb = _neighbours(nx, ny, nz)
        keep = (g.ravel() <= np.float32(t))
        assert np.array_equal(lab != FFFF, keep)
        comp = _components_bfs(keep, nb)
        flat = [float(x) for x in f.ravel()]
        for c in range(comp.max() + 1):
            members = np.nonzero(comp == c)[0]
            deepest = min(members, key=lambda w: (flat[w], w))
            assert np.all(lab[members] == deepest)
        checked += int(keep.sum())
    assert checked > 0


def test_simplified_diagram_equals_filled_fields_diagram():
    for f, _, eps in _cases(150, 21, ties=False):
        W = brute_merge_tree(f)
        g = _filled(f, W, eps)
        Wg = brute_merge_tree(g)
        pg = oracle.simplified_pairs(g, Wg, 1e-30)  # the filled field's pairs of positive persistence
        pf = oracle.simplified_pairs(f, oracle.merge_tree(f), eps)
        assert np.array_equal(pg, pf)


def test_simplification_limits():
    rng = np.random.default_rng(5)
    f = rng.random((9, 7, 11), dtype=np.float32)
    W = oracle.merge_tree(f)
    p, roots = oracle.pairs(W)
    assert np.array_equal(oracle.simplified_pairs(f, W, 0.0), p)
    assert len(oracle.simplified_pairs(f, W, np.inf)) == 0
    t = float(np.median(f))
    lab = oracle.components(f, t)
    assert np.array_equal(oracle.simplified_components(f, W, t, 0.0), lab)
    # eps above every persistence keeps only the root's component
    big = oracle.simplified_components(f, W, t, np.inf)
    kept = np.unique(big[big != FFFF])
    assert list(kept) == [int(roots[0])] or (len(kept) == 0 and lab[roots[0]] == FFFF)


def test_eps_equal_to_a_persistence_keeps_that_pair():
    """A pair whose persistence equals eps is kept (p >= eps); its component
    stays in G_t. The filled field agrees at exactly that boundary."""
    rng = np.random.default_rng(41)
    for _ in range(40):
        f = rng.integers(0, 7, size=(4, 5, 5)).astype(np.float32)
        W = oracle.merge_tree(f)
        p, _ = oracle.pairs(W)
        if len(p) == 0:
            continue
        pers = oracle.persistence(f, W, p[:, 0])
        eps = float(pers[rng.integers(0, len(pers))])
        kept = oracle.simplified_pairs(f, W, eps)
        assert np.array_equal(kept, p[pers >= np.float32(eps)])
        if eps > 0:
            assert len(kept) >= 1 and np.any(oracle.persistence(f, W, kept[:, 0]) == np.float32(eps))
        t = float(rng.uniform(f.min(), f.max()))
        g = _filled(f, brute_merge_tree(f), eps)
        lab = oracle.simplified_components(f, W, t, eps)
        assert np.array_equal(lab != FFFF, g.ravel() <= np.float32(t))
        # a component whose representative's persistence is exactly eps stays
        lab0 = oracle.components(f, t)
        for r in np.unique(lab0[lab0 != FFFF]):
            r = int(r)
            if (int(W[r]) >> 32) == r:
                continue
            er = float(oracle.persistence(f, W, [r])[0])
            lab_r = oracle.simplified_components(f, W, t, er)
            assert np.all(lab_r[lab0 == r] == r)
            gr = _filled(f, brute_merge_tree(f), er)
            assert np.array_equal(lab_r != FFFF, gr.ravel() <= np.float32(t))


def _cases_large(count, seed, ties):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        shape = tuple(int(x) for x in rng.integers(8, 11, size=3))
        f = rng.integers(0, 12, size=shape).astype(np.float32) if ties else rng.random(shape, dtype=np.float32)
        lo, hi = float(f.min()), float(f.max())
        yield f, float(np.float32(rng.uniform(lo, hi))), float(np.float32(rng.uniform(0.0, (hi - lo) * 0.5)))


@pytest.mark.parametrize("ties", [False, True])
def test_filled_field_pins_on_larger_grids(ties):
    """The pit-filling pins on grids of 8 to 10 vertices per side (512 to
    1000 vertices, many nested pits): labels of the simplified G_t, and, on
    distinct values, the simplified diagram."""
    for f, t, eps in _cases_large(8, 31 + ties, ties):
        Wb = brute_merge_tree(f)
        W = oracle.merge_tree(f)
        assert np.array_equal(W, Wb)
        g = _filled(f, Wb, eps)
        lab = oracle.simplified_components(f, W, t, eps)
        nz, ny, nx = f.shape
        nb = _neighbours(nx, ny, nz)
        keep = g.ravel() <= np.float32(t)
        assert np.array_equal(lab != FFFF, keep)
        comp = _components_bfs(keep, nb)
        flat = [float(x) for x in f.ravel()]
        for c in range(comp.max() + 1):
            members = np.nonzero(comp == c)[0]
            deepest = min(members, key=lambda w: (flat[w], w))
            assert np.all(lab[members] == deepest)
        if not ties:
            pg = oracle.simplified_pairs(g, brute_merge_tree(g), 1e-30)
            assert np.array_equal(pg, oracle.simplified_pairs(f, W, eps))
