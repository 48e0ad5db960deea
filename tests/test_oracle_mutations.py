"""Planted mistakes in the oracle are caught by its pins (CPU only).

Each case compiles a copy of oracle/mt_oracle.c with one deliberate mistake
into a temporary library, loads it in place of the real one, and checks that
the definition-based pins reject it: the brute-force tree of brute.py
(breadth-first searches over sublevel sets) on tiny grids with ties, and a
breadth-first labelling of G_t. The unmodified source passes the same checks.
"""

from __future__ import annotations

from collections import deque

import numpy as np
import pytest

import oracle
from brute import _neighbours, brute_merge_tree

with open(oracle._SRC) as fh:
    SOURCE = fh.read()

MUTATIONS = {
    "youngest component survives": ("if (before(f, cmin[roots[q]], cmin[e])) e = roots[q];",
                                    "if (before(f, cmin[e], cmin[roots[q]])) e = roots[q];"),
    "dying branch links to the saddle": ("W[cmin[roots[q]]] = pack(u, cmin[e]);",
                                         "W[cmin[roots[q]]] = pack(u, u);"),
    "inner vertex takes its first neighbour's component": ("W[u] = pack(u, cmin[e]);",
                                                         "W[u] = pack(u, cmin[roots[0]]);"),
    "ties broken by the larger index": ("    return a < b;\n}", "    return a > b;\n}"),
    "no +z neighbour": ("    if (z + 1 < g->nz) nb[k++] = u + g->nx * g->ny;\n", ""),
    "sort breaks ties by the larger index": ("    if (a->idx < b->idx) return -1;\n    if (a->idx > b->idx) return 1;",
                                             "    if (a->idx < b->idx) return 1;\n    if (a->idx > b->idx) return -1;"),
    "strict sublevel set": ("        if (!(f[u] <= t)) continue;\n        uint64_t nb[6];",
                            "        if (!(f[u] < t)) continue;\n        uint64_t nb[6];"),
}


def _bfs_labels(f, t):
    nz, ny, nx = f.shape
    flat = [float(x) for x in f.ravel()]
    nb = _neighbours(nx, ny, nz)
    lab = np.full(f.size, 0xFFFFFFFF, dtype=np.uint32)
    for u in range(f.size):
        if flat[u] > t or lab[u] != 0xFFFFFFFF:
            continue
        comp, q = [u], deque([u])
        seen = {u}
        while q:
            x = q.popleft()
            for w in nb[x]:
                if w not in seen and flat[w] <= t:
                    seen.add(w)
                    comp.append(w)
                    q.append(w)
        deep = min(comp, key=lambda w: (flat[w], w))
        lab[comp] = deep
    return lab


def _pins_pass() -> bool:
    rng = np.random.default_rng(77)
    for i in range(60):
        shape = tuple(int(x) for x in rng.integers(1, 5, size=3))
        f = rng.integers(0, 4, size=shape).astype(np.float32) if i % 2 else rng.random(shape, dtype=np.float32)
        if not np.array_equal(oracle.merge_tree(f), brute_merge_tree(f)):
            return False
        t = float(f.ravel()[rng.integers(0, f.size)])  # a threshold equal to a value
        if not np.array_equal(oracle.components(f, t), _bfs_labels(f, t)):
            return False
    return True


def _with_source(src, tmp_path, monkeypatch):
    path = tmp_path / "mt_oracle.c"
    path.write_text(src)
    monkeypatch.setattr(oracle, "_SRC", str(path))
    monkeypatch.setattr(oracle, "_BUILD", str(tmp_path / "_build"))
    monkeypatch.setattr(oracle, "_LIB", str(tmp_path / "_build" / "liboracle.so"))
    monkeypatch.setattr(oracle, "_lib", None)


def test_unmodified_source_passes(tmp_path, monkeypatch):
    _with_source(SOURCE, tmp_path, monkeypatch)
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    assert SOURCE.count(old) == 1, name
    _with_source(SOURCE.replace(old, new), tmp_path, monkeypatch)
    assert not _pins_pass(), f"the pins did not catch: {name}"
