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
    "sort breaks ties by the larger index": (
        "*b = (const keyed_t *)pb;\n    if (a->val < b->val) return -1;\n    if (a->val > b->val) return 1;\n"
        "    if (a->idx < b->idx) return -1;\n    if (a->idx > b->idx) return 1;",
        "*b = (const keyed_t *)pb;\n    if (a->val < b->val) return -1;\n    if (a->val > b->val) return 1;\n"
        "    if (a->idx < b->idx) return 1;\n    if (a->idx > b->idx) return -1;"),
    "strict sublevel set": (
        "        if (!(f[u] <= t)) continue;\n        uint64_t nb[6];\n        int nn = neighbours(&g, u, nb);\n"
        "        for (int j = 0; j < nn; j++) {\n            if (!(f[nb[j]] <= t)) continue;\n            uint32_t a",
        "        if (!(f[u] < t)) continue;\n        uint64_t nb[6];\n        int nn = neighbours(&g, u, nb);\n"
        "        for (int j = 0; j < nn; j++) {\n            if (!(f[nb[j]] <= t)) continue;\n            uint32_t a"),
    "key keeps -0 below +0": ("        if (x == 0.0f) x = 0.0f; /* -0 -> +0 */\n", ""),
    "key of a negative value not flipped": ("uint32_t m = (b & 0x80000000u) ? ~b : (b | 0x80000000u);",
                                           "uint32_t m = (b & 0x80000000u) ? b : (b | 0x80000000u);"),
    "key is the raw bit pattern": ("uint32_t m = (b & 0x80000000u) ? ~b : (b | 0x80000000u);",
                                   "uint32_t m = b;"),
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


SIGNED = np.array([-0.0, 0.0, -1.5, 2.0, -2.5, 1e-45, -1e-45], np.float32)


def _pins_pass() -> bool:
    rng = np.random.default_rng(77)
    for i in range(60):
        shape = tuple(int(x) for x in rng.integers(1, 5, size=3))
        if i % 3 == 2:  # signed zeros, negative values and subnormals
            f = rng.choice(SIGNED, size=shape)
        else:
            f = rng.integers(0, 4, size=shape).astype(np.float32) if i % 2 else rng.random(shape, dtype=np.float32)
        want = brute_merge_tree(f)
        for method in ("keys", "qsort"):  # both sorts of the sweep
            if not np.array_equal(oracle.merge_tree(f, method), want):
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


# ---- the numpy layer of the oracle: simplification and branches

def _simplify_pins_pass() -> bool:
    from test_oracle_simplify import FFFF, _cases, _filled

    for ties in (False, True):
        for f, t, eps in _cases(60, 101 + ties, ties):
            W = oracle.merge_tree(f)
            g = _filled(f, brute_merge_tree(f), eps)
            lab = oracle.simplified_components(f, W, t, eps)
            if not np.array_equal(lab != FFFF, g.ravel() <= np.float32(t)):
                return False
            # eps equal to a representative's persistence keeps its component
            lab0 = oracle.components(f, t)
            reps = [int(r) for r in np.unique(lab0[lab0 != FFFF]) if (int(W[r]) >> 32) != int(r)]
            if reps:
                e1 = float(oracle.persistence(f, W, [reps[0]])[0])
                lab1 = oracle.simplified_components(f, W, t, e1)
                g1 = _filled(f, brute_merge_tree(f), e1)
                if not np.array_equal(lab1 != FFFF, g1.ravel() <= np.float32(t)) or np.any(lab1[lab0 == reps[0]] == FFFF):
                    return False
            # eps equal to a persistence keeps that pair
            p, _ = oracle.pairs(W)
            if len(p):
                pers = oracle.persistence(f, W, p[:, 0])
                e0 = float(pers[0])
                if not np.array_equal(oracle.simplified_pairs(f, W, e0), p[pers >= np.float32(e0)]):
                    return False
    return True


def _branch_pins_pass() -> bool:
    from test_oracle_branches import _brute_branch

    rng = np.random.default_rng(9)
    for _ in range(40):
        shape = tuple(int(x) for x in rng.integers(1, 5, size=3))
        f = rng.integers(0, 4, size=shape).astype(np.float32)
        W = oracle.merge_tree(f)
        if not np.array_equal(oracle.branch_of(W), _brute_branch(f)):
            return False
        order, offsets = oracle.branches(f, W)
        flat = [float(x) for x in f.ravel()]
        b = oracle.branch_of(W)
        if [int(x) for x in order] != sorted(range(f.size), key=lambda i: (int(b[i]), flat[i], i)):
            return False
    return True


def test_numpy_layer_passes_unmodified():
    assert _simplify_pins_pass() and _branch_pins_pass()


def _persistence_from_target(f, W, u):
    g = np.ascontiguousarray(np.asarray(f, dtype=np.float32)).ravel()
    u = np.asarray(u, dtype=np.int64)
    v = (np.asarray(W, dtype=np.uint64).ravel()[u] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    return g[v] - g[u]


def _simplified_components_le(f, W, t, eps):
    lab = oracle.components(f, t)
    inside = lab != np.uint32(0xFFFFFFFF)
    reps = np.unique(lab[inside]).astype(np.int64)
    if len(reps) == 0:
        return lab
    Wf = np.asarray(W, dtype=np.uint64).ravel()
    s = (Wf[reps] >> np.uint64(32)).astype(np.int64)
    short = (s != reps) & (oracle.persistence(f, Wf, reps) <= np.float32(eps))  # planted: <= for <
    out = lab.copy()
    out[np.isin(lab, reps[short].astype(np.uint32)) & inside] = np.uint32(0xFFFFFFFF)
    return out


def _branch_of_self(W):
    return np.arange(np.asarray(W).size, dtype=np.uint32)  # planted: every vertex heads its own branch


def _branches_descending(f, W):
    g = np.ascontiguousarray(np.asarray(f, dtype=np.float32)).ravel()
    b = oracle.branch_of(W)
    order = np.lexsort((np.arange(b.size), -g, b)).astype(np.uint32)  # planted: values descending
    sb = b[order]
    heads = np.nonzero(np.r_[True, sb[1:] != sb[:-1]])[0].astype(np.uint32)
    return order, np.r_[heads, np.uint32(b.size)].astype(np.uint32)


@pytest.mark.parametrize("name,attr,fake,pins", [
    ("persistence from the target, not the saddle", "persistence", _persistence_from_target, "simplify"),
    ("a pair at exactly eps dropped", "simplified_components", _simplified_components_le, "simplify"),
    ("every vertex its own branch", "branch_of", _branch_of_self, "branches"),
    ("groups in descending value", "branches", _branches_descending, "branches"),
])
def test_numpy_layer_mistake_is_caught(name, attr, fake, pins, monkeypatch):
    monkeypatch.setattr(oracle, attr, fake)
    ok = _simplify_pins_pass() if pins == "simplify" else _branch_pins_pass()
    assert not ok, f"the pins did not catch: {name}"


# ---- the 64-bit-id constructions

WIDE_MUTATIONS = {
    "wide: youngest component survives": ("if (before(f, cmin[roots[c]], cmin[e])) e = roots[c];",
                                          "if (before(f, cmin[e], cmin[roots[c]])) e = roots[c];"),
    "wide: dying branch links to the saddle": ("W2[2 * cmin[roots[c]] + 1] = cmin[e];",
                                               "W2[2 * cmin[roots[c]] + 1] = u;"),
    "wide: labels keep the first vertex": ("if (deep[r] == UINT64_MAX || before(f, u, deep[r])) deep[r] = u;",
                                           "if (deep[r] == UINT64_MAX) deep[r] = u;"),
}


def _wide_pins_pass() -> bool:
    rng = np.random.default_rng(78)
    for i in range(60):
        shape = tuple(int(x) for x in rng.integers(1, 5, size=3))
        f = rng.integers(0, 4, size=shape).astype(np.float32) if i % 2 else rng.random(shape, dtype=np.float32)
        W = brute_merge_tree(f)
        W2 = oracle.merge_tree_wide(f)
        if not (np.array_equal(W2[:, 0], W >> np.uint64(32)) and np.array_equal(W2[:, 1], W & np.uint64(0xFFFFFFFF))):
            return False
        t = float(f.ravel()[rng.integers(0, f.size)])
        lab = _bfs_labels(f, t).astype(np.uint64)
        lab[lab == 0xFFFFFFFF] = np.uint64(0xFFFFFFFFFFFFFFFF)
        if not np.array_equal(oracle.components_wide(f, t), lab):
            return False
    return True


def test_wide_unmodified_source_passes(tmp_path, monkeypatch):
    _with_source(SOURCE, tmp_path, monkeypatch)
    assert _wide_pins_pass()


@pytest.mark.parametrize("name", sorted(WIDE_MUTATIONS))
def test_wide_planted_mistake_is_caught(name, tmp_path, monkeypatch):
    old, new = WIDE_MUTATIONS[name]
    assert SOURCE.count(old) == 1, name
    _with_source(SOURCE.replace(old, new), tmp_path, monkeypatch)
    assert not _wide_pins_pass(), f"the pins did not catch: {name}"
