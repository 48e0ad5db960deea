"""Brute-force triplet merge tree straight from the definitions (tiny grids).

Used only to pin the oracle. It uses no sort-and-sweep and no union-find:
for every vertex it runs breadth-first searches over sublevel sets
(Section 2.1 of the paper: merge tree, sublevel set G_c, triplets,
normalisation and minimality).

For each vertex u, with the total order (value, linear index):
  * C = u's component of {w : w <= u}. If u is not the deepest vertex of C,
    u lies inside a branch: T[u] = (u, deepest(C)).
  * Otherwise u is a minimum. Walk the levels x after u in order; the first x
    at which u's component of {w : w <= x} holds a vertex before u is the
    saddle s where u's branch merges into an older one, and
    T[u] = (s, deepest of that component).
  * If no level does, u is the deepest vertex of its whole (connected) grid:
    T[u] = (u, u).
Cost is O(n^2) breadth-first searches; keep n to a few hundred.
"""

from __future__ import annotations

from collections import deque

import numpy as np


def _neighbours(nx: int, ny: int, nz: int):
    n = nx * ny * nz
    nb = [[] for _ in range(n)]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                u = x + nx * (y + ny * z)
                if x > 0:
                    nb[u].append(u - 1)
                if x + 1 < nx:
                    nb[u].append(u + 1)
                if y > 0:
                    nb[u].append(u - nx)
                if y + 1 < ny:
                    nb[u].append(u + nx)
                if z > 0:
                    nb[u].append(u - nx * ny)
                if z + 1 < nz:
                    nb[u].append(u + nx * ny)
    return nb


def _component(nb, rank, u, level_rank):
    """Vertices reachable from u through vertices of rank <= level_rank."""
    seen = {u}
    q = deque([u])
    while q:
        x = q.popleft()
        for w in nb[x]:
            if w not in seen and rank[w] <= level_rank:
                seen.add(w)
                q.append(w)
    return seen


def brute_merge_tree(f) -> np.ndarray:
    f = np.asarray(f, dtype=np.float32)
    if f.ndim == 1:
        f = f.reshape(1, 1, -1)
    if f.ndim == 2:
        f = f.reshape(1, *f.shape)
    nz, ny, nx = f.shape
    n = f.size
    flat = [float(x) for x in f.ravel()]
    # total order (value, index) by Python's own tuple sort
    order = sorted(range(n), key=lambda i: (flat[i], i))
    rank = [0] * n
    for r, i in enumerate(order):
        rank[i] = r
    nb = _neighbours(nx, ny, nz)
    W = np.zeros(n, dtype=np.uint64)
    for u in range(n):
        comp = _component(nb, rank, u, rank[u])
        deep = min(comp, key=lambda w: rank[w])
        if deep != u:
            W[u] = (u << 32) | deep
            continue
        W[u] = (u << 32) | u
        for r in range(rank[u] + 1, n):
            comp = _component(nb, rank, u, r)
            deep = min(comp, key=lambda w: rank[w])
            if rank[deep] < rank[u]:
                s = order[r]
                W[u] = (s << 32) | deep
                break
    return W


def elder_rule_1d(values) -> np.ndarray:
    """Triplets of a 1-D line (nx = n, ny = nz = 1) by intervals.

    On a path graph the component of u in {w <= c} is the maximal interval
    around u of vertices <= c, so:
      * a vertex with a lower neighbour: T[u] = (u, deepest of its interval
        at level u);
      * a minimum u: walk left and right until the first vertex before u;
        the latest vertex passed on a side is that side's barrier. The saddle
        is the earlier of the barriers that exist (the elder rule), and v is
        the deepest vertex of the interval at the saddle's level. With no
        barrier on either side u is the global minimum, T[u] = (u, u).
    """
    vals = [float(x) for x in np.asarray(values, dtype=np.float32).ravel()]
    n = len(vals)

    def before(a, b):
        return (vals[a], a) < (vals[b], b)

    def interval_deepest(u, c):
        lo = u
        while lo - 1 >= 0 and not before(c, lo - 1):
            lo -= 1
        hi = u
        while hi + 1 < n and not before(c, hi + 1):
            hi += 1
        return min(range(lo, hi + 1), key=lambda w: (vals[w], w))

    W = np.zeros(n, dtype=np.uint64)
    for u in range(n):
        lower = [w for w in (u - 1, u + 1) if 0 <= w < n and before(w, u)]
        if lower:
            W[u] = (u << 32) | interval_deepest(u, u)
            continue
        barriers = []
        for step in (-1, 1):
            w, top = u + step, None
            while 0 <= w < n and not before(w, u):
                if top is None or before(top, w):
                    top = w
                w += step
            if 0 <= w < n and top is not None:
                barriers.append(top)
        if not barriers:
            W[u] = (u << 32) | u
            continue
        s = min(barriers, key=lambda w: (vals[w], w))
        W[u] = (s << 32) | interval_deepest(u, s)
    return W
