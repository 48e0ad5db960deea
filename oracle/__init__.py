"""CPU oracle for the triplet merge tree (TEST INFRASTRUCTURE ONLY).

The oracle is the plain, slow, sequential construction of Section 2.1 of the
paper (sort the vertices, sweep them with union-find), written in C in
``mt_oracle.c`` and loaded here with ctypes. It shares no code with the CUDA
library. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package; the library itself
never does.

Functions
  merge_tree(f)            -> W   (uint64[n], W[u] = (s << 32) | v)
  sort_order(f), sweep(f, order) the two phases of merge_tree, for timing;
                           sort_order sorts 64-bit order keys with numpy
                           (method="keys") or runs qsort with a comparison
                           function (method="qsort"): the same order
  pairs(W)                 -> (pairs uint32[k, 2] = (minimum, saddle), roots)
  components(f, t)         -> labels (uint32[n]; 0xFFFFFFFF outside G_t)
  point_triplet(f, u, budget) -> W[u] or None if the query exceeds budget
  simplified_pairs(f, W, eps) -> the pairs of persistence >= eps
  simplified_components(f, W, t, eps) -> labels of G_t after filling every
                           branch of persistence < eps up to its saddle
  branches(f, W)           -> (order, offsets): vertices grouped by branch
  tmt_openmp(f, threads)   -> W from the paper's parallel algorithm on the
                           host cores with OpenMP (tmt_openmp.c): a CPU
                           baseline beside the oracle, not the oracle
  merge_tree_wide(f), pairs_wide(W2), components_wide(f, t),
  point_triplet_wide(f, u, budget)   the same with 64-bit ids: W2 is
                           uint64[n, 2] = (s, v), pairs uint64[k, 2], labels
                           uint64 (all ones outside G_t)
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", -1: "invalid", -2: "too large", -3: "non-finite", -4: "capacity", -6: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code} ({STATUS.get(code, '?')})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile mt_oracle.c into oracle/_build/liboracle.so (plain C, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            U32, U64 = ctypes.c_uint32, ctypes.c_uint64
            for name, args in {
                "oracle_sort_order": [P, U32, U32, U32, P],
                "oracle_order_keys": [P, U32, U32, U32, P],
                "oracle_sweep": [P, U32, U32, U32, P, P],
                "oracle_merge_tree": [P, U32, U32, U32, P],
                "oracle_pairs": [P, U64, P, U64, P, P, P],
                "oracle_components": [P, U32, U32, U32, ctypes.c_float, P],
                "oracle_point_triplet": [P, U32, U32, U32, U64, U64, P],
                "oracle_merge_tree_wide": [P, U32, U32, U32, P],
                "oracle_components_wide": [P, U32, U32, U32, ctypes.c_float, P],
                "oracle_point_triplet_wide": [P, U32, U32, U32, U64, U64, P],
            }.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _field(f):
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
    if f.ndim == 1:
        f = f.reshape(1, 1, -1)
    if f.ndim == 2:
        f = f.reshape(1, *f.shape)
    if f.ndim != 3:
        raise ValueError("field must be (nz, ny, nx)")
    nz, ny, nx = f.shape
    return f, nx, ny, nz


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(code: int):
    if code != 0:
        raise OracleError(code)


def sort_order(f, method: str = "keys") -> np.ndarray:
    """Vertex ids in the order (value, linear index) of Section 2.1's sweep.

    method "keys": oracle_order_keys writes one 64-bit key per vertex whose
    unsigned order is that order, numpy sorts the keys (a library sort of
    plain integers) and their low halves are the ids. method "qsort": the C
    library's qsort with a comparison function on (value, index). Both give
    the same order; the second takes minutes at 1024^3.
    """
    f, nx, ny, nz = _field(f)
    if method == "qsort":
        order = np.empty(f.size, dtype=np.uint32)
        _check(_load().oracle_sort_order(_ptr(f), nx, ny, nz, _ptr(order)))
        return order
    if method != "keys":
        raise ValueError(method)
    keys = np.empty(f.size, dtype=np.uint64)
    _check(_load().oracle_order_keys(_ptr(f), nx, ny, nz, _ptr(keys)))
    keys.sort()
    np.bitwise_and(keys, np.uint64(0xFFFFFFFF), out=keys)
    return keys.astype(np.uint32)


def sweep(f, order: np.ndarray) -> np.ndarray:
    f, nx, ny, nz = _field(f)
    order = np.ascontiguousarray(order, dtype=np.uint32)
    W = np.empty(f.size, dtype=np.uint64)
    _check(_load().oracle_sweep(_ptr(f), nx, ny, nz, _ptr(order), _ptr(W)))
    return W


def merge_tree(f, method: str = "keys") -> np.ndarray:
    """Triplet merge tree W[u] = (s << 32) | v of the sublevel sets of f:
    sort the vertices (``sort_order``), then sweep them (``sweep``)."""
    return sweep(f, sort_order(f, method))


def pairs(W: np.ndarray):
    """(pairs[k, 2] = (minimum u, saddle s) by ascending u, roots list).

    oracle_pairs runs twice: once to count, once to write exactly that many
    pairs (no n-sized temporaries, so that 1024^3 trees fit in host memory).
    """
    W = np.ascontiguousarray(W, dtype=np.uint64).ravel()
    n = W.size
    lib = _load()
    npairs = ctypes.c_uint64(0)
    nroots = ctypes.c_uint64(0)
    root = ctypes.c_uint32(0xFFFFFFFF)
    code = lib.oracle_pairs(_ptr(W), n, None, 0, ctypes.byref(npairs), ctypes.byref(nroots), ctypes.byref(root))
    if code not in (0, -4):
        _check(code)
    k = int(npairs.value)
    out = np.empty((max(k, 1), 2), dtype=np.uint32)
    _check(lib.oracle_pairs(_ptr(W), n, _ptr(out), k, ctypes.byref(npairs), ctypes.byref(nroots),
                            ctypes.byref(root)))
    if int(nroots.value) == 1:
        roots = np.array([root.value], dtype=np.uint32)
    else:  # a forest (never for a grid): list every root
        u = np.arange(n, dtype=np.uint64)
        roots = np.nonzero(((W >> np.uint64(32)) == u) & ((W & np.uint64(0xFFFFFFFF)) == u))[0].astype(np.uint32)
        assert len(roots) == int(nroots.value)
    return out[:k].copy() if k else out[:0].copy(), roots


def components(f, t: float) -> np.ndarray:
    """Labels of the components of G_t = {f <= t}: the deepest vertex of each
    component, 0xFFFFFFFF outside G_t. Built from f alone (no merge tree)."""
    f, nx, ny, nz = _field(f)
    lab = np.empty(f.size, dtype=np.uint32)
    _check(_load().oracle_components(_ptr(f), nx, ny, nz, ctypes.c_float(t), _ptr(lab)))
    return lab


def point_triplet(f, u: int, budget: int = 1 << 20):
    """W[u] computed for the single vertex u from the definitions, or None if
    the query would visit more than ``budget`` vertices."""
    f, nx, ny, nz = _field(f)
    out = ctypes.c_uint64(0)
    r = _load().oracle_point_triplet(_ptr(f), nx, ny, nz, int(u), int(budget), ctypes.byref(out))
    if r < 0:
        raise OracleError(r)
    return int(out.value) if r == 1 else None


def persistence(f, W: np.ndarray, u) -> np.ndarray:
    """float32 persistence f(s) - f(u) of the branches born at the minima u
    (s = W[u].s; the subtraction is done in float32, as the GPU path does)."""
    g = np.ascontiguousarray(np.asarray(f, dtype=np.float32)).ravel()
    u = np.asarray(u, dtype=np.int64)
    s = (np.asarray(W, dtype=np.uint64).ravel()[u] >> np.uint64(32)).astype(np.int64)
    return g[s] - g[u]


def simplified_pairs(f, W: np.ndarray, eps: float) -> np.ndarray:
    """Persistence simplification of the diagram (Section 1: a branch's
    persistence measures its importance; short ones are noise): the pairs
    (minimum u, saddle s) with float32 f(s) - f(u) >= eps, by ascending u."""
    p, _ = pairs(W)
    if len(p) == 0:
        return p
    keep = persistence(f, W, p[:, 0]) >= np.float32(eps)
    return p[keep]


def simplified_components(f, W: np.ndarray, t: float, eps: float) -> np.ndarray:
    """Components of G_t after filling every branch of persistence < eps up to
    its saddle. The components of G_t come from ``components`` (union-find
    over the mask, no tree); a component whose deepest vertex r heads a branch
    of W (r not a root) with float32 persistence < eps lies inside a filled
    pit and leaves G_t (label 0xFFFFFFFF); every other component keeps its
    label."""
    lab = components(f, t)
    inside = lab != np.uint32(0xFFFFFFFF)
    reps = np.unique(lab[inside]).astype(np.int64)
    if len(reps) == 0:
        return lab
    Wf = np.asarray(W, dtype=np.uint64).ravel()
    s = (Wf[reps] >> np.uint64(32)).astype(np.int64)
    short = (s != reps) & (persistence(f, Wf, reps) < np.float32(eps))
    out = lab.copy()
    out[np.isin(lab, reps[short].astype(np.uint32)) & inside] = np.uint32(0xFFFFFFFF)
    return out


def branch_of(W: np.ndarray) -> np.ndarray:
    """The branch of every vertex (Section 2.1): a minimum (W[u].s != u) or the
    root heads its own branch; an inner vertex u (W[u] = (u, v), v != u) lies
    on the branch of v, the deepest vertex of its component at level f(u)."""
    W = np.asarray(W, dtype=np.uint64).ravel()
    u = np.arange(W.size, dtype=np.uint64)
    s = W >> np.uint64(32)
    v = W & np.uint64(0xFFFFFFFF)
    return np.where((s == u) & (v != u), v, u).astype(np.uint32)


def branches(f, W: np.ndarray):
    """(order, offsets): every vertex grouped by branch, branches by ascending
    id of their minimum, each group in the vertex order (value, then index) so
    that it starts with its minimum; offsets[i] = start of group i,
    offsets[-1] = n. A stable lexicographic sort (numpy)."""
    g = np.ascontiguousarray(np.asarray(f, dtype=np.float32)).ravel()
    b = branch_of(W)
    n = b.size
    order = np.lexsort((np.arange(n), g, b)).astype(np.uint32)
    sb = b[order]
    heads = np.nonzero(np.r_[True, sb[1:] != sb[:-1]])[0].astype(np.uint32)
    return order, np.r_[heads, np.uint32(n)].astype(np.uint32)


# ---- wide ids (64-bit): the same constructions, for grids of 2^32+ vertices

def merge_tree_wide(f) -> np.ndarray:
    """Triplets with 64-bit ids: W2[u] = (s, v), uint64 array of shape (n, 2).
    The sort (qsort on (value, index)) and sweep of merge_tree, widened."""
    f, nx, ny, nz = _field(f)
    W2 = np.empty((f.size, 2), dtype=np.uint64)
    _check(_load().oracle_merge_tree_wide(_ptr(f), nx, ny, nz, _ptr(W2)))
    return W2


def pairs_wide(W2: np.ndarray):
    """(pairs uint64[k, 2] = (minimum u, saddle s) by ascending u, roots):
    every u with s != u, and the u with (s, v) = (u, u)."""
    W2 = np.asarray(W2, dtype=np.uint64).reshape(-1, 2)
    u = np.arange(W2.shape[0], dtype=np.uint64)
    m = W2[:, 0] != u
    pairs = np.stack([u[m], W2[m, 0]], axis=1) if m.any() else np.zeros((0, 2), np.uint64)
    roots = u[(W2[:, 0] == u) & (W2[:, 1] == u)]
    return np.ascontiguousarray(pairs, dtype=np.uint64), roots


def components_wide(f, t: float) -> np.ndarray:
    """components() with 64-bit labels (all ones outside G_t)."""
    f, nx, ny, nz = _field(f)
    lab = np.empty(f.size, dtype=np.uint64)
    _check(_load().oracle_components_wide(_ptr(f), nx, ny, nz, ctypes.c_float(t), _ptr(lab)))
    return lab


def point_triplet_wide(f, u: int, budget: int = 1 << 20):
    """(s, v) of the single vertex u from the definitions, on grids of any
    size, or None if the query would visit more than ``budget`` vertices."""
    f, nx, ny, nz = _field(f)
    out = np.zeros(2, dtype=np.uint64)
    r = _load().oracle_point_triplet_wide(_ptr(f), nx, ny, nz, int(u), int(budget), _ptr(out))
    if r < 0:
        raise OracleError(r)
    return (int(out[0]), int(out[1])) if r == 1 else None


# ---- CPU baseline: the paper's parallel algorithm with OpenMP (not the oracle)

_OMP_SRC = os.path.join(_HERE, "tmt_openmp.c")
_OMP_LIB = os.path.join(_BUILD, "libtmt_openmp.so")
_omp = None


def build_openmp(force: bool = False) -> str:
    """Compile tmt_openmp.c (gcc -fopenmp) into oracle/_build/libtmt_openmp.so."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_OMP_LIB) or os.path.getmtime(_OMP_LIB) < os.path.getmtime(_OMP_SRC)
    if stale:
        tmp = _OMP_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _OMP_SRC, "-lm"])
        os.replace(tmp, _OMP_LIB)
    return _OMP_LIB


def tmt_openmp(f, threads: int | None = None) -> np.ndarray:
    """Triplets W[u] = (s << 32) | v from Algorithm 1 of the paper run in
    parallel on `threads` host cores (default: all), seeded with (u, u), every
    edge merged with a 64-bit compare-and-swap, then repaired. The result is
    unique, so it equals merge_tree(f); the tests check that."""
    global _omp
    with _lock:
        if _omp is None:
            lib = ctypes.CDLL(build_openmp())
            lib.tmt_openmp.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_int, ctypes.c_void_p]
            lib.tmt_openmp.restype = ctypes.c_int
            _omp = lib
    f, nx, ny, nz = _field(f)
    W = np.empty(f.size, dtype=np.uint64)
    _check(_omp.tmt_openmp(_ptr(f), nx, ny, nz, int(threads or os.cpu_count() or 1), _ptr(W)))
    return W
