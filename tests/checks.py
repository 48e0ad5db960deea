"""Structural checks on a triplet array W (test helpers, torch CPU or CUDA).

These are properties that any correct triplet merge tree of a connected grid
has at every size (Section 2.1 of the paper: normalisation, minimality, one
triplet (u, u, u) per connected component), plus independent recomputations
(local minima by a stencil, component counts), so they can check outputs too
large for the oracle to recompute in full.
"""

from __future__ import annotations

import numpy as np
import torch

MASK32 = 0xFFFFFFFF


def _t(a, device=None):
    if isinstance(a, torch.Tensor):
        return a if device is None else a.to(device)
    return torch.from_numpy(np.ascontiguousarray(a)).to(device or "cpu")


def split(W):
    """W -> (s, v) as int64 tensors."""
    W = _t(W).view(torch.int64).reshape(-1)
    s = (W >> 32) & MASK32
    v = W & MASK32
    return s, v


def before(fv_a, ia, fv_b, ib):
    """Elementwise total order (value, index): a before b."""
    return (fv_a < fv_b) | ((fv_a == fv_b) & (ia < ib))


def local_minima_mask(f) -> torch.Tensor:
    """Vertices with no 6-neighbour before them in (value, index) order,
    computed from the field alone by shifted comparisons."""
    f = _t(f)
    nz, ny, nx = f.shape
    dev = f.device
    idx = torch.arange(f.numel(), device=dev, dtype=torch.int64).view(nz, ny, nx)
    is_min = torch.ones_like(f, dtype=torch.bool)
    for dim in range(3):
        L = f.shape[dim]
        if L < 2:
            continue
        a = f.narrow(dim, 0, L - 1)
        b = f.narrow(dim, 1, L - 1)
        ia = idx.narrow(dim, 0, L - 1)
        ib = idx.narrow(dim, 1, L - 1)
        b_first = before(b, ib, a, ia)  # the upper neighbour is before the lower one
        is_min.narrow(dim, 0, L - 1).logical_and_(~b_first)
        is_min.narrow(dim, 1, L - 1).logical_and_(b_first)
    return is_min.reshape(-1)


def check_triplets(f, W, chunk: int = 1 << 26) -> dict:
    """Assert the properties every exact result has; return summary counts.

    1. normalisation: a root has s = v = u; otherwise v before u and u <= s;
    2. minimality: for a non-root (u, s, v), T[v] is a root or T[v].s after s;
    3. exactly one root (the grid is connected);
    4. the branch-starting vertices {u : s != u} plus the root are exactly the
       local minima found by the stencil;
    5. a vertex inside a branch (s == u != v) points at a branch-starting
       vertex;
    6. #pairs = #minima - 1.
    """
    f = _t(f)
    dev = f.device
    ff = f.reshape(-1)
    n = ff.numel()
    s, v = split(_t(W, dev))
    assert s.numel() == n
    nroots = 0
    nbranch = 0
    minmask = local_minima_mask(f)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        u = torch.arange(a, b, device=dev, dtype=torch.int64)
        sc, vc = s[a:b], v[a:b]
        assert int(sc.max()) < n and int(vc.max()) < n, "ids out of range"
        root = (sc == u) & (vc == u)
        nonroot = ~root
        fu, fs, fv = ff[u], ff[sc], ff[vc]
        ok_v = before(fv, vc, fu, u)
        ok_s = (sc == u) | before(fu, u, fs, sc)
        assert bool((ok_v | root).all()), "normalisation: v must come before u"
        assert bool((ok_s | root).all()), "normalisation: u must not come after s"
        sv, vv = s[vc], v[vc]
        v_root = (sv == vc) & (vv == vc)
        later = before(fs, sc, ff[sv], sv)
        assert bool((v_root | later | root).all()), "minimality violated"
        branch = sc != u
        starts = branch | root
        assert bool((starts == minmask[a:b]).all()), "branch starts differ from the stencil minima"
        inner = (sc == u) & nonroot
        v_start = (sv != vc) | v_root
        assert bool((v_start | ~inner).all()), "an inner vertex must point at a branch start"
        nroots += int(root.sum())
        nbranch += int(branch.sum())
    assert nroots == 1, f"expected one root, got {nroots}"
    nmin = int(minmask.sum())
    assert nbranch == nmin - 1
    return {"n": n, "minima": nmin, "pairs": nbranch, "roots": nroots}


def diagram(f, W) -> np.ndarray:
    """Off-diagonal 0-dim persistence diagram {(f(u), f(s)) : f(s) > f(u)}
    as a sorted float64 array of shape (k, 2)."""
    f = np.asarray(f, dtype=np.float32).ravel()
    W = np.asarray(W, dtype=np.uint64).ravel()
    u = np.arange(W.size, dtype=np.uint64)
    s = W >> np.uint64(32)
    m = s != u
    pts = np.stack([f[u[m].astype(np.int64)], f[s[m].astype(np.int64)]], axis=1).astype(np.float64)
    pts = pts[pts[:, 1] > pts[:, 0]]
    order = np.lexsort((pts[:, 1], pts[:, 0]))
    return pts[order]
