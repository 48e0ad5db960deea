"""The wide-id path (64-bit vertex ids, grids of 2^32 vertices and more).

Small grids: triplets, pairs and labels equal the 64-bit-id oracle bit for
bit, and equal the 32-bit path's with the ids widened. A grid of 4.6e9
vertices (above 2^32): structural properties over every vertex on the
device, single-vertex oracle queries on a sample that includes ids above
2^32, and label properties.
"""

from __future__ import annotations

import zlib

import numpy as np
import pytest
import torch

import oracle
import paper_2301_10838_gb300 as mt
from paper_2301_10838_gb300 import fields

pytestmark = pytest.mark.gpu

ALL_ONES = np.uint64(0xFFFFFFFFFFFFFFFF)


def run_wide(f_np, t=None, flags=0):
    f = torch.from_numpy(np.ascontiguousarray(f_np, dtype=np.float32)).cuda()
    n = f.numel()
    g = mt.grid_of(f)
    W2 = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    ws = mt.wide_workspace(g)
    mt.mt_build_triplets_wide(f, W2, ws, flags)
    pairs = torch.empty((n // 2 + 1, 2), dtype=torch.int64, device="cuda")
    k, root = mt.mt_persistence_pairs_wide(W2, g, pairs, ws)
    out = {"W2": W2.cpu().numpy().view(np.uint64), "pairs": pairs[:k].cpu().numpy().view(np.uint64), "root": root}
    if t is not None:
        lab = torch.empty(n, dtype=torch.int64, device="cuda")
        mt.mt_components_at_wide(f, W2, t, flags, lab, ws)
        mt.mt_sync_status(ws)
        out["labels"] = lab.cpu().numpy().view(np.uint64)
    return out


RAGGED = [(1, 1, 1), (1, 1, 2), (1, 1, 100), (1, 50, 3), (2, 2, 2), (5, 7, 9), (3, 1, 4), (17, 19, 23),
          (33, 31, 65), (8, 8, 4096 + 5), (40, 40, 40)]


@pytest.mark.parametrize("shape", RAGGED)
@pytest.mark.parametrize("kind", ["uniform", "ties", "zeros", "grf"])
def test_wide_parity_small(shape, kind):
    seed = zlib.crc32(repr((shape, kind, "wide")).encode()) % 1000
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        f = rng.random(shape, dtype=np.float32)
    elif kind == "ties":
        f = rng.integers(0, 4, size=shape).astype(np.float32)
    elif kind == "zeros":
        f = rng.choice(np.array([-0.0, 0.0, 2.0], np.float32), size=shape)
    else:
        if min(shape) < 2:
            pytest.skip("GRF needs 3-D extent")
        f = fields.quantize(fields.grf(shape, -3.0, seed), levels=64)
    t = float(np.median(f))
    got = run_wide(f, t)
    W2 = oracle.merge_tree_wide(f)
    bad = np.nonzero((got["W2"] != W2).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} triplets differ, first at {bad[:5]}"
    p, roots = oracle.pairs_wide(W2)
    assert np.array_equal(got["pairs"], p) and got["root"] == int(roots[0])
    assert np.array_equal(got["labels"], oracle.components_wide(f, t))


def test_wide_superlevel_and_plateaus():
    rng = np.random.default_rng(4)
    f = rng.random((30, 30, 30), dtype=np.float32)
    f[:, :, 15:] = 0.5  # a plateau that joins many basins at one value
    got = run_wide(f, t=0.5, flags=mt.MT_SUPERLEVEL)
    W2 = oracle.merge_tree_wide(-f)
    assert np.array_equal(got["W2"], W2)
    # superlevel labels at t = 0.5: the components of {f >= 0.5}, i.e. of {-f <= -0.5}
    assert np.array_equal(got["labels"], oracle.components_wide(-f, -0.5))


@pytest.mark.parametrize("name", ["white64", "grf256q12"])
def test_wide_equals_narrow_path(name):
    """At the two smaller benchmark configs the wide path's triplets and pairs
    are the 32-bit path's with the ids widened, and the oracle's."""
    f_np = fields.named_field(name, seed=1)
    got = run_wide(f_np)
    f = torch.from_numpy(f_np).cuda()
    W = torch.empty(f.numel(), dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(f))
    mt.mt_build_triplets(f, W, ws)
    mt.mt_sync_status(ws)
    Wn = W.cpu().numpy().view(np.uint64)
    assert np.array_equal(got["W2"][:, 0], Wn >> np.uint64(32))
    assert np.array_equal(got["W2"][:, 1], Wn & np.uint64(0xFFFFFFFF))
    assert np.array_equal(got["W2"], oracle.merge_tree_wide(f_np))


def test_wide_errors():
    f = torch.zeros((4, 4, 4), device="cuda")
    g = mt.grid_of(f)
    ws = mt.wide_workspace(g)
    W2 = torch.empty((64, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(mt.MtError) as e:  # a workspace too small
        mt.mt_build_triplets_wide(f, W2, ws[:256])
    assert e.value.code == -1
    bad = torch.zeros((4, 4, 4), device="cuda")
    bad[1, 2, 3] = float("nan")
    mt.mt_build_triplets_wide(bad, W2, ws)
    with pytest.raises(mt.MtError) as e:
        mt.mt_sync_status(ws)
    assert e.value.code == -3


# ---------------------------------------------------------------- 4.6e9 vertices

def _minima_slab(f, z0, z1):
    """Stencil minima (no 6-neighbour before the vertex in (value, index)
    order) of the z-slab [z0, z1), flattened; computed from the field alone."""
    nz, ny, nx = f.shape
    a, b = max(0, z0 - 1), min(nz, z1 + 1)
    blk = f[a:b]
    nxy = nx * ny
    idx = torch.arange(a * nxy, b * nxy, device=f.device, dtype=torch.int64).view(b - a, ny, nx)
    is_min = torch.ones_like(blk, dtype=torch.bool)
    for dim in range(3):
        L = blk.shape[dim]
        if L < 2:
            continue
        lo, hi = blk.narrow(dim, 0, L - 1), blk.narrow(dim, 1, L - 1)
        ilo, ihi = idx.narrow(dim, 0, L - 1), idx.narrow(dim, 1, L - 1)
        hi_first = (hi < lo) | ((hi == lo) & (ihi < ilo))
        is_min.narrow(dim, 0, L - 1).logical_and_(~hi_first)
        is_min.narrow(dim, 1, L - 1).logical_and_(hi_first)
        del lo, hi, ilo, ihi, hi_first
    return is_min[z0 - a:z0 - a + (z1 - z0)].reshape(-1)


def _before(fa, a, fb, b):
    return (fa < fb) | ((fa == fb) & (a < b))


def check_wide(f, W2, slab=24):
    """Normalisation, minimality, one root, branch starts = stencil minima,
    inner vertices point at branch starts, #pairs = #minima - 1; z-slab by
    z-slab on the device. Returns (minima, pairs)."""
    nz, ny, nx = f.shape
    nxy = nx * ny
    ff = f.reshape(-1)
    s_all, v_all = W2[:, 0], W2[:, 1]
    n = ff.numel()
    nroots = nbranch = nmin = 0
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        a, b = z0 * nxy, z1 * nxy
        u = torch.arange(a, b, device=f.device, dtype=torch.int64)
        s, v = s_all[a:b], v_all[a:b]
        assert int(s.min()) >= 0 and int(s.max()) < n and int(v.min()) >= 0 and int(v.max()) < n
        root = (s == u) & (v == u)
        fu, fs, fv = ff[a:b], ff[s], ff[v]
        assert bool((_before(fv, v, fu, u) | root).all()), "normalisation: v before u"
        assert bool(((s == u) | _before(fu, u, fs, s) | root).all()), "normalisation: u not after s"
        sv, vv = s_all[v], v_all[v]
        v_root = (sv == v) & (vv == v)
        assert bool((v_root | _before(fs, s, ff[sv], sv) | root).all()), "minimality"
        branch = s != u
        mins = _minima_slab(f, z0, z1)
        assert bool(((branch | root) == mins).all()), "branch starts differ from the stencil minima"
        inner = (s == u) & ~root
        assert bool((((sv != v) | v_root) | ~inner).all()), "inner vertex not pointing at a branch start"
        nroots += int(root.sum())
        nbranch += int(branch.sum())
        nmin += int(mins.sum())
        del u, s, v, root, fu, fs, fv, sv, vv, v_root, branch, mins, inner
    assert nroots == 1 and nbranch == nmin - 1
    return nmin, nbranch


def big_field(shape, seed):
    """Seeded uniform noise plus a separable low-frequency product of sines
    (long descent valleys between many small basins), generated slab by slab
    on the device: no FFT of 4.6e9 points is needed."""
    nz, ny, nx = shape
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    ax = [torch.sin(torch.arange(m, device="cuda", dtype=torch.float32) * w + p)
          for m, w, p in ((nz, 0.0213, 0.4), (ny, 0.0187, 1.1), (nx, 0.0241, 2.3))]
    f = torch.empty(shape, dtype=torch.float32, device="cuda")
    for z0 in range(0, nz, 64):
        z1 = min(nz, z0 + 64)
        f[z0:z1] = torch.rand((z1 - z0, ny, nx), generator=gen, device="cuda", dtype=torch.float32)
        f[z0:z1] += 2.0 * ax[0][z0:z1, None, None] * ax[1][None, :, None] * ax[2][None, None, :]
    return f


@pytest.mark.slow
def test_wide_grid_above_2_32_vertices():
    """1700 x 1700 x 1600 = 4,624,000,000 vertices: ids above 2^32 occur in
    triplets, pairs and labels."""
    nz, ny, nx = 1600, 1700, 1700
    n = nx * ny * nz
    assert n > 2**32
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    if free < 170 * 2**30:
        pytest.skip(f"needs ~170 GB of free device memory, {free / 2**30:.0f} GB free")
    f = big_field((nz, ny, nx), seed=3)
    g = mt.grid_of(f)
    W2 = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    ws = mt.wide_workspace(g)
    mt.mt_build_triplets_wide(f, W2, ws)
    mt.mt_sync_status(ws)
    nmin, npairs_chk = check_wide(f, W2)
    probe = torch.empty((0, 2), dtype=torch.int64, device="cuda")
    k, root = mt.mt_persistence_pairs_wide(W2, g, probe, ws, allow_partial=True)
    assert k == npairs_chk == nmin - 1
    pairs = torch.empty((k, 2), dtype=torch.int64, device="cuda")
    k2, root2 = mt.mt_persistence_pairs_wide(W2, g, pairs, ws)
    assert (k2, root2) == (k, root)
    assert int(pairs[:, 0].max()) >= 2**32, "no pair with a minimum id above 2^32"
    assert bool((pairs[1:, 0] > pairs[:-1, 0]).all()), "pairs not in ascending minimum order"
    ff = f.reshape(-1)
    t = float(ff[:: 100003].float().median())
    lab = torch.empty(n, dtype=torch.int64, device="cuda")
    mt.mt_components_at_wide(f, W2, t, 0, lab, ws)
    mt.mt_sync_status(ws)
    # single-vertex oracle queries on a sample, half of it above 2^32
    f_host = f.cpu().numpy()
    rng = np.random.default_rng(0)
    sample = np.concatenate([rng.integers(0, n, 150), rng.integers(2**32, n, 150)])
    mins = pairs[:, 0].cpu().numpy()
    sample = np.concatenate([sample, rng.choice(mins[mins >= 2**32], 100), rng.choice(mins, 50)])
    W2s = W2[torch.from_numpy(sample.astype(np.int64)).cuda()].cpu().numpy().view(np.uint64)
    # (a query is skipped when its flood would visit more than 2^20
    # vertices: the minima of this field's large basins)
    checked = high = 0
    for u, w in zip(sample, W2s):
        r = oracle.point_triplet_wide(f_host, int(u), budget=1 << 20)
        if r is not None:
            checked += 1
            high += int(u) >= 2**32
            assert r == (int(w[0]), int(w[1])), f"vertex {u}: oracle {r} gpu {tuple(int(x) for x in w)}"
    assert checked >= 150 and high >= 50, (checked, high)
    # labels: inside G_t a label is a vertex of G_t labelled by itself, and a
    # vertex and its triplet target share a label
    labs = lab[torch.from_numpy(sample.astype(np.int64)).cuda()].cpu().numpy().view(np.uint64)
    flat = f_host.reshape(-1)
    for u, w, L in zip(sample, W2s, labs):
        if flat[u] <= t:
            assert L != ALL_ONES and flat[int(L)] <= t and int(lab[int(L)].item()) == int(L)
            v = int(w[1]) if int(w[0]) == int(u) else int(u)  # an inner vertex's target lies in its component
            assert int(lab[v].item()) == int(L)
        else:
            assert L == ALL_ONES
