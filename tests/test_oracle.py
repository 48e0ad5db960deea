"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: hand-derived
fixtures, a brute-force construction from the definitions, closed forms,
a 1-D interval construction of the elder rule, a stencil for the local
minima, scipy's connected-component labelling, and the invariance of the
off-diagonal persistence diagram under a change of tie-break.
"""

from __future__ import annotations

import itertools
import os

import numpy as np
import pytest

import oracle
from brute import brute_merge_tree, elder_rule_1d
from checks import check_triplets, diagram, local_minima_mask
from paper_2301_10838_gb300 import fields

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    field, shape, W, pairs, roots = None, None, {}, [], []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if not line:
                continue
            tag, rest = line[0], line[1:]
            if tag == "field":
                field = np.array([float(x) for x in rest], dtype=np.float32)
            elif tag == "shape":
                shape = tuple(int(x) for x in rest)
            elif tag == "W":
                u, s, v = (int(x) for x in rest)
                W[u] = (s << 32) | v
            elif tag == "pair":
                pairs.append(tuple(int(x) for x in rest))
            elif tag == "root":
                roots.append(int(rest[0]))
    Wa = np.array([W[u] for u in range(len(W))], dtype=np.uint64)
    return field.reshape(shape), Wa, np.array(pairs, dtype=np.uint32).reshape(-1, 2), roots


@pytest.mark.parametrize("name", ["line8.txt", "ties2x3.txt"])
def test_hand_derived_fixture(name):
    f, W, pairs, roots = _load_golden(name)
    got = oracle.merge_tree(f)
    assert np.array_equal(got, W)
    p, r = oracle.pairs(got)
    assert np.array_equal(p, pairs)
    assert list(r) == roots
    # the brute force agrees with the hand derivation too
    assert np.array_equal(brute_merge_tree(f), W)


def _tiny_fields(seed):
    rng = np.random.default_rng(seed)
    shapes = [(1, 1, 7), (1, 1, 1), (1, 3, 5), (2, 2, 2), (3, 1, 4), (2, 3, 4), (4, 4, 4), (1, 5, 5), (3, 3, 3)]
    shape = shapes[seed % len(shapes)]
    kind = seed % 4
    if kind == 0:
        f = rng.random(shape, dtype=np.float32)
    elif kind == 1:  # heavy ties
        f = rng.integers(0, 3, size=shape).astype(np.float32)
    elif kind == 2:  # ties with signed zeros mixed in
        f = rng.choice(np.array([-0.0, 0.0, 1.0, -1.0], dtype=np.float32), size=shape)
    else:
        f = rng.integers(0, 8, size=shape).astype(np.float32) * np.float32(0.25)
    return f


@pytest.mark.parametrize("block", range(6))
def test_brute_force_tiny(block):
    for seed in range(block * 150, (block + 1) * 150):
        f = _tiny_fields(seed)
        want = brute_merge_tree(f)
        got = oracle.merge_tree(f)
        assert np.array_equal(got, want), f"seed {seed} shape {f.shape}"


def test_brute_force_6cube():
    for seed in range(6):
        rng = np.random.default_rng(100 + seed)
        f = rng.integers(0, 5 if seed % 2 else 1000, size=(6, 6, 6)).astype(np.float32)
        assert np.array_equal(oracle.merge_tree(f), brute_merge_tree(f))


def test_all_equal_and_ramp():
    for shape in [(1, 1, 9), (3, 4, 5), (8, 8, 8)]:
        n = int(np.prod(shape))
        for f in (np.zeros(shape, np.float32),
                  np.add.outer(np.add.outer(np.arange(shape[0]), np.arange(shape[1])),
                               np.arange(shape[2])).astype(np.float32)):
            W = oracle.merge_tree(f)
            s = W >> np.uint64(32)
            v = W & np.uint64(0xFFFFFFFF)
            assert np.array_equal(s, np.arange(n, dtype=np.uint64)), "no vertex starts a branch but 0"
            assert np.all(v == 0), "every vertex points at vertex 0"
            p, roots = oracle.pairs(W)
            assert len(p) == 0 and list(roots) == [0]


@pytest.mark.parametrize("seed", range(12))
def test_elder_rule_line(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 400))
    if seed % 3 == 0:
        f = rng.integers(0, 6, size=n).astype(np.float32)
    else:
        f = rng.random(n, dtype=np.float32)
    assert np.array_equal(oracle.merge_tree(f.reshape(1, 1, n)), elder_rule_1d(f))
    # the same line laid along y and along z is the same graph with other ids
    Wy = oracle.merge_tree(f.reshape(1, n, 1))
    Wz = oracle.merge_tree(f.reshape(n, 1, 1))
    assert np.array_equal(Wy, Wz)
    assert np.array_equal(Wy, elder_rule_1d(f))


def _minima_1d(g):
    g = np.asarray(g)
    m = 0
    for i in range(len(g)):
        left = i == 0 or g[i - 1] > g[i]
        right = i == len(g) - 1 or g[i + 1] > g[i]
        m += left and right
    return m


@pytest.mark.parametrize("seed", range(4))
def test_separable_sum_counts(seed):
    """f = gz[z] + gy[y] + gx[x] with distinct integer g: u is a local minimum
    iff each coordinate is a 1-D local minimum, so #minima = mz*my*mx and
    #pairs = #minima - 1 (connected grid)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = (int(x) for x in rng.integers(5, 24, size=3))
    gz, gy, gx = (rng.permutation(k).astype(np.float32) for k in (nz, ny, nx))
    f = (gz[:, None, None] + gy[None, :, None] + gx[None, None, :]).astype(np.float32)
    W = oracle.merge_tree(f)
    p, roots = oracle.pairs(W)
    nmin = _minima_1d(gz) * _minima_1d(gy) * _minima_1d(gx)
    assert len(p) == nmin - 1
    assert len(roots) == 1


@pytest.mark.parametrize("name,side", [("white64", 32), ("grf256q12", 32), ("lognorm1024", 24)])
def test_structure_and_minima_stencil(name, side):
    f = fields.named_field(name, seed=3, side=side)
    W = oracle.merge_tree(f)
    info = check_triplets(f, W)
    assert info["minima"] == int(local_minima_mask(f).sum())


def test_white_noise_minima_density():
    """i.i.d. values: a vertex with k neighbours is a minimum with probability
    1/(k+1); the oracle's branch count must follow that expectation."""
    f = fields.named_field("white64", seed=1)
    W = oracle.merge_tree(f)
    p, roots = oracle.pairs(W)
    n = 64
    expect = ((n - 2) ** 3) / 7 + 6 * ((n - 2) ** 2) / 6 + 12 * (n - 2) / 5 + 8 / 4
    assert abs((len(p) + 1) - expect) < 5 * np.sqrt(expect)


@pytest.mark.parametrize("seed", range(3))
def test_tie_break_independence(seed):
    """Reversing the index order changes how ties are broken but not the
    off-diagonal diagram {(f(u), f(s)) : f(s) > f(u)}."""
    f = fields.quantize(fields.grf((20, 18, 22), -3.0, seed), levels=32)
    d1 = diagram(f, oracle.merge_tree(f))
    fr = np.ascontiguousarray(f[::-1, ::-1, ::-1])
    d2 = diagram(fr, oracle.merge_tree(fr))
    assert d1.shape == d2.shape and d1.shape[0] > 10
    assert np.array_equal(d1, d2)


@pytest.mark.parametrize("seed", range(3))
def test_components_vs_scipy(seed):
    nd = pytest.importorskip("scipy.ndimage")
    f = fields.named_field("grf256q12", seed=seed + 1, side=28)
    rng = np.random.default_rng(seed)
    for t in rng.uniform(0.2, 0.8, size=3).astype(np.float32):
        lab = oracle.components(f, float(t)).reshape(f.shape)
        ref, nref = nd.label(f <= t, structure=nd.generate_binary_structure(3, 1))
        mask = f <= t
        assert np.array_equal(lab != 0xFFFFFFFF, mask)
        flat = f.ravel()
        for c in range(1, nref + 1):
            members = np.nonzero(ref.ravel() == c)[0]
            labs = np.unique(lab.ravel()[members])
            assert len(labs) == 1
            deepest = members[np.lexsort((members, flat[members]))[0]]
            assert labs[0] == deepest


def test_component_count_identity():
    """#components(G_t) = #{minima with f <= t} - #{pairs with f(s) <= t}."""
    f = fields.named_field("white64", seed=2, side=30)
    W = oracle.merge_tree(f)
    p, roots = oracle.pairs(W)
    flat = f.ravel()
    mins = np.nonzero(local_minima_mask(f).numpy())[0]
    for t in (0.05, 0.2, 0.5, 0.9):
        lab = oracle.components(f, t)
        ncomp = len(np.unique(lab[lab != 0xFFFFFFFF]))
        want = int((flat[mins] <= t).sum()) - int((flat[p[:, 1]] <= t).sum())
        assert ncomp == want


def test_point_query_matches_full():
    f = fields.named_field("grf256q12", seed=2, side=12)
    W = oracle.merge_tree(f)
    for u in range(f.size):
        assert oracle.point_triplet(f, u, budget=f.size) == int(W[u])
    g = fields.named_field("white64", seed=5)
    Wg = oracle.merge_tree(g)
    rng = np.random.default_rng(0)
    hits = 0
    for u in rng.integers(0, g.size, size=300):
        r = oracle.point_triplet(g, int(u), budget=1 << 16)
        if r is not None:
            hits += 1
            assert r == int(Wg[u])
    assert hits > 50


def test_point_query_budget():
    f = np.zeros((10, 10, 10), np.float32)
    assert oracle.point_triplet(f, 999, budget=10) is None
    assert oracle.point_triplet(f, 999, budget=1000) == (999 << 32)


def test_status_codes():
    f = np.zeros((2, 2, 2), np.float32)
    f[1, 1, 1] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.merge_tree(f)
    assert e.value.code == -3
    f[1, 1, 1] = np.inf
    with pytest.raises(oracle.OracleError):
        oracle.merge_tree(f)
    with pytest.raises(oracle.OracleError) as e:
        oracle.merge_tree(np.zeros((0, 2, 2), np.float32))
    assert e.value.code == -1


def test_split_phases_equal_whole():
    f = fields.named_field("white64", seed=4, side=20)
    order = oracle.sort_order(f)
    assert np.array_equal(oracle.sweep(f, order), oracle.merge_tree(f))
    flat = f.ravel()
    keys = list(zip(flat[order].tolist(), order.tolist()))
    assert keys == sorted(keys)


def test_key_sort_equals_comparison_sort():
    """The two sorts of the sweep give the same order: 64-bit keys sorted by
    numpy and qsort with a comparison on (value, index). Inputs with heavy
    ties, signed zeros, negative values and subnormals; the qsort order is
    itself pinned by the brute-force trees above."""
    rng = np.random.default_rng(3)
    pool = np.array([-0.0, 0.0, -1.5, 2.0, -2.5, 1e-45, -1e-45, -3.4e38, 3.4e38], np.float32)
    for i in range(200):
        shape = tuple(int(x) for x in rng.integers(1, 9, size=3))
        if i % 3 == 0:
            f = rng.choice(pool, size=shape)
        elif i % 3 == 1:
            f = rng.integers(-3, 3, size=shape).astype(np.float32)
        else:
            f = rng.standard_normal(shape).astype(np.float32)
        a = oracle.sort_order(f, "keys")
        b = oracle.sort_order(f, "qsort")
        assert np.array_equal(a, b), shape
        # and the order is the Python tuple sort by (value, index), with -0 == +0
        flat = [float(x) for x in f.ravel()]
        assert [int(x) for x in a] == sorted(range(f.size), key=lambda j: (flat[j], j))


def test_order_keys_non_finite_refused():
    for bad in (np.nan, np.inf, -np.inf):
        f = np.zeros((2, 2, 2), np.float32)
        f[1, 0, 1] = bad
        with pytest.raises(oracle.OracleError) as e:
            oracle.sort_order(f, "keys")
        assert e.value.code == -3


def test_wide_oracle_equals_brute_force_and_widened_oracle():
    """The 64-bit-id oracle (grids of 2^32+ vertices): on tiny grids with
    ties and signed zeros its triplets are the brute-force tree's, and on
    larger ones they, its pairs, labels and point queries equal the 32-bit
    oracle's with the ids widened."""
    rng = np.random.default_rng(11)
    for i in range(120):
        shape = tuple(int(x) for x in rng.integers(1, 5, size=3))
        f = rng.choice(np.array([-0.0, 0.0, 1.0, 2.0], np.float32), size=shape) if i % 2 else \
            rng.random(shape, dtype=np.float32)
        W = brute_merge_tree(f)
        W2 = oracle.merge_tree_wide(f)
        assert np.array_equal(W2[:, 0], W >> np.uint64(32)) and np.array_equal(W2[:, 1], W & np.uint64(0xFFFFFFFF))
    for i in range(30):
        shape = tuple(int(x) for x in rng.integers(3, 14, size=3))
        f = rng.integers(0, 6, size=shape).astype(np.float32) if i % 2 else rng.random(shape, dtype=np.float32)
        W = oracle.merge_tree(f)
        W2 = oracle.merge_tree_wide(f)
        assert np.array_equal(W2[:, 0], W >> np.uint64(32)) and np.array_equal(W2[:, 1], W & np.uint64(0xFFFFFFFF))
        p, r = oracle.pairs(W)
        p2, r2 = oracle.pairs_wide(W2)
        assert np.array_equal(p.astype(np.uint64), p2) and np.array_equal(r.astype(np.uint64), r2)
        t = float(np.median(f))
        lab = oracle.components(f, t).astype(np.uint64)
        lab[lab == 0xFFFFFFFF] = np.uint64(0xFFFFFFFFFFFFFFFF)
        assert np.array_equal(lab, oracle.components_wide(f, t))
        for u in rng.integers(0, f.size, 5):
            assert oracle.point_triplet_wide(f, int(u)) == (int(W2[u, 0]), int(W2[u, 1]))


def _extrema_1d(g):
    """Indices of the strict 1-D local minima and maxima of g (an end compares
    with its one neighbour)."""
    n = len(g)
    mins, maxs = set(), set()
    for i in range(n):
        lo = all(g[j] > g[i] for j in (i - 1, i + 1) if 0 <= j < n)
        hi = all(g[j] < g[i] for j in (i - 1, i + 1) if 0 <= j < n)
        if lo:
            mins.add(i)
        if hi:
            maxs.add(i)
    return mins, maxs


@pytest.mark.parametrize("seed", range(4))
def test_sin_product_closed_form(seed):
    """f = gz(z) gy(y) gx(x), each factor a sampled sine with a phase that
    keeps every sample away from 0. Along one axis only that axis's factor
    changes, multiplied by the product p of the other two: where p > 0 the
    vertex is a minimum along the axis iff its factor is a 1-D minimum, where
    p < 0 iff its factor is a 1-D maximum. So the local minima are exactly
    the (z, y, x) whose coordinates each lie in Min or Max of their axis, as
    the signs of the other two factors decide -- a closed form in the three
    1-D extrema lists -- and #pairs = #minima - 1. Float32 rounding of the
    product is monotone in each factor, and no two neighbours tie, so the
    comparisons of the field are those of the exact products."""
    rng = np.random.default_rng(100 + seed)
    sides = [int(x) for x in rng.integers(12, 30, size=3)]
    gs = []
    for m in sides:
        while True:
            w, ph = rng.uniform(0.3, 1.4), rng.uniform(0, 2 * np.pi)
            g = np.sin(w * np.arange(m) + ph)
            if np.abs(g).min() > 1e-2:
                break
        gs.append(g)
    gz, gy, gx = gs
    f = ((gz[:, None, None] * gy[None, :, None]) * gx[None, None, :]).astype(np.float32)
    for d in range(3):  # no ties between neighbours
        assert np.all(np.diff(f, axis=d) != 0)
    ext = [_extrema_1d(g) for g in gs]
    sign = [np.sign(g) for g in gs]
    want = set()
    for z in range(sides[0]):
        for y in range(sides[1]):
            for x in range(sides[2]):
                c = (z, y, x)
                ok = True
                for a in range(3):
                    p = sign[(a + 1) % 3][c[(a + 1) % 3]] * sign[(a + 2) % 3][c[(a + 2) % 3]]
                    mins, maxs = ext[a]
                    ok &= c[a] in (mins if p > 0 else maxs)
                if ok:
                    want.add(x + sides[2] * (y + sides[1] * z))
    # the same count from the 1-D lists alone, sign pattern by sign pattern
    count = 0
    for e in itertools.product((1, -1), repeat=3):
        prod = 1
        for a in range(3):
            mins, maxs = ext[a]
            pick = mins if e[(a + 1) % 3] * e[(a + 2) % 3] > 0 else maxs
            prod *= sum(1 for i in pick if sign[a][i] == e[a])
        count += prod
    assert count == len(want)
    W = oracle.merge_tree(f)
    u = np.arange(f.size, dtype=np.uint64)
    s, v = W >> np.uint64(32), W & np.uint64(0xFFFFFFFF)
    starts = set(np.nonzero((s != u) | ((s == u) & (v == u)))[0].tolist())
    assert starts == want
    p, roots = oracle.pairs(W)
    assert len(p) == count - 1 and len(roots) == 1


def test_openmp_baseline_equals_oracle():
    """The CPU baseline (the paper's parallel algorithm with OpenMP, lock-free
    merges racing on 4 and 8 threads) gives the oracle's unique triplets on
    grids with ties, signed zeros, plateaus and monotone ramps."""
    rng = np.random.default_rng(8)
    cases = []
    for i in range(40):
        shape = tuple(int(x) for x in rng.integers(1, 20, size=3))
        k = i % 4
        if k == 0:
            f = rng.random(shape, dtype=np.float32)
        elif k == 1:
            f = rng.integers(0, 5, size=shape).astype(np.float32)
        elif k == 2:
            f = rng.choice(np.array([-0.0, 0.0, -1.0, 3.0], np.float32), size=shape)
        else:
            f = rng.random(shape, dtype=np.float32)
            f[..., : shape[2] // 2] = 0.5
        cases.append(f)
    nz = ny = nx = 12
    cases.append(np.add.outer(np.add.outer(np.arange(nz), np.arange(ny)), np.arange(nx)).astype(np.float32))
    cases.append(fields_grf_like(rng))
    for f in cases:
        want = oracle.merge_tree(f)
        for threads in (4, 8):
            assert np.array_equal(oracle.tmt_openmp(f, threads), want), f.shape


def fields_grf_like(rng):
    from paper_2301_10838_gb300 import fields

    return fields.quantize(fields.grf((24, 20, 28), -3.0, int(rng.integers(0, 1000))), 128)
