"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Triplets, pairs and labels are integers, so the bar is bit-exact equality.
Sizes run from single vertices to several compaction chunks with ragged
tails; the 1024^3 workload is compared in full in test_gpu_full_size.py.
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


def run_path(f_np, t=None, cap=None, stream=None):
    f = torch.from_numpy(np.ascontiguousarray(f_np, dtype=np.float32)).cuda()
    n = f.numel()
    W = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(f))
    mt.mt_build_triplets(f, W, ws, stream=stream)
    pairs = torch.empty((n if cap is None else cap, 2), dtype=torch.int32, device="cuda")
    npairs, root = mt.mt_persistence_pairs(f, W, pairs, ws, stream=stream)
    out = {
        "W": W.cpu().numpy().view(np.uint64),
        "pairs": pairs[:npairs].cpu().numpy().view(np.uint32),
        "root": root,
    }
    if t is not None:
        labels = torch.empty(n, dtype=torch.int32, device="cuda")
        mt.mt_components_at(f, W, t, labels, ws, stream=stream)
        mt.mt_sync_status(ws, stream=stream)
        out["labels"] = labels.cpu().numpy().view(np.uint32)
    return out


def assert_parity(f_np, thresholds=()):
    W_ref = oracle.merge_tree(f_np)
    p_ref, roots = oracle.pairs(W_ref)
    got = run_path(f_np)
    bad = np.nonzero(got["W"] != W_ref)[0]
    assert bad.size == 0, f"{bad.size} triplets differ, first at {bad[:5]}: {got['W'][bad[:5]]} vs {W_ref[bad[:5]]}"
    assert np.array_equal(got["pairs"], p_ref)
    assert got["root"] == int(roots[0])
    f_dev = torch.from_numpy(np.ascontiguousarray(f_np, dtype=np.float32)).cuda()
    W_dev = torch.from_numpy(W_ref.view(np.int64)).cuda()
    ws = mt.workspace(mt.grid_of(f_dev))
    for t in thresholds:
        lab = torch.empty(f_np.size, dtype=torch.int32, device="cuda")
        mt.mt_components_at(f_dev, W_dev, float(t), lab, ws)
        mt.mt_sync_status(ws)
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), oracle.components(f_np, float(t)))


RAGGED = [(1, 1, 1), (1, 1, 2), (1, 1, 100), (1, 50, 3), (2, 2, 2), (5, 7, 9), (3, 1, 4), (17, 19, 23),
          (33, 31, 65), (8, 8, 4096 + 5), (40, 40, 40)]


@pytest.mark.parametrize("shape", RAGGED)
@pytest.mark.parametrize("kind", ["uniform", "ties", "zeros", "grf"])
def test_parity_small(shape, kind):
    seed = zlib.crc32(repr((shape, kind)).encode()) % 1000
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
    assert_parity(f, thresholds=(float(np.median(f)),))


def test_parity_constant_and_ramps():
    for shape in [(9, 10, 11), (1, 1, 5000), (64, 3, 2)]:
        nz, ny, nx = shape
        assert_parity(np.zeros(shape, np.float32))
        ramp = np.add.outer(np.add.outer(np.arange(nz), np.arange(ny)), np.arange(nx)).astype(np.float32)
        assert_parity(ramp)
        assert_parity(-ramp)


def test_parity_plateau_flood():
    """Half of the domain sits on one value that joins many basins at once
    (the sudden volume change of the paper's Richtmyer-Meshkov discussion)."""
    rng = np.random.default_rng(5)
    f = rng.random((30, 30, 30), dtype=np.float32)
    f[:, :, 15:] = 0.5
    assert_parity(f, thresholds=(0.49, 0.5, 0.51))


def test_parity_six_lower_components():
    """A vertex whose 6 neighbours lie in 6 different components below it."""
    f = np.full((3, 3, 3), 10.0, np.float32)
    c = (1, 1, 1)
    f[c] = 5.0
    for k, (dz, dy, dx) in enumerate([(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]):
        f[1 + dz, 1 + dy, 1 + dx] = float(k)
    assert_parity(f)


def test_parity_snake():
    """A long monotone path folded through the grid: deep descent chains."""
    nz, ny, nx = 4, 16, 32
    f = np.zeros((nz, ny, nx), np.float32)
    k = 0
    for z in range(nz):
        for y in range(ny):
            xs = range(nx) if (y + z) % 2 == 0 else range(nx - 1, -1, -1)
            for x in xs:
                f[z, y, x] = k
                k += 1
    assert_parity(f)
    assert_parity(-f)


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_parity_white64(seed):
    f = fields.named_field("white64", seed=seed)
    assert_parity(f, thresholds=(0.1, 0.5))


@pytest.mark.parametrize("seed", [1, 2])
def test_parity_grf256q12(seed):
    f = fields.named_field("grf256q12", seed=seed)
    assert_parity(f, thresholds=(0.3,))


def test_parity_lognormal_128():
    f = fields.named_field("lognorm1024", seed=1, side=128)
    assert_parity(f, thresholds=(1.0,))


def test_unaligned_field_pointer():
    """A field that is not 16-byte aligned takes the scalar stencil path."""
    f_np = fields.white_noise((10, 12, 16), seed=9)
    big = torch.from_numpy(np.concatenate([np.zeros(1, np.float32), f_np.ravel()])).cuda()
    f = big[1:].view(10, 12, 16)
    assert f.data_ptr() % 16 != 0
    W = torch.empty(f.numel(), dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(f))
    mt.mt_build_triplets(f, W, ws)
    mt.mt_sync_status(ws)
    assert np.array_equal(W.cpu().numpy().view(np.uint64), oracle.merge_tree(f_np))


def test_deterministic_repeat_and_stream():
    f = fields.named_field("white64", seed=7)
    a = run_path(f)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = run_path(f, stream=s)
    assert np.array_equal(a["W"], b["W"]) and np.array_equal(a["pairs"], b["pairs"])


def test_nonfinite_is_reported():
    f = fields.white_noise((8, 8, 8), seed=1)
    for bad in (np.nan, np.inf, -np.inf):
        g = f.copy()
        g[3, 4, 5] = bad
        with pytest.raises(mt.MtError) as e:
            run_path(g)
        assert e.value.code == -3
    # the workspace is usable again afterwards
    run_path(f)


def test_capacity_reports_true_count():
    f = fields.white_noise((16, 16, 16), seed=2)
    W_ref = oracle.merge_tree(f)
    p_ref, _ = oracle.pairs(W_ref)
    fd = torch.from_numpy(f).cuda()
    W = torch.empty(f.size, dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(fd))
    mt.mt_build_triplets(fd, W, ws)
    cap = 10
    pairs = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(mt.MtError) as e:
        mt.mt_persistence_pairs(fd, W, pairs, ws)
    assert e.value.code == -4
    npairs, root = mt.mt_persistence_pairs(fd, W, pairs, ws, allow_partial=True)
    assert npairs == len(p_ref)
    assert np.array_equal(pairs.cpu().numpy().view(np.uint32), p_ref[:cap])


def test_bad_arguments_on_device():
    f = torch.zeros((4, 4, 4), device="cuda")
    W = torch.empty(10, dtype=torch.int64, device="cuda")  # too short
    ws = mt.workspace(mt.grid_of(f))
    with pytest.raises(ValueError):
        mt.mt_build_triplets(f, W, ws)
    with pytest.raises(mt.MtError) as e:
        mt.mt_build_triplets(f, torch.empty(64, dtype=torch.int64, device="cuda"), ws[1:])
    assert e.value.code == -1


def test_corrupt_triplets_are_reported_not_followed():
    """Labels follow the caller's triplets: out-of-range ids and cycles are
    reported through the status word, without reads outside the arrays."""
    f = torch.from_numpy(fields.white_noise((10, 10, 10), 3)).cuda()
    n = f.numel()
    ws = mt.workspace(mt.grid_of(f))
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    # every vertex points at vertex 0 below it, and vertex 0 points at n + 5
    W = (torch.arange(n, dtype=torch.int64, device="cuda") << 32)
    W[0] = n + 5
    mt.mt_components_at(f, W, 2.0, lab, ws)
    with pytest.raises(mt.MtError) as e:
        mt.mt_sync_status(ws)
    assert e.value.code == -1
    # a two-cycle: 1 -> 2 -> 1 with saddles inside G_t
    W = torch.arange(n, dtype=torch.int64, device="cuda") * ((1 << 32) + 1)  # all roots
    W[1] = (1 << 32) | 2
    W[2] = (2 << 32) | 1
    mt.mt_components_at(f, W, 2.0, lab, ws)
    with pytest.raises(mt.MtError) as e:
        mt.mt_sync_status(ws)
    assert e.value.code == -7
    # the workspace stays usable
    W_ok = torch.from_numpy(oracle.merge_tree(f.cpu().numpy()).view(np.int64)).cuda()
    mt.mt_components_at(f, W_ok, 0.5, lab, ws)
    mt.mt_sync_status(ws)
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), oracle.components(f.cpu().numpy(), 0.5))
