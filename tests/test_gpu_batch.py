"""Batched build: every field of a packed batch gets exactly the triplets
and pairs the single-field calls give, for both tile variants, one-shot and
replayed from a CUDA graph."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2301_10838_gb300 as mt
from paper_2301_10838_gb300 import fields
from paper_2301_10838_gb300.batch import Batch

pytestmark = pytest.mark.gpu


def _single(f):
    fd = torch.as_tensor(f).cuda().contiguous()
    W = torch.empty(fd.numel(), dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(fd))
    mt.mt_build_triplets(fd, W, ws)
    p = torch.empty((fd.numel(), 2), dtype=torch.int32, device="cuda")
    k, _ = mt.mt_persistence_pairs(fd, W, p, ws)
    return W.cpu().numpy().view(np.uint64), p[:k].cpu().numpy().view(np.uint32)


def _make(count, seed):
    shapes = fields.batch_shapes(count, 5, 40, seed=seed)
    flds = [fields.batch_field(i if i % 2 == 0 else 300 + i, s) for i, s in enumerate(shapes)]
    return shapes, flds


@pytest.mark.parametrize("variant", [0, 1])
def test_batch_matches_single(variant):
    shapes, flds = _make(24, 3)
    b = Batch(shapes)
    b.load(flds)
    b.variant = variant
    b.launch()
    mt.mt_sync_status(b.ws)
    for i, f in enumerate(flds):
        W_ref, p_ref = _single(f)
        W, p = b.results(i)
        assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref), f"field {i} {shapes[i]}"
        assert np.array_equal(p.cpu().numpy().view(np.uint32), p_ref)
    # two fields against the oracle too
    for i in (0, 5):
        assert np.array_equal(b.results(i)[0].cpu().numpy().view(np.uint64), oracle.merge_tree(flds[i]))


def test_batch_graph_replay_and_autotune(tmp_path, monkeypatch):
    monkeypatch.setenv("MT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    shapes, flds = _make(16, 9)
    b = Batch(shapes)
    b.load(flds)
    v = b.tune()
    assert v in (0, 1)
    assert b.tune() == v  # now from the cache
    b.capture()
    for rep in range(2):
        b.W.zero_()
        b.launch()
        torch.cuda.synchronize()
        for i, f in enumerate(flds):
            W_ref, p_ref = _single(f)
            W, p = b.results(i)
            assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref)
            assert np.array_equal(p.cpu().numpy().view(np.uint32), p_ref)


def test_batch_oneshot_and_nonfinite():
    shapes, flds = _make(6, 4)
    flds[3] = flds[3].copy()
    flds[3].flat[7] = np.nan
    total = sum(int(np.prod(s)) for s in shapes)
    arena = torch.cat([torch.as_tensor(f).reshape(-1) for f in flds]).cuda()
    grids = [mt.Grid(s[2], s[1], s[0]) for s in shapes]
    W = torch.empty(total, dtype=torch.int64, device="cuda")
    P = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    npairs = torch.zeros(len(shapes), dtype=torch.int64, device="cuda")
    ws = torch.empty(mt.mt_batch_workspace_bytes(grids), dtype=torch.uint8, device="cuda")
    mt.mt_batch_build(arena, grids, W, P, npairs, ws)
    with pytest.raises(mt.MtError) as e:
        mt.mt_sync_status(ws)
    assert e.value.code == -3


@pytest.mark.slow
def test_batch_512_config_equals_oracle(tmp_path, monkeypatch):
    """The batch workload in the configuration the benchmark runs: 512 fields
    with sides log-uniform in [16, 128] per axis (half white noise, half GRF
    P(k)~k^-3), autotuned and replayed from a CUDA graph. Every field's
    triplets and pair list equal the oracle's."""
    monkeypatch.setenv("MT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    shapes = fields.batch_shapes(512, 16, 128, seed=7)
    flds = [fields.batch_field(i, s) for i, s in enumerate(shapes)]
    b = Batch(shapes)
    b.load(flds)
    b.tune()
    b.capture()
    b.W.zero_()
    b.launch()
    torch.cuda.synchronize()
    mt.mt_sync_status(b.ws)
    W_all = b.W.cpu().numpy().view(np.uint64)
    P_all = b.pairs.cpu().numpy().view(np.uint32)
    npairs = b.npairs.cpu().numpy()
    for i, f in enumerate(flds):
        a, e = b.offsets[i], b.offsets[i + 1]
        W_ref = oracle.merge_tree(f)
        assert np.array_equal(W_all[a:e], W_ref), f"field {i} {shapes[i]}: triplets differ"
        p_ref, _ = oracle.pairs(W_ref)
        assert int(npairs[i]) == len(p_ref), f"field {i}: pair count"
        assert np.array_equal(P_all[a:a + len(p_ref)], p_ref), f"field {i}: pairs differ"
