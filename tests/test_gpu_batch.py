"""Batched build: every field of a packed batch gets exactly the triplets
and pairs the single-field calls give, for every launch configuration,
one-shot and replayed from a CUDA graph; the single-field configurations
give the oracle's triplets too."""

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


@pytest.mark.parametrize("cfg", range(mt.MT_CFG_COUNT))
def test_batch_matches_single(cfg):
    shapes, flds = _make(24, 3)
    b = Batch(shapes)
    b.load(flds)
    b.cfg = cfg
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
    assert 0 <= v < mt.MT_CFG_COUNT and len(b.tuned_ms) == mt.MT_CFG_COUNT
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


def test_single_field_configurations_equal_oracle(tmp_path, monkeypatch):
    """mt_build_triplets_cfg: every single-field configuration (level buckets,
    repair CTA size, tile shape) gives the oracle's triplets, on a full-tile grid and on
    ragged ones; the single-field tuner picks one and caches it."""
    monkeypatch.setenv("MT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2301_10838_gb300 import autotune

    for shape, seed in (((32, 32, 64), 1), ((19, 37, 45), 2), ((1, 3, 200), 3)):
        f_np = fields.grf(shape, -3.0, seed).astype(np.float32) if min(shape) > 1 else \
            fields.white_noise(shape, seed)
        f_np = fields.quantize(f_np, 256)
        W_ref = oracle.merge_tree(f_np)
        f = torch.from_numpy(f_np).cuda()
        W = torch.empty(f.numel(), dtype=torch.int64, device="cuda")
        ws = mt.workspace(mt.grid_of(f))
        for cfg in range(0, mt.MT_CFG_SINGLE_MASK + 1, 2):
            W.zero_()
            mt.mt_build_triplets_cfg(f, W, ws, 0, cfg)
            mt.mt_sync_status(ws)
            assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref), (shape, cfg)
        cfg, ms = autotune.tune_single(f, W, ws)
        assert cfg in ms and len(ms) == 8
        assert autotune.tune_single(f, W, ws) == (cfg, None)  # from the cache
    with pytest.raises(mt.MtError):
        mt.mt_build_triplets_cfg(f, W, ws, 0, mt.MT_CFG_SMALL_TILES)
