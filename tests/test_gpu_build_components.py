"""mt_build_components and mt_build_step against the oracle and the separate
calls (bit-exact).

The call builds the triplets and labels the components of G_t inside the
repair pass. Its triplets must equal mt_build_triplets_cfg's and the oracle's,
its labels those of the oracle's union-find over G_t (and, with eps > 0, the
oracle's simplified components), for ragged and tile-aligned grids, tied
values, thresholds at and beyond the extremes, the split tree, and every
single-field launch configuration."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2301_10838_gb300 as mt
from paper_2301_10838_gb300 import fields

pytestmark = pytest.mark.gpu

OUT = np.uint32(0xFFFFFFFF)


def _field(case):
    rng = np.random.default_rng(21)
    if case == "white":
        return fields.white_noise((37, 30, 45), 5)
    if case == "ties":
        return rng.integers(0, 6, size=(21, 34, 40)).astype(np.float32)
    if case == "grf":
        return fields.quantize(fields.grf((32, 32, 64), -3.0, 2), 256)
    if case == "lognorm":
        return fields.named_field("lognorm1024", seed=3, side=96)
    if case == "plane":
        return fields.white_noise((1, 70, 90), 8)
    if case == "line":
        return fields.white_noise((1, 1, 300), 9)
    raise KeyError(case)


def _fused(f_np, t, eps=0.0, flags=0, cfg=0):
    f = torch.from_numpy(np.ascontiguousarray(f_np, dtype=np.float32)).cuda()
    n = f.numel()
    W = torch.empty(n, dtype=torch.int64, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = mt.workspace(mt.grid_of(f))
    mt.mt_build_components(f, W, t, lab, ws, eps=eps, flags=flags, cfg=cfg)
    mt.mt_sync_status(ws)
    return W.cpu().numpy().view(np.uint64), lab.cpu().numpy().view(np.uint32)


def _thresholds(f):
    v = np.asarray(f, dtype=np.float32).ravel()
    qs = [float(np.quantile(v, q)) for q in (0.1, 0.5, 0.9)]
    return qs + [float(v.min()), float(v.max()), -np.inf, np.inf]


@pytest.mark.parametrize("case", ["white", "ties", "grf", "lognorm", "plane", "line"])
def test_triplets_and_labels_equal_oracle(case):
    f = _field(case)
    W_ref = oracle.merge_tree(f)
    for t in _thresholds(f):
        W, lab = _fused(f, t)
        assert np.array_equal(W, W_ref), (case, t)
        assert np.array_equal(lab, oracle.components(f, t)), (case, t)


@pytest.mark.parametrize("case", ["ties", "lognorm"])
def test_simplified_labels_equal_oracle(case):
    f = _field(case)
    W_ref = oracle.merge_tree(f)
    p, _ = oracle.pairs(W_ref)
    pers = np.sort(oracle.persistence(f, W_ref, p[:, 0]))
    for eps in (float(pers[len(pers) // 4]), float(pers[len(pers) // 2]), float(pers[-2]), np.inf):
        for q in (0.3, 0.7):
            t = float(np.quantile(f, q))
            W, lab = _fused(f, t, eps=eps)
            assert np.array_equal(W, W_ref)
            assert np.array_equal(lab, oracle.simplified_components(f, W_ref, t, eps)), (case, eps, q)


def test_split_tree_labels_equal_oracle():
    f = _field("grf")
    W_ref = oracle.merge_tree(-f)
    for q in (0.2, 0.5, 0.8):
        t = float(np.quantile(f, q))
        W, lab = _fused(f, t, flags=mt.MT_SUPERLEVEL)
        assert np.array_equal(W, W_ref)
        assert np.array_equal(lab, oracle.components(-f, -t)), q


@pytest.mark.parametrize("cfg", [0, 2, 4, 6, 8, 10, 12, 14])
def test_every_configuration(cfg):
    f = _field("lognorm")
    t = float(np.median(f))
    W, lab = _fused(f, t, cfg=cfg)
    assert np.array_equal(W, oracle.merge_tree(f))
    assert np.array_equal(lab, oracle.components(f, t))


@pytest.mark.parametrize("shape", [(256, 256, 256), (190, 203, 250)])
def test_equals_separate_calls(shape):
    """At sizes where the oracle is slow: the fused call against the separate
    build and labelling calls, whose parity tests run on the same fields."""
    g = fields.lognormal(shape, seed=5, sigma=0.8, slope=-2.0, device="cuda").contiguous()
    n = g.numel()
    ws = mt.workspace(mt.grid_of(g))
    W0 = torch.empty(n, dtype=torch.int64, device="cuda")
    W1 = torch.empty_like(W0)
    L0 = torch.empty(n, dtype=torch.int32, device="cuda")
    L1 = torch.empty_like(L0)
    for q in (0.25, 0.5, 0.75):
        t = float(torch.quantile(g.reshape(-1)[::97].float(), q))
        mt.mt_build_triplets(g, W0, ws)
        mt.mt_components_at(g, W0, t, L0, ws)
        mt.mt_build_components(g, W1, t, L1, ws)
        mt.mt_sync_status(ws)
        assert torch.equal(W0, W1), q
        assert torch.equal(L0, L1), q


def test_rejects_nan_and_bad_cfg():
    f = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    W = torch.empty(64, dtype=torch.int64, device="cuda")
    lab = torch.empty(64, dtype=torch.int32, device="cuda")
    ws = mt.workspace(mt.grid_of(f))
    with pytest.raises(mt.MtError):
        mt.mt_build_components(f, W, float("nan"), lab, ws)
    with pytest.raises(mt.MtError):
        mt.mt_build_components(f, W, 0.0, lab, ws, eps=float("nan"))
    with pytest.raises(mt.MtError):
        mt.mt_build_components(f, W, 0.0, lab, ws, cfg=mt.MT_CFG_SMALL_TILES)


def _step(f_np, t, eps=0.0, flags=0, cfg=0, cap=None):
    f = torch.from_numpy(np.ascontiguousarray(f_np, dtype=np.float32)).cuda()
    n = f.numel()
    W = torch.empty(n, dtype=torch.int64, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    P = torch.empty((n // 2 + 1 if cap is None else cap, 2), dtype=torch.int32, device="cuda")
    ws = mt.workspace(mt.grid_of(f))
    k, root = mt.mt_build_step(f, W, t, lab, P, ws, eps=eps, flags=flags, cfg=cfg, allow_partial=cap is not None)
    return (W.cpu().numpy().view(np.uint64), lab.cpu().numpy().view(np.uint32),
            P[:min(k, P.shape[0])].cpu().numpy().view(np.uint32), k, root)


@pytest.mark.parametrize("case", ["white", "ties", "grf", "lognorm", "plane", "line"])
def test_step_equals_oracle(case):
    """mt_build_step: triplets, labels, pairs (counted in the repair pass)
    and the root, against the oracle."""
    f = _field(case)
    W_ref = oracle.merge_tree(f)
    p_ref, roots = oracle.pairs(W_ref)
    for t in (float(np.median(f)), float(np.max(f))):
        W, lab, P, k, root = _step(f, t)
        assert np.array_equal(W, W_ref)
        assert np.array_equal(lab, oracle.components(f, t))
        assert k == len(p_ref) and root == int(roots[0])
        assert np.array_equal(P, p_ref)


@pytest.mark.parametrize("case", ["ties", "lognorm"])
def test_step_simplified_equals_oracle(case):
    f = _field(case)
    W_ref = oracle.merge_tree(f)
    p, _ = oracle.pairs(W_ref)
    eps = float(np.sort(oracle.persistence(f, W_ref, p[:, 0]))[len(p) // 2])
    t = float(np.quantile(f, 0.6))
    W, lab, P, k, _ = _step(f, t, eps=eps)
    ref = oracle.simplified_pairs(f, W_ref, eps)
    assert k == len(ref) and np.array_equal(P, ref)
    assert np.array_equal(lab, oracle.simplified_components(f, W_ref, t, eps))


def test_step_split_tree_and_capacity():
    f = _field("grf")
    W_ref = oracle.merge_tree(-f)
    p_ref, _ = oracle.pairs(W_ref)
    t = float(np.median(f))
    W, lab, P, k, _ = _step(f, t, flags=mt.MT_SUPERLEVEL)
    assert np.array_equal(W, W_ref) and np.array_equal(P, p_ref)
    assert np.array_equal(lab, oracle.components(-f, -t))
    cap = len(p_ref) // 3
    W, lab, P, k, _ = _step(f, t, flags=mt.MT_SUPERLEVEL, cap=cap)
    assert k == len(p_ref)  # the true count, with the first cap pairs written
    assert np.array_equal(P, p_ref[:cap])


def test_step_equals_separate_calls_large():
    g = fields.lognormal((200, 256, 250), seed=6, sigma=0.8, slope=-2.0, device="cuda").contiguous()
    n = g.numel()
    ws = mt.workspace(mt.grid_of(g))
    t = float(torch.quantile(g.reshape(-1)[::97].float(), 0.5))
    W0, W1 = torch.empty(n, dtype=torch.int64, device="cuda"), torch.empty(n, dtype=torch.int64, device="cuda")
    L0, L1 = torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda")
    P0, P1 = (torch.empty((n // 2, 2), dtype=torch.int32, device="cuda") for _ in range(2))
    mt.mt_build_triplets(g, W0, ws)
    k0, r0 = mt.mt_persistence_pairs(g, W0, P0, ws)
    mt.mt_components_at(g, W0, t, L0, ws)
    k1, r1 = mt.mt_build_step(g, W1, t, L1, P1, ws)
    assert (k0, r0) == (k1, r1)
    assert torch.equal(W0, W1) and torch.equal(L0, L1) and torch.equal(P0[:k0], P1[:k1])
