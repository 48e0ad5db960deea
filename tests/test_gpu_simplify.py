"""Persistence simplification on the GPU against the oracle (bit-exact).

mt_simplified_pairs keeps the pairs of float32 persistence >= eps;
mt_simplified_components_at labels G_t of the field whose branches of
persistence < eps are filled up to their saddles. The oracle's versions are
pinned in test_oracle_simplify.py against an explicit filling."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2301_10838_gb300 as mt
from paper_2301_10838_gb300 import fields

pytestmark = pytest.mark.gpu


def _field(case):
    rng = np.random.default_rng(9)
    if case == "white":
        return fields.white_noise((37, 30, 45), 3)
    if case == "ties":
        return rng.integers(0, 7, size=(24, 19, 40)).astype(np.float32)
    if case == "grf":
        return fields.quantize(fields.grf((48, 40, 36), -3.0, 6), 256)
    return fields.named_field("lognorm1024", seed=4, side=96)


def _run(f, flags=0):
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    n = fd.numel()
    W = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(fd))
    mt.mt_build_triplets_ex(fd, W, ws, flags)
    return fd, W, ws


@pytest.mark.parametrize("case", ["white", "ties", "grf", "lognorm"])
def test_simplified_pairs_and_labels(case):
    f = _field(case)
    fd, W, ws = _run(f)
    n = f.size
    W_ref = oracle.merge_tree(f)
    p_all, roots = oracle.pairs(W_ref)
    pers = np.sort(oracle.persistence(f, W_ref, p_all[:, 0]))
    # eps at quantiles of the persistence itself (so every cut keeps and drops some), plus the limits
    epss = [0.0, float(pers[len(pers) // 4]), float(pers[len(pers) // 2]), float(pers[-2]), np.inf]
    P = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    for eps in epss:
        k, root = mt.mt_simplified_pairs(fd, W, eps, 0, P, ws)
        ref = oracle.simplified_pairs(f, W_ref, eps)
        assert root == int(roots[0])
        assert k == len(ref) and np.array_equal(P[:k].cpu().numpy().view(np.uint32), ref), eps
        for q in (0.2, 0.5, 0.9):
            t = float(np.quantile(f, q))
            mt.mt_simplified_components_at(fd, W, t, eps, 0, lab, ws)
            mt.mt_sync_status(ws)
            assert np.array_equal(lab.cpu().numpy().view(np.uint32),
                                  oracle.simplified_components(f, W_ref, t, eps)), (eps, q)


def test_eps_zero_equals_plain_calls():
    f = _field("lognorm")
    fd, W, ws = _run(f)
    n = f.size
    P0 = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    P1 = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    k0, r0 = mt.mt_persistence_pairs(fd, W, P0, ws)
    k1, r1 = mt.mt_simplified_pairs(fd, W, 0.0, 0, P1, ws)
    assert (k0, r0) == (k1, r1) and torch.equal(P0[:k0], P1[:k1])
    t = float(np.median(f))
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    b = torch.empty(n, dtype=torch.int32, device="cuda")
    mt.mt_components_at(fd, W, t, a, ws)
    mt.mt_simplified_components_at(fd, W, t, -1.0, 0, b, ws)
    mt.mt_sync_status(ws)
    assert torch.equal(a, b)


def test_superlevel_simplification_is_that_of_minus_f():
    f = _field("grf")
    fd, W, ws = _run(f, mt.MT_SUPERLEVEL)
    n = f.size
    neg = -f
    W_ref = oracle.merge_tree(neg)
    p_all, _ = oracle.pairs(W_ref)
    eps = float(np.median(oracle.persistence(neg, W_ref, p_all[:, 0])))
    P = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    k, _ = mt.mt_simplified_pairs(fd, W, eps, mt.MT_SUPERLEVEL, P, ws)
    assert np.array_equal(P[:k].cpu().numpy().view(np.uint32), oracle.simplified_pairs(neg, W_ref, eps))
    t = float(np.median(f))
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    mt.mt_simplified_components_at(fd, W, t, eps, mt.MT_SUPERLEVEL, lab, ws)
    mt.mt_sync_status(ws)
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), oracle.simplified_components(neg, W_ref, -t, eps))


def test_nan_eps_is_rejected():
    f = _field("white")
    fd, W, ws = _run(f)
    P = torch.empty((f.size, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(mt.MtError):
        mt.mt_simplified_pairs(fd, W, float("nan"), 0, P, ws)
    lab = torch.empty(f.size, dtype=torch.int32, device="cuda")
    with pytest.raises(mt.MtError):
        mt.mt_simplified_components_at(fd, W, 0.5, float("nan"), 0, lab, ws)
