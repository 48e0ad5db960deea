"""Branch decomposition on the GPU against the oracle (bit-exact)."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2301_10838_gb300 as mt
from paper_2301_10838_gb300 import fields

pytestmark = pytest.mark.gpu


def _field(case):
    rng = np.random.default_rng(17)
    if case == "white":
        return fields.white_noise((45, 38, 29), 2)
    if case == "ties":
        return rng.integers(0, 9, size=(31, 22, 35)).astype(np.float32)
    if case == "grf":
        return fields.quantize(fields.grf((64, 48, 40), -3.0, 7), 512)
    if case == "line":
        return fields.white_noise((1, 1, 5000), 3)
    return fields.named_field("lognorm1024", seed=5, side=128)


def _branches(f, flags=0, cap=None):
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    n = fd.numel()
    W = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(fd))
    mt.mt_build_triplets_ex(fd, W, ws, flags)
    mt.mt_sync_status(ws)
    bws = mt.branches_workspace(mt.grid_of(fd))
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    offsets = torch.empty(n + 1 if cap is None else cap, dtype=torch.int32, device="cuda")
    nb = mt.mt_branch_decomposition(fd, W, flags, order, offsets, bws)
    return W, order, offsets, nb


@pytest.mark.parametrize("case", ["white", "ties", "grf", "line", "lognorm"])
def test_branches_match_oracle(case):
    f = _field(case)
    W, order, offsets, nb = _branches(f)
    W_ref = oracle.merge_tree(f)
    assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref)
    o_ref, off_ref = oracle.branches(f, W_ref)
    assert nb == len(off_ref) - 1
    assert np.array_equal(order.cpu().numpy().view(np.uint32), o_ref)
    assert np.array_equal(offsets[:nb + 1].cpu().numpy().view(np.uint32), off_ref)


def test_split_tree_branches():
    f = _field("grf")
    W, order, offsets, nb = _branches(f, mt.MT_SUPERLEVEL)
    neg = -f
    o_ref, off_ref = oracle.branches(neg, oracle.merge_tree(neg))
    assert np.array_equal(order.cpu().numpy().view(np.uint32), o_ref)
    assert np.array_equal(offsets[:nb + 1].cpu().numpy().view(np.uint32), off_ref)


def test_offsets_capacity_reports_true_count():
    f = _field("white")
    with pytest.raises(mt.MtError) as e:
        _branches(f, cap=5)
    assert e.value.code == -4
