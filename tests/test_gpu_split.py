"""The split tree (MT_SUPERLEVEL): the merge tree of -f, which is what the
paper's experiments report (Section 4, "Setup"). The oracle of -f decides."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2301_10838_gb300 as mt
from paper_2301_10838_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["white", "ties", "grf", "lognorm"])
def test_split_tree_is_the_tree_of_minus_f(case):
    rng = np.random.default_rng(3)
    if case == "white":
        f = fields.white_noise((33, 20, 47), 5)
    elif case == "ties":
        f = rng.integers(0, 5, size=(17, 24, 40)).astype(np.float32)
        f[0, 0, :7] = -0.0  # signed zeros: -(+0) and -(-0) compare equal
    elif case == "grf":
        f = fields.quantize(fields.grf((40, 36, 32), -3.0, 4), 64)
    else:
        f = fields.named_field("lognorm1024", seed=2, side=64)
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    n = fd.numel()
    W = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(fd))
    mt.mt_build_triplets_ex(fd, W, ws, mt.MT_SUPERLEVEL)
    P = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    k, root = mt.mt_persistence_pairs(fd, W, P, ws)
    neg = -f
    W_ref = oracle.merge_tree(neg)
    p_ref, roots = oracle.pairs(W_ref)
    assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref)
    assert np.array_equal(P[:k].cpu().numpy().view(np.uint32), p_ref) and root == int(roots[0])
    t = float(np.median(f))
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    mt.mt_components_at_ex(fd, W, t, mt.MT_SUPERLEVEL, lab, ws)
    mt.mt_sync_status(ws)
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), oracle.components(neg, -t))


def test_plain_ex_equals_plain():
    f = fields.white_noise((20, 20, 20), 8)
    fd = torch.from_numpy(f).cuda()
    a = torch.empty(f.size, dtype=torch.int64, device="cuda")
    b = torch.empty(f.size, dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(fd))
    mt.mt_build_triplets(fd, a, ws)
    mt.mt_build_triplets_ex(fd, b, ws, 0)
    mt.mt_sync_status(ws)
    assert torch.equal(a, b)
    with pytest.raises(mt.MtError):
        mt.mt_build_triplets_ex(fd, b, ws, 4)
