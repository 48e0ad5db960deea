"""Parity cases run against a libmt stress build (MT_LIBRARY names it).

Run by test_gpu_stress_tables.py in a child process: the library is loaded
from MT_LIBRARY, and every case compares the CUDA path with the oracle bit
for bit. With the stress build's tables (one probe in the tile kernel's edge
hash; 16 target slots, 8 chain copies and a 32-entry minima list per
repair tile; 64 chain starts per label brick) the fields below
overflow every table, so the paths for a full table -- merge in place,
repair a branch minimum from the overflow bitmap, chase a target or a chain start along
the global chain -- carry most of the work.
"""

from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import paper_2301_10838_gb300 as mt  # noqa: E402
from paper_2301_10838_gb300 import fields  # noqa: E402
from paper_2301_10838_gb300.batch import Batch  # noqa: E402


def check_single(f_np, t):
    f = torch.from_numpy(np.ascontiguousarray(f_np, dtype=np.float32)).cuda()
    n = f.numel()
    W = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = mt.workspace(mt.grid_of(f))
    mt.mt_build_triplets(f, W, ws)
    pairs = torch.empty((n // 2 + 1, 2), dtype=torch.int32, device="cuda")
    k, root = mt.mt_persistence_pairs(f, W, pairs, ws)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    mt.mt_components_at(f, W, t, lab, ws)
    mt.mt_sync_status(ws)
    W_ref = oracle.merge_tree(f_np)
    p_ref, roots = oracle.pairs(W_ref)
    assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref), f"triplets {f_np.shape}"
    assert k == len(p_ref) and root == int(roots[0])
    assert np.array_equal(pairs[:k].cpu().numpy().view(np.uint32), p_ref), f"pairs {f_np.shape}"
    lab_ref = oracle.components(f_np, t)
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), lab_ref), f"labels {f_np.shape}"
    # the labels taken inside the repair pass (its full-table paths included)
    mt.mt_build_components(f, W, t, lab, ws)
    mt.mt_sync_status(ws)
    assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref), f"fused triplets {f_np.shape}"
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), lab_ref), f"fused labels {f_np.shape}"
    pairs.zero_()
    k2, root2 = mt.mt_build_step(f, W, t, lab, pairs, ws)
    assert (k2, root2) == (k, root) and np.array_equal(pairs[:k].cpu().numpy().view(np.uint32), p_ref)
    assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref), f"step triplets {f_np.shape}"
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), lab_ref), f"step labels {f_np.shape}"


def check_wide(f_np, t):
    f = torch.from_numpy(np.ascontiguousarray(f_np, dtype=np.float32)).cuda()
    n = f.numel()
    g = mt.grid_of(f)
    W2 = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    ws = mt.wide_workspace(g)
    mt.mt_build_triplets_wide(f, W2, ws)
    lab = torch.empty(n, dtype=torch.int64, device="cuda")
    mt.mt_components_at_wide(f, W2, t, 0, lab, ws)
    mt.mt_sync_status(ws)
    assert np.array_equal(W2.cpu().numpy().view(np.uint64), oracle.merge_tree_wide(f_np)), "wide triplets"
    assert np.array_equal(lab.cpu().numpy().view(np.uint64), oracle.components_wide(f_np, t)), "wide labels"


def check_batch():
    shapes = fields.batch_shapes(24, 16, 80, seed=5)
    flds = [fields.batch_field(i if i % 2 == 0 else 300 + i, s) for i, s in enumerate(shapes)]
    for cfg in (0, mt.MT_CFG_SMALL_TILES):
        b = Batch(shapes)
        b.load(flds)
        b.cfg = cfg
        b.launch()
        mt.mt_sync_status(b.ws)
        for i, f in enumerate(flds):
            W, p = b.results(i)
            W_ref = oracle.merge_tree(f)
            assert np.array_equal(W.cpu().numpy().view(np.uint64), W_ref), f"batch field {i} cfg {cfg}"
            assert np.array_equal(p.cpu().numpy().view(np.uint32), oracle.pairs(W_ref)[0])


def main():
    lib = os.environ.get("MT_LIBRARY", "")
    assert lib and os.path.samefile(mt.load()._name, lib), "the stress build is not the library loaded"
    for seed in (1, 2):
        f = fields.named_field("white64", seed=seed)
        check_single(f, 0.3)
    f = fields.named_field("grf256q12", seed=1)
    check_single(f, 0.5)
    f = fields.named_field("lognorm1024", seed=1, side=128)
    check_single(f, float(np.median(f)))
    rng = np.random.default_rng(3)
    for shape in ((33, 31, 65), (17, 19, 23), (8, 8, 4101)):
        f = rng.integers(0, 8, size=shape).astype(np.float32)
        check_single(f, 3.0)
    check_batch()
    check_wide(fields.named_field("white64", seed=3), 0.4)
    check_wide(fields.quantize(fields.grf((40, 48, 64), -3.0, 8), 64), 0.5)
    print("stress build: all cases equal the oracle")


if __name__ == "__main__":
    main()
