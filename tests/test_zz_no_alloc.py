"""The allocation-free pairs entry point (mt_persistence_pairs_noalloc).

It serves callers that cannot allocate device memory for a workspace: its
scratch is an array compiled into libmt. The GPU test checks, through the C
ABI, that two calls in a row return exactly what mt_persistence_pairs
returns (pairs are integers, so the tolerance is zero). This file is named
so that pytest collects it after every other test file; it passes both alone
in a fresh process and after the rest of the suite.
"""

from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import paper_2301_10838_gb300 as mt
from paper_2301_10838_gb300 import fields


def test_noalloc_rejects_grids_above_its_limit():
    """n > 2^30 is refused on the host before any CUDA call (no GPU needed)."""
    lib = mt.load()
    npairs = ctypes.c_uint64(0)
    big = mt.Grid(2048, 1024, 1024)
    code = lib.mt_persistence_pairs_noalloc(ctypes.c_void_p(256), ctypes.c_void_p(256), big, ctypes.c_void_p(256),
                                            1, ctypes.byref(npairs), None, None)
    assert code == -2
    assert lib.mt_persistence_pairs_noalloc(None, None, mt.Grid(4, 4, 4), None, 0, None, None, None) == -1


@pytest.mark.gpu
def test_noalloc_pairs_match_workspace_pairs_twice():
    for shape, seed in (((40, 36, 52), 3), ((17, 64, 33), 4)):
        f = torch.from_numpy(fields.white_noise(shape, seed)).cuda()
        n = f.numel()
        W = torch.empty(n, dtype=torch.int64, device="cuda")
        ws = mt.workspace(mt.grid_of(f))
        mt.mt_build_triplets(f, W, ws)
        ref = torch.empty((n, 2), dtype=torch.int32, device="cuda")
        k_ref, root_ref = mt.mt_persistence_pairs(f, W, ref, ws)
        ref_np = ref[:k_ref].cpu().numpy()
        for _ in range(2):
            out = torch.full((n, 2), -1, dtype=torch.int32, device="cuda")
            k, root = mt.mt_persistence_pairs_noalloc(f, W, out)
            assert (k, root) == (k_ref, root_ref)
            assert np.array_equal(out[:k].cpu().numpy(), ref_np)


@pytest.mark.gpu
def test_noalloc_capacity_and_small_after_large():
    """The capacity path reports the true count, and a small grid right after
    a large one (whose per-chunk counts are still in the shared array) gets
    exactly the pairs mt_persistence_pairs gives."""
    outs = []
    for shape, seed in (((96, 96, 96), 5), ((9, 11, 13), 6)):
        f = torch.from_numpy(fields.white_noise(shape, seed)).cuda()
        n = f.numel()
        W = torch.empty(n, dtype=torch.int64, device="cuda")
        ws = mt.workspace(mt.grid_of(f))
        mt.mt_build_triplets(f, W, ws)
        ref = torch.empty((n, 2), dtype=torch.int32, device="cuda")
        k_ref, root_ref = mt.mt_persistence_pairs(f, W, ref, ws)
        out = torch.full((n, 2), -1, dtype=torch.int32, device="cuda")
        k, root = mt.mt_persistence_pairs_noalloc(f, W, out)
        assert (k, root) == (k_ref, root_ref)
        assert np.array_equal(out[:k].cpu().numpy(), ref[:k_ref].cpu().numpy())
        outs.append((f, W, ref[:k_ref].cpu().numpy(), k_ref))
    f, W, ref_np, k_ref = outs[0]
    cap = 10
    part = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(mt.MtError) as e:
        mt.mt_persistence_pairs_noalloc(f, W, part)
    assert e.value.code == -4
    k, _ = mt.mt_persistence_pairs_noalloc(f, W, part, allow_partial=True)
    assert k == k_ref
    assert np.array_equal(part.cpu().numpy(), ref_np[:cap])
    empty = torch.empty((0, 2), dtype=torch.int32, device="cuda")
    k, _ = mt.mt_persistence_pairs_noalloc(f, W, empty, allow_partial=True)
    assert k == k_ref
