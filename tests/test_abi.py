"""The C-ABI library loads and exports every entry point include/*.h declares
(no compute calls: this runs without a GPU)."""

from __future__ import annotations

import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_2301_10838_gb300 as mt
from paper_2301_10838_gb300 import binding
from paper_2301_10838_gb300 import build as mtbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(mt_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    mtbuild.build()
    return mt.load()


def test_header_declares_the_path_entry_points():
    names = _declared()
    for need in ("mt_build_triplets", "mt_persistence_pairs", "mt_components_at", "mt_workspace_bytes"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", mtbuild.LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in _declared():
        assert getattr(lib, name) is not None


def test_binding_covers_the_header():
    assert set(binding.exported_symbols()) <= _declared()


def test_status_strings(lib):
    for code in range(-8, 1):
        s = mt.mt_status_str(code)
        assert s and s != "unknown status"


def test_workspace_query(lib):
    assert mt.mt_workspace_bytes(mt.Grid(0, 4, 4)) == 0
    assert mt.mt_workspace_bytes(mt.Grid(65536, 65536, 1)) == 0  # n = 2^32: too large
    a = mt.mt_workspace_bytes(mt.Grid(64, 64, 64))
    b = mt.mt_workspace_bytes(mt.Grid(1024, 1024, 1024))
    assert 0 < a <= b
    assert a % 256 == 0 and b % 256 == 0


def test_argument_errors_need_no_gpu(lib):
    """Argument checks return before touching the device."""
    g = mt.Grid(4, 4, 4)
    nbytes = lib.mt_workspace_bytes(g)
    assert lib.mt_build_triplets(None, g, None, None, nbytes, None) == -1
    assert lib.mt_build_triplets(ctypes.c_void_p(256), mt.Grid(0, 1, 1), ctypes.c_void_p(256),
                                 ctypes.c_void_p(256), nbytes, None) == -1
    assert lib.mt_build_triplets(ctypes.c_void_p(256), mt.Grid(65536, 65536, 1), ctypes.c_void_p(256),
                                 ctypes.c_void_p(256), nbytes, None) == -2
    # misaligned workspace / short workspace
    assert lib.mt_build_triplets(ctypes.c_void_p(256), g, ctypes.c_void_p(256), ctypes.c_void_p(260),
                                 nbytes, None) == -1
    assert lib.mt_build_triplets(ctypes.c_void_p(256), g, ctypes.c_void_p(256), ctypes.c_void_p(256),
                                 nbytes - 1, None) == -1
    assert lib.mt_components_at(ctypes.c_void_p(256), ctypes.c_void_p(256), g, float("nan"),
                                ctypes.c_void_p(256), ctypes.c_void_p(256), nbytes, None) == -1
    npairs = ctypes.c_uint64(0)
    assert lib.mt_persistence_pairs(ctypes.c_void_p(256), ctypes.c_void_p(256), g, None, 0, None, None,
                                    ctypes.c_void_p(256), nbytes, None) == -1


def test_simplification_and_branch_argument_errors_need_no_gpu(lib):
    """The simplification and branch-decomposition calls reject bad arguments
    (NaN thresholds, null outputs, bad flags, short workspaces) before any
    device work."""
    g = mt.Grid(4, 4, 4)
    nbytes = lib.mt_workspace_bytes(g)
    P = ctypes.c_void_p(256)
    npairs = ctypes.c_uint64(0)
    nan = float("nan")
    assert lib.mt_simplified_pairs(P, P, g, nan, 0, P, 8, ctypes.byref(npairs), None, P, nbytes, None) == -1
    assert lib.mt_simplified_pairs(P, P, g, 0.5, 4, P, 8, ctypes.byref(npairs), None, P, nbytes, None) == -1
    assert lib.mt_simplified_pairs(P, P, g, 0.5, 0, P, 8, None, None, P, nbytes, None) == -1
    assert lib.mt_simplified_components_at(P, P, g, nan, 0.1, 0, P, P, nbytes, None) == -1
    assert lib.mt_simplified_components_at(P, P, g, 0.5, nan, 0, P, P, nbytes, None) == -1
    assert lib.mt_simplified_components_at(P, P, g, 0.5, 0.1, 0, None, P, nbytes, None) == -1
    bbytes = lib.mt_branches_workspace_bytes(g)
    assert bbytes > 0 and bbytes % 256 == 0
    big = lib.mt_branches_workspace_bytes(mt.Grid(1024, 1024, 1024))
    assert big >= 20 * 1024 ** 3  # two 64-bit key arrays and one 32-bit value array per vertex
    assert lib.mt_branches_workspace_bytes(mt.Grid(0, 1, 1)) == 0
    assert lib.mt_branches_workspace_bytes(mt.Grid(65536, 65536, 1)) == 0
    nb = ctypes.c_uint64(0)
    assert lib.mt_branch_decomposition(P, P, g, 0, P, P, 65, ctypes.byref(nb), P, bbytes - 1, None) == -1
    assert lib.mt_branch_decomposition(P, P, g, 0, None, P, 65, ctypes.byref(nb), P, bbytes, None) == -1
    assert lib.mt_branch_decomposition(P, P, g, 2, P, P, 65, ctypes.byref(nb), P, bbytes, None) == -1
    assert lib.mt_branch_decomposition(P, P, mt.Grid(65536, 65536, 1), 0, P, P, 65, ctypes.byref(nb), P, bbytes,
                                       None) == -2


def test_launch_configurations_need_no_gpu(lib):
    """A single field takes the even configurations 0 .. 14 (level buckets,
    repair CTA size, tile shape); the batch-only small-tile bit and unknown
    bits are rejected before any device work, and the workspace holds the
    face buffers of both tile shapes a single field can use."""
    P = ctypes.c_void_p(256)
    for cfg in (mt.MT_CFG_SMALL_TILES, 16, 0x80000000, mt.MT_CFG_SMALL_TILES | mt.MT_CFG_LARGE_TILES):
        g = mt.Grid(4, 4, 4)
        nbytes = lib.mt_workspace_bytes(g)
        assert lib.mt_build_triplets_cfg(P, g, P, P, nbytes, 0, cfg, None) == -1, cfg
    assert mt.MT_CFG_SINGLE_MASK == mt.MT_CFG_FOUR_ROUNDS | mt.MT_CFG_REPAIR_256 | mt.MT_CFG_LARGE_TILES
    assert not mt.MT_CFG_SINGLE_MASK & mt.MT_CFG_SMALL_TILES

    def faces(shape, tile):
        nt = 1
        for a, b in zip(shape, tile):
            nt *= -(-a // b)
        tx, ty, tz = tile
        return nt * 2 * (ty * tz + tx * tz + tx * ty) * 4  # u32 per tile: both sides of three faces

    for shape in ((1024, 1024, 1024), (33, 16, 16), (17, 17, 17), (40, 3, 300), (1, 1, 1)):
        nx, ny, nz = shape
        n = nx * ny * nz
        chunks = -(-n // 4096)
        need = 512 + max(faces(shape, (16, 16, 16)), faces(shape, (32, 16, 16)))
        got = lib.mt_workspace_bytes(mt.Grid(nx, ny, nz))
        assert got >= need + 4 * chunks, (shape, got, need)


def test_library_is_sm103a_only():
    """The build passes exactly one -gencode, for sm_103a."""
    assert mtbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
