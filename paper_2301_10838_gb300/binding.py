"""Thin ctypes binding of libmt (include/mt.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it checks tensor placement, dtypes and sizes,
passes raw device pointers and the current CUDA stream, and turns a non-OK
status into ``MtError``. Every step of the path runs in libmt's kernels;
there is no CPU fallback — if libmt.so is missing the call raises.

Tensors: the field is float32 (nz, ny, nx) on a CUDA device; triplets are
int64 (bit pattern of uint64 (s << 32) | v); pairs and labels are int32
tensors holding uint32 bit patterns (view them with ``.view(torch.uint32)``
or ``numpy().view(np.uint32)``).
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

__all__ = [
    "MtError",
    "Grid",
    "load",
    "grid_of",
    "mt_status_str",
    "mt_workspace_bytes",
    "mt_build_triplets",
    "mt_persistence_pairs",
    "mt_components_at",
    "mt_sync_status",
    "MT_SUPERLEVEL",
    "mt_build_triplets_ex",
    "mt_build_triplets_cfg",
    "mt_build_autotune",
    "mt_build_components",
    "mt_build_step",
    "MT_CFG_SMALL_TILES",
    "MT_CFG_FOUR_ROUNDS",
    "MT_CFG_REPAIR_256",
    "MT_CFG_LARGE_TILES",
    "MT_CFG_COUNT",
    "MT_CFG_SINGLE_MASK",
    "mt_components_at_ex",
    "mt_persistence_pairs_noalloc",
    "mt_wide_workspace_bytes",
    "wide_workspace",
    "mt_build_triplets_wide",
    "mt_persistence_pairs_wide",
    "mt_components_at_wide",
    "mt_simplified_pairs",
    "mt_simplified_components_at",
    "mt_branches_workspace_bytes",
    "mt_branch_decomposition",
    "branches_workspace",
    "BatchPlan",
    "mt_batch_workspace_bytes",
    "mt_batch_prepare",
    "mt_batch_launch",
    "mt_batch_build",
    "mt_batch_autotune",
    "MtResult",
    "mt_server_create",
    "mt_server_submit",
    "mt_server_submit_resident",
    "mt_server_evict",
    "mt_server_resident",
    "mt_server_poll",
    "mt_server_wait",
    "mt_server_destroy",
    "mt_trace_enable",
    "mt_trace_read",
    "mt_kernel_launches",
    "workspace",
]

MT_OK = 0
MT_SUPERLEVEL = 1  # flag of the _ex calls: the tree of -f (superlevel sets, the split tree)
# launch configurations (bits; every one gives the same results)
MT_CFG_SMALL_TILES = 1  # 16x16x8 tiles of 256 threads (batches only)
MT_CFG_FOUR_ROUNDS = 2  # 4 level buckets (merge/repair rounds) per tile instead of 8
MT_CFG_REPAIR_256 = 4   # repair CTAs of 256 threads instead of 512
MT_CFG_LARGE_TILES = 8  # 32x16x16 tiles of 1024 threads (single fields only)
MT_CFG_COUNT = 8        # batch configurations 0 .. 7
MT_CFG_SINGLE_MASK = MT_CFG_FOUR_ROUNDS | MT_CFG_REPAIR_256 | MT_CFG_LARGE_TILES
STATUS_NAMES = {0: "MT_OK", -1: "MT_ERR_INVALID", -2: "MT_ERR_TOO_LARGE", -3: "MT_ERR_NONFINITE",
                -4: "MT_ERR_CAPACITY", -5: "MT_ERR_CUDA", -6: "MT_ERR_NOMEM", -7: "MT_ERR_TIMEOUT",
                -8: "MT_ERR_BUSY"}


class MtError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = int(code)
        name = STATUS_NAMES.get(self.code, str(code))
        super().__init__(f"{where}: {name} ({mt_status_str(code)}){detail}")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_uint32), ("ny", ctypes.c_uint32), ("nz", ctypes.c_uint32)]


class MtResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("npairs", ctypes.c_uint64), ("root", ctypes.c_uint32),
                ("reused", ctypes.c_uint32), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class BatchPlan(ctypes.Structure):
    _fields_ = [("nfields", ctypes.c_uint32), ("tiles", ctypes.c_uint32 * 2), ("chunks", ctypes.c_uint64),
                ("vertices", ctypes.c_uint64), ("ws_bytes", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_SIGS = {
    "mt_status_str": ([ctypes.c_int32], ctypes.c_char_p),
    "mt_workspace_bytes": ([Grid], ctypes.c_size_t),
    "mt_build_triplets": ([_P, Grid, _P, _P, ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_persistence_pairs": ([_P, _P, Grid, _P, _U64, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_components_at": ([_P, _P, Grid, ctypes.c_float, _P, _P, ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_sync_status": ([_P, _P], ctypes.c_int32),
    "mt_build_triplets_ex": ([_P, Grid, _P, _P, ctypes.c_size_t, ctypes.c_uint32, _P], ctypes.c_int32),
    "mt_build_triplets_cfg": ([_P, Grid, _P, _P, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint32, _P],
                              ctypes.c_int32),
    "mt_build_autotune": ([_P, Grid, _P, _P, ctypes.c_size_t, ctypes.c_uint32, _P, _P, _P], ctypes.c_int32),
    "mt_build_components": ([_P, Grid, _P, ctypes.c_float, ctypes.c_float, ctypes.c_uint32, ctypes.c_uint32, _P, _P,
                             ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_build_step": ([_P, Grid, _P, ctypes.c_float, ctypes.c_float, ctypes.c_uint32, ctypes.c_uint32, _P, _P, _U64,
                       _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_components_at_ex": ([_P, _P, Grid, ctypes.c_float, ctypes.c_uint32, _P, _P, ctypes.c_size_t, _P],
                            ctypes.c_int32),
    "mt_persistence_pairs_noalloc": ([_P, _P, Grid, _P, _U64, _P, _P, _P], ctypes.c_int32),
    "mt_wide_workspace_bytes": ([Grid], ctypes.c_size_t),
    "mt_build_triplets_wide": ([_P, Grid, _P, _P, ctypes.c_size_t, ctypes.c_uint32, _P], ctypes.c_int32),
    "mt_persistence_pairs_wide": ([_P, Grid, _P, _U64, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_components_at_wide": ([_P, _P, Grid, ctypes.c_float, ctypes.c_uint32, _P, _P, ctypes.c_size_t, _P],
                              ctypes.c_int32),
    "mt_simplified_pairs": ([_P, _P, Grid, ctypes.c_float, ctypes.c_uint32, _P, _U64, _P, _P, _P, ctypes.c_size_t, _P],
                            ctypes.c_int32),
    "mt_simplified_components_at": ([_P, _P, Grid, ctypes.c_float, ctypes.c_float, ctypes.c_uint32, _P, _P,
                                     ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_branches_workspace_bytes": ([Grid], ctypes.c_size_t),
    "mt_branch_decomposition": ([_P, _P, Grid, ctypes.c_uint32, _P, _P, _U64, _P, _P, ctypes.c_size_t, _P],
                                ctypes.c_int32),
    "mt_batch_workspace_bytes": ([_P, ctypes.c_uint32], ctypes.c_size_t),
    "mt_batch_prepare": ([_P, _P, ctypes.c_uint32, _P, _P, _P, ctypes.c_size_t, _P, _P], ctypes.c_int32),
    "mt_batch_launch": ([_P, ctypes.c_int, _P, _P, ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_batch_build": ([_P, _P, ctypes.c_uint32, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int32),
    "mt_batch_autotune": ([_P, _P, _P, ctypes.c_size_t, _P, _P, _P], ctypes.c_int32),
    "mt_server_create": ([ctypes.c_size_t, ctypes.c_int, ctypes.c_int], _P),
    "mt_server_submit": ([_P, _P, Grid, ctypes.c_float, _P, _U64, _P, _P], ctypes.c_int32),
    "mt_server_submit_resident": ([_P, _U64, _P, Grid, ctypes.c_float, _P, _U64, _P, _P], ctypes.c_int32),
    "mt_server_evict": ([_P, _U64], ctypes.c_int32),
    "mt_server_resident": ([_P, _P, _P], ctypes.c_int32),
    "mt_server_poll": ([_P, _U64, _P], ctypes.c_int32),
    "mt_server_wait": ([_P, _U64, _P], ctypes.c_int32),
    "mt_server_destroy": ([_P], None),
    "mt_trace_enable": ([ctypes.c_int], None),
    "mt_trace_read": ([_P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "mt_kernel_launches": ([], ctypes.c_ulonglong),
}


def load() -> ctypes.CDLL:
    """Load libmt.so (built in-tree by ``paper_2301_10838_gb300.build``), or
    the library the MT_LIBRARY environment variable names (another in-tree
    build of the same sources, such as the tests' stress build)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("MT_LIBRARY") or _build.LIB
            if not os.path.exists(path):
                raise ImportError(f"libmt is not built ({path}); run "
                                  "`python -m paper_2301_10838_gb300.build` on a machine with nvcc")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def mt_status_str(code: int) -> str:
    try:
        return load().mt_status_str(int(code)).decode()
    except ImportError:
        return STATUS_NAMES.get(int(code), "?")


def grid_of(f: torch.Tensor) -> Grid:
    if f.dim() != 3:
        raise ValueError("field must be 3-D (nz, ny, nx)")
    nz, ny, nx = (int(s) for s in f.shape)
    return Grid(nx, ny, nz)


def _stream_ptr(stream) -> int:
    """The cudaStream_t of ``stream`` (a torch stream, a raw handle, or None
    for the current stream). A torch stream must belong to the current
    device: libmt launches on the current device."""
    if stream is None:
        stream = torch.cuda.current_stream()
    if hasattr(stream, "cuda_stream"):
        dev = getattr(stream, "device", None)
        if dev is not None and dev.index is not None and dev.index != torch.cuda.current_device():
            raise ValueError(f"stream is on {dev}, but the current device is cuda:{torch.cuda.current_device()}")
        return int(stream.cuda_stream)
    return int(stream)


def _dev(t: torch.Tensor, name: str, dtypes, numel=None) -> int:
    """Device pointer of ``t`` after checking placement, dtype, layout and
    size. The tensor must live on the current CUDA device: libmt launches
    there (and the allocation-free call takes its scratch from it), so a
    tensor on another GPU would be reached through peer addressing."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, but the current device is cuda:{torch.cuda.current_device()}; "
                         "call under torch.cuda.device(...) of the tensors' device")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} must have dtype in {dtypes}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements, has {t.numel()}")
    return t.data_ptr()


def _check(code: int, where: str, detail: str = ""):
    if code != MT_OK:
        raise MtError(code, where, detail)


_I64 = (torch.int64, getattr(torch, "uint64", torch.int64))
_I32 = (torch.int32, getattr(torch, "uint32", torch.int32))


def mt_workspace_bytes(grid: Grid) -> int:
    return int(load().mt_workspace_bytes(grid))


def workspace(grid: Grid, device=None) -> torch.Tensor:
    """A device byte tensor big enough for ``grid`` (torch allocations are
    256-byte aligned) with its status word cleared."""
    nbytes = mt_workspace_bytes(grid)
    if nbytes == 0:
        raise MtError(-1, "mt_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
    ws[:256].zero_()
    return ws


def mt_build_triplets(f: torch.Tensor, W: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    g = grid_of(f)
    n = f.numel()
    pf = _dev(f, "f", (torch.float32,))
    pW = _dev(W, "W", _I64, n)
    pws = _dev(ws, "ws", (torch.uint8,))
    _check(load().mt_build_triplets(pf, g, pW, pws, ws.numel(), _stream_ptr(stream)), "mt_build_triplets")


def mt_build_triplets_ex(f: torch.Tensor, W: torch.Tensor, ws: torch.Tensor, flags: int, stream=None) -> None:
    """mt_build_triplets with flags (MT_SUPERLEVEL: the split tree, i.e. the
    merge tree of -f)."""
    g = grid_of(f)
    n = f.numel()
    _check(load().mt_build_triplets_ex(_dev(f, "f", (torch.float32,)), g, _dev(W, "W", _I64, n),
                                       _dev(ws, "ws", (torch.uint8,)), ws.numel(), int(flags), _stream_ptr(stream)),
           "mt_build_triplets_ex")


def mt_build_triplets_cfg(f: torch.Tensor, W: torch.Tensor, ws: torch.Tensor, flags: int, cfg: int,
                          stream=None) -> None:
    """mt_build_triplets_ex with a launch configuration (MT_CFG_FOUR_ROUNDS,
    MT_CFG_REPAIR_256, MT_CFG_LARGE_TILES bits); the triplets do not depend
    on it."""
    g = grid_of(f)
    n = f.numel()
    _check(load().mt_build_triplets_cfg(_dev(f, "f", (torch.float32,)), g, _dev(W, "W", _I64, n),
                                        _dev(ws, "ws", (torch.uint8,)), ws.numel(), int(flags), int(cfg),
                                        _stream_ptr(stream)), "mt_build_triplets_cfg")


def mt_build_autotune(f: torch.Tensor, W: torch.Tensor, ws: torch.Tensor, flags: int = 0, stream=None):
    """Times the single-field configurations (cfg 0, 2, .., 14); returns
    ({cfg: best ms}, best cfg). W receives the triplets."""
    g = grid_of(f)
    n = f.numel()
    ms = (ctypes.c_float * 8)()
    best = ctypes.c_uint32(0)
    _check(load().mt_build_autotune(_dev(f, "f", (torch.float32,)), g, _dev(W, "W", _I64, n),
                                    _dev(ws, "ws", (torch.uint8,)), ws.numel(), int(flags), _stream_ptr(stream),
                                    ctypes.cast(ms, ctypes.c_void_p), ctypes.byref(best)), "mt_build_autotune")
    return {2 * i: float(ms[i]) for i in range(8)}, int(best.value)


def mt_build_components(f: torch.Tensor, W: torch.Tensor, t: float, labels: torch.Tensor, ws: torch.Tensor,
                        eps: float = 0.0, flags: int = 0, cfg: int = 0, stream=None) -> None:
    """One build that also labels G_t: the triplets of mt_build_triplets_cfg
    and the labels of mt_simplified_components_at (eps <= 0: those of
    mt_components_at_ex), the labels taken inside the repair pass."""
    g = grid_of(f)
    n = f.numel()
    _check(load().mt_build_components(_dev(f, "f", (torch.float32,)), g, _dev(W, "W", _I64, n), float(t), float(eps),
                                      int(flags), int(cfg), _dev(labels, "labels", _I32, n),
                                      _dev(ws, "ws", (torch.uint8,)), ws.numel(), _stream_ptr(stream)),
           "mt_build_components")


def mt_build_step(f: torch.Tensor, W: torch.Tensor, t: float, labels: torch.Tensor, pairs: torch.Tensor,
                  ws: torch.Tensor, eps: float = 0.0, flags: int = 0, cfg: int = 0, stream=None,
                  allow_partial: bool = False) -> tuple[int, int]:
    """The whole path in one call: triplets, labels of G_t and the pairs
    (mt_build_components + mt_simplified_pairs / mt_persistence_pairs);
    returns (npairs, root). Synchronises the stream."""
    g = grid_of(f)
    n = f.numel()
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape (cap, 2)")
    cap = int(pairs.shape[0])
    pp = _dev(pairs, "pairs", _I32) if cap else 0
    npairs = ctypes.c_uint64(0)
    root = ctypes.c_uint32(0xFFFFFFFF)
    code = load().mt_build_step(_dev(f, "f", (torch.float32,)), g, _dev(W, "W", _I64, n), float(t), float(eps),
                                int(flags), int(cfg), _dev(labels, "labels", _I32, n), pp, cap, ctypes.byref(npairs),
                                ctypes.byref(root), _dev(ws, "ws", (torch.uint8,)), ws.numel(), _stream_ptr(stream))
    if code == -4 and allow_partial:
        return int(npairs.value), int(root.value)
    _check(code, "mt_build_step", f" npairs={npairs.value} cap={cap}")
    return int(npairs.value), int(root.value)


def mt_components_at_ex(f: torch.Tensor, W: torch.Tensor, t: float, flags: int, labels: torch.Tensor,
                        ws: torch.Tensor, stream=None) -> None:
    """mt_components_at with flags (MT_SUPERLEVEL: components of f >= t)."""
    g = grid_of(f)
    n = f.numel()
    _check(load().mt_components_at_ex(_dev(f, "f", (torch.float32,)), _dev(W, "W", _I64, n), g, float(t),
                                      int(flags), _dev(labels, "labels", _I32, n), _dev(ws, "ws", (torch.uint8,)),
                                      ws.numel(), _stream_ptr(stream)), "mt_components_at_ex")


def mt_persistence_pairs(f: torch.Tensor, W: torch.Tensor, pairs: torch.Tensor, ws: torch.Tensor,
                         stream=None, allow_partial: bool = False) -> tuple[int, int]:
    """Writes (minimum, saddle) rows into ``pairs`` (int32, shape (cap, 2));
    returns (npairs, root). Synchronises the stream."""
    g = grid_of(f)
    n = f.numel()
    pf = _dev(f, "f", (torch.float32,))
    pW = _dev(W, "W", _I64, n)
    pws = _dev(ws, "ws", (torch.uint8,))
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape (cap, 2)")
    cap = int(pairs.shape[0])
    pp = _dev(pairs, "pairs", _I32) if cap else 0
    npairs = ctypes.c_uint64(0)
    root = ctypes.c_uint32(0xFFFFFFFF)
    code = load().mt_persistence_pairs(pf, pW, g, pp, cap, ctypes.byref(npairs), ctypes.byref(root), pws,
                                       ws.numel(), _stream_ptr(stream))
    if code == -4 and allow_partial:
        return int(npairs.value), int(root.value)
    _check(code, "mt_persistence_pairs", f" npairs={npairs.value} cap={cap}")
    return int(npairs.value), int(root.value)


def mt_simplified_pairs(f: torch.Tensor, W: torch.Tensor, eps: float, flags: int, pairs: torch.Tensor,
                        ws: torch.Tensor, stream=None, allow_partial: bool = False) -> tuple[int, int]:
    """The pairs of persistence >= eps (float32 f(s) - f(u), on -f with
    MT_SUPERLEVEL) as (minimum, saddle) rows of ``pairs``; returns
    (npairs, root). Synchronises the stream."""
    g = grid_of(f)
    n = f.numel()
    pf = _dev(f, "f", (torch.float32,))
    pW = _dev(W, "W", _I64, n)
    pws = _dev(ws, "ws", (torch.uint8,))
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape (cap, 2)")
    cap = int(pairs.shape[0])
    pp = _dev(pairs, "pairs", _I32) if cap else 0
    npairs = ctypes.c_uint64(0)
    root = ctypes.c_uint32(0xFFFFFFFF)
    code = load().mt_simplified_pairs(pf, pW, g, float(eps), int(flags), pp, cap, ctypes.byref(npairs),
                                      ctypes.byref(root), pws, ws.numel(), _stream_ptr(stream))
    if code == -4 and allow_partial:
        return int(npairs.value), int(root.value)
    _check(code, "mt_simplified_pairs", f" npairs={npairs.value} cap={cap}")
    return int(npairs.value), int(root.value)


def mt_simplified_components_at(f: torch.Tensor, W: torch.Tensor, t: float, eps: float, flags: int,
                                labels: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    """Labels of G_t after filling every branch of persistence < eps up to its
    saddle (0xFFFFFFFF outside the simplified G_t)."""
    g = grid_of(f)
    n = f.numel()
    _check(load().mt_simplified_components_at(_dev(f, "f", (torch.float32,)), _dev(W, "W", _I64, n), g, float(t),
                                              float(eps), int(flags), _dev(labels, "labels", _I32, n),
                                              _dev(ws, "ws", (torch.uint8,)), ws.numel(), _stream_ptr(stream)),
           "mt_simplified_components_at")


def mt_branches_workspace_bytes(grid: Grid) -> int:
    return int(load().mt_branches_workspace_bytes(grid))


def branches_workspace(grid: Grid, device=None) -> torch.Tensor:
    """A device byte tensor for mt_branch_decomposition on ``grid`` with its
    status word cleared."""
    nbytes = mt_branches_workspace_bytes(grid)
    if nbytes == 0:
        raise MtError(-1, "mt_branches_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
    ws[:256].zero_()
    return ws


def mt_branch_decomposition(f: torch.Tensor, W: torch.Tensor, flags: int, order: torch.Tensor,
                            offsets: torch.Tensor, ws: torch.Tensor, stream=None) -> int:
    """Vertices grouped by branch into ``order`` (int32[n]) with group starts in
    ``offsets`` (int32[cap], offsets[nbranches] = n); returns the number of
    branches. Synchronises the stream."""
    g = grid_of(f)
    n = f.numel()
    cap = int(offsets.numel())
    nb = ctypes.c_uint64(0)
    code = load().mt_branch_decomposition(_dev(f, "f", (torch.float32,)), _dev(W, "W", _I64, n), g, int(flags),
                                          _dev(order, "order", _I32, n),
                                          _dev(offsets, "offsets", _I32) if cap else 0, cap, ctypes.byref(nb),
                                          _dev(ws, "ws", (torch.uint8,)), ws.numel(), _stream_ptr(stream))
    _check(code, "mt_branch_decomposition", f" nbranches={nb.value} cap={cap}")
    return int(nb.value)


def mt_persistence_pairs_noalloc(f: torch.Tensor, W: torch.Tensor, pairs: torch.Tensor, stream=None,
                                 allow_partial: bool = False) -> tuple[int, int]:
    """mt_persistence_pairs without a workspace: the C call takes its scratch
    from an array inside libmt (for callers that cannot allocate device
    memory). Returns (npairs, root); synchronises the stream."""
    g = grid_of(f)
    n = f.numel()
    pf = _dev(f, "f", (torch.float32,))
    pW = _dev(W, "W", _I64, n)
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape (cap, 2)")
    cap = int(pairs.shape[0])
    pp = _dev(pairs, "pairs", _I32) if cap else 0
    npairs = ctypes.c_uint64(0)
    root = ctypes.c_uint32(0xFFFFFFFF)
    code = load().mt_persistence_pairs_noalloc(pf, pW, g, pp, cap, ctypes.byref(npairs), ctypes.byref(root),
                                               _stream_ptr(stream))
    if code == -4 and allow_partial:
        return int(npairs.value), int(root.value)
    _check(code, "mt_persistence_pairs_noalloc", f" npairs={npairs.value} cap={cap}")
    return int(npairs.value), int(root.value)


def mt_wide_workspace_bytes(grid: Grid) -> int:
    return int(load().mt_wide_workspace_bytes(grid))


def wide_workspace(grid: Grid, device=None) -> torch.Tensor:
    """A device byte tensor for the wide-id calls on ``grid``, status cleared."""
    nbytes = mt_wide_workspace_bytes(grid)
    if nbytes == 0:
        raise MtError(-2 if grid.nx and grid.ny and grid.nz else -1, "mt_wide_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
    ws[:768].zero_()
    return ws


def mt_build_triplets_wide(f: torch.Tensor, W2: torch.Tensor, ws: torch.Tensor, flags: int = 0, stream=None) -> None:
    """Triplets with 64-bit ids: W2 is int64 (n, 2) = (s, v) (uint64 bit
    patterns), 16-byte aligned. Asynchronous."""
    g = grid_of(f)
    n = f.numel()
    _check(load().mt_build_triplets_wide(_dev(f, "f", (torch.float32,)), g, _dev(W2, "W2", _I64, 2 * n),
                                         _dev(ws, "ws", (torch.uint8,)), ws.numel(), int(flags), _stream_ptr(stream)),
           "mt_build_triplets_wide")


def mt_persistence_pairs_wide(W2: torch.Tensor, grid: Grid, pairs: torch.Tensor, ws: torch.Tensor, stream=None,
                              allow_partial: bool = False) -> tuple[int, int]:
    """(minimum, saddle) rows with 64-bit ids into ``pairs`` (int64 (cap, 2));
    returns (npairs, root). Synchronises the stream."""
    n = grid.nx * grid.ny * grid.nz
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape (cap, 2)")
    cap = int(pairs.shape[0])
    pp = _dev(pairs, "pairs", _I64) if cap else 0
    npairs = ctypes.c_uint64(0)
    root = ctypes.c_uint64(~0 & 0xFFFFFFFFFFFFFFFF)
    code = load().mt_persistence_pairs_wide(_dev(W2, "W2", _I64, 2 * n), grid, pp, cap, ctypes.byref(npairs),
                                            ctypes.byref(root), _dev(ws, "ws", (torch.uint8,)), ws.numel(),
                                            _stream_ptr(stream))
    if code == -4 and allow_partial:
        return int(npairs.value), int(root.value)
    _check(code, "mt_persistence_pairs_wide", f" npairs={npairs.value} cap={cap}")
    return int(npairs.value), int(root.value)


def mt_components_at_wide(f: torch.Tensor, W2: torch.Tensor, t: float, flags: int, labels: torch.Tensor,
                          ws: torch.Tensor, stream=None) -> None:
    """64-bit labels (int64[n]; all ones outside G_t). Asynchronous."""
    g = grid_of(f)
    n = f.numel()
    _check(load().mt_components_at_wide(_dev(f, "f", (torch.float32,)), _dev(W2, "W2", _I64, 2 * n), g, float(t),
                                        int(flags), _dev(labels, "labels", _I64, n), _dev(ws, "ws", (torch.uint8,)),
                                        ws.numel(), _stream_ptr(stream)), "mt_components_at_wide")


def _grid_array(grids):
    arr = (Grid * len(grids))()
    for i, g in enumerate(grids):
        arr[i] = g if isinstance(g, Grid) else Grid(*g)
    return arr


def mt_batch_workspace_bytes(grids) -> int:
    arr = _grid_array(grids)
    return int(load().mt_batch_workspace_bytes(ctypes.cast(arr, ctypes.c_void_p), len(grids)))


def mt_batch_prepare(arena: torch.Tensor, grids, W_arena: torch.Tensor, pairs_arena: torch.Tensor,
                     ws: torch.Tensor, stream=None) -> BatchPlan:
    """Writes the batch's field table into ``ws``; returns the plan. ``grids``
    are Grid(nx, ny, nz) (or (nx, ny, nz) tuples) in arena order."""
    arr = _grid_array(grids)
    total = sum(g.nx * g.ny * g.nz for g in arr)
    pa = _dev(arena, "arena", (torch.float32,), total)
    pW = _dev(W_arena, "W_arena", _I64, total)
    pp = _dev(pairs_arena, "pairs_arena", _I32, 2 * total)
    pws = _dev(ws, "ws", (torch.uint8,))
    plan = BatchPlan()
    _check(load().mt_batch_prepare(pa, ctypes.cast(arr, ctypes.c_void_p), len(grids), pW, pp, pws, ws.numel(),
                                   ctypes.byref(plan), _stream_ptr(stream)), "mt_batch_prepare")
    return plan


def mt_batch_launch(plan: BatchPlan, cfg: int, npairs: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    """Enqueues the batched build + pairs with launch configuration cfg."""
    pn = _dev(npairs, "npairs", _I64, plan.nfields)
    pws = _dev(ws, "ws", (torch.uint8,))
    _check(load().mt_batch_launch(ctypes.byref(plan), int(cfg), pn, pws, ws.numel(), _stream_ptr(stream)),
           "mt_batch_launch")


def mt_batch_build(arena: torch.Tensor, grids, W_arena: torch.Tensor, pairs_arena: torch.Tensor,
                   npairs: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    arr = _grid_array(grids)
    total = sum(g.nx * g.ny * g.nz for g in arr)
    _check(load().mt_batch_build(_dev(arena, "arena", (torch.float32,), total), ctypes.cast(arr, ctypes.c_void_p),
                                 len(grids), _dev(W_arena, "W_arena", _I64, total),
                                 _dev(pairs_arena, "pairs_arena", _I32, 2 * total),
                                 _dev(npairs, "npairs", _I64, len(grids)), _dev(ws, "ws", (torch.uint8,)),
                                 ws.numel(), _stream_ptr(stream)), "mt_batch_build")


def mt_batch_autotune(plan: BatchPlan, npairs: torch.Tensor, ws: torch.Tensor, stream=None):
    """Times every launch configuration of the batch; returns ([ms per cfg],
    best cfg)."""
    ms = (ctypes.c_float * MT_CFG_COUNT)()
    best = ctypes.c_int(0)
    _check(load().mt_batch_autotune(ctypes.byref(plan), _dev(npairs, "npairs", _I64, plan.nfields),
                                    _dev(ws, "ws", (torch.uint8,)), ws.numel(), _stream_ptr(stream),
                                    ctypes.cast(ms, ctypes.c_void_p), ctypes.byref(best)), "mt_batch_autotune")
    return [float(x) for x in ms], int(best.value)


def mt_server_create(hbm_budget_bytes: int, max_slots: int, device: int = 0) -> int:
    h = load().mt_server_create(int(hbm_budget_bytes), int(max_slots), int(device))
    if not h:
        raise MtError(-6, "mt_server_create")
    return h


def _host(t: torch.Tensor, name: str, dtypes, numel=None) -> int:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if t.dtype not in dtypes or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous tensor of {dtypes}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements")
    return t.data_ptr()


def mt_server_submit(srv: int, f: torch.Tensor, t: float, pairs: torch.Tensor | None,
                     labels: torch.Tensor | None) -> int:
    """Queues (f, t) on the server; f, pairs ((cap, 2) int32) and labels (n
    int32) are host tensors the server reads/writes until the ticket is done."""
    g = Grid(int(f.shape[2]), int(f.shape[1]), int(f.shape[0]))
    n = f.numel()
    pf = _host(f, "f", (torch.float32,))
    pp = _host(pairs, "pairs", _I32) if pairs is not None else 0
    cap = int(pairs.shape[0]) if pairs is not None else 0
    pl = _host(labels, "labels", _I32, n) if labels is not None else 0
    ticket = ctypes.c_uint64(0)
    _check(load().mt_server_submit(srv, pf, g, float(t), pp, cap, pl, ctypes.byref(ticket)), "mt_server_submit")
    return int(ticket.value)


def mt_server_submit_resident(srv: int, key: int, f: torch.Tensor | None, grid: Grid, t: float,
                              pairs: torch.Tensor | None, labels: torch.Tensor | None) -> int:
    """Queues (key, t): builds and keeps the field under ``key`` if it is not
    resident yet (f, a host float32 tensor, is then required), else reuses
    the resident tree (f may be None). Returns the ticket."""
    n = grid.nx * grid.ny * grid.nz
    pf = _host(f, "f", (torch.float32,), n) if f is not None else 0
    pp = _host(pairs, "pairs", _I32) if pairs is not None else 0
    cap = int(pairs.shape[0]) if pairs is not None else 0
    pl = _host(labels, "labels", _I32, n) if labels is not None else 0
    ticket = ctypes.c_uint64(0)
    _check(load().mt_server_submit_resident(srv, int(key), pf, grid, float(t), pp, cap, pl, ctypes.byref(ticket)),
           "mt_server_submit_resident")
    return int(ticket.value)


def mt_server_evict(srv: int, key: int) -> None:
    _check(load().mt_server_evict(srv, int(key)), "mt_server_evict")


def mt_server_resident(srv: int) -> tuple[int, int]:
    """(number of built resident entries, device bytes they hold)."""
    c, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(load().mt_server_resident(srv, ctypes.byref(c), ctypes.byref(b)), "mt_server_resident")
    return int(c.value), int(b.value)


def mt_server_poll(srv: int, ticket: int):
    """MtResult once done, None while pending."""
    r = MtResult()
    code = load().mt_server_poll(srv, int(ticket), ctypes.byref(r))
    if code == -8:
        return None
    _check(code, "mt_server_poll")
    return r


def mt_server_wait(srv: int, ticket: int) -> MtResult:
    r = MtResult()
    _check(load().mt_server_wait(srv, int(ticket), ctypes.byref(r)), "mt_server_wait")
    return r


def mt_server_destroy(srv: int) -> None:
    load().mt_server_destroy(srv)


def mt_components_at(f: torch.Tensor, W: torch.Tensor, t: float, labels: torch.Tensor, ws: torch.Tensor,
                     stream=None) -> None:
    g = grid_of(f)
    n = f.numel()
    pf = _dev(f, "f", (torch.float32,))
    pW = _dev(W, "W", _I64, n)
    pl = _dev(labels, "labels", _I32, n)
    pws = _dev(ws, "ws", (torch.uint8,))
    _check(load().mt_components_at(pf, pW, g, float(t), pl, pws, ws.numel(), _stream_ptr(stream)),
           "mt_components_at")


def mt_sync_status(ws: torch.Tensor, stream=None) -> None:
    _check(load().mt_sync_status(_dev(ws, "ws", (torch.uint8,)), _stream_ptr(stream)), "mt_sync_status")


class PhaseTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("calls", ctypes.c_ulonglong), ("total_ms", ctypes.c_double)]


def mt_trace_enable(on: bool = True) -> None:
    load().mt_trace_enable(1 if on else 0)


def mt_trace_read(reset: bool = True) -> dict[str, tuple[int, float]]:
    """{step name: (calls, total device ms)} accumulated since the last reset."""
    rows = (PhaseTime * 16)()
    k = load().mt_trace_read(ctypes.cast(rows, ctypes.c_void_p), 16, 1 if reset else 0)
    return {rows[i].name.decode(): (int(rows[i].calls), float(rows[i].total_ms)) for i in range(min(k, 16))}


def mt_kernel_launches() -> int:
    return int(load().mt_kernel_launches())
