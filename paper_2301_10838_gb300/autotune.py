"""Autotuner cache: the fastest launch configuration per GPU and shape class.

libmt times the configurations itself (mt_batch_autotune for a packed batch,
mt_build_autotune for one field); this module keeps the winner in a JSON
file (``MT_AUTOTUNE_CACHE``, default ``~/.cache/mt_gb300_autotune.json``)
keyed by the GPU name and a shape class, so that later runs on the same kind
of input skip the timing. Every configuration gives the same results.

Configurations are the MT_CFG_* bits of include/mt.h: tile shape (batches:
16x16x8 or 16x16x16; single fields: 16x16x16 or 32x16x16), level buckets per
tile (the merge/repair rounds) and the repair CTA size.
"""

from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import binding as B

_LOCK = threading.Lock()


def cache_path() -> str:
    return os.environ.get("MT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mt_gb300_autotune.json"))


def batch_class(shapes) -> str:
    """Batch shape class: field count and the log2 of the mean and largest
    field size (vertices)."""
    sizes = [s[0] * s[1] * s[2] for s in shapes]
    mean = sum(sizes) / len(sizes)
    return f"batch-n{len(sizes)}-mean{round(math.log2(mean))}-max{round(math.log2(max(sizes)))}"


def single_class(shape, flags: int = 0) -> str:
    """Single-field shape class: log2 of the vertex count and of the x side,
    and the flags."""
    nz, ny, nx = (int(v) for v in shape)
    return f"single-n{round(math.log2(nx * ny * nz))}-x{round(math.log2(nx))}-f{int(flags)}"


def _key(device, cls: str) -> str:
    return f"{torch.cuda.get_device_name(device)}|{cls}"


def lookup(device, cls: str):
    """The cached entry {"cfg": .., "ms": ..} or None."""
    with _LOCK:
        try:
            with open(cache_path()) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            return None
    return cache.get(_key(device, cls))


def store(device, cls: str, cfg: int, ms) -> None:
    path = cache_path()
    with _LOCK:
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
        cache[_key(device, cls)] = {"cfg": int(cfg), "ms": ms}
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + f".{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, path)


def tune_single(f: torch.Tensor, W: torch.Tensor, ws: torch.Tensor, flags: int = 0, use_cache: bool = True):
    """The fastest configuration for building the tree of fields like f:
    cached for this GPU and shape class, else timed by libmt (W then holds
    the triplets). Returns (cfg, {cfg: ms} or None when cached)."""
    cls = single_class(f.shape, flags)
    if use_cache:
        hit = lookup(f.device, cls)
        if hit is not None:
            return int(hit["cfg"]), None
    ms, best = B.mt_build_autotune(f, W, ws, flags)
    if use_cache:
        store(f.device, cls, best, {str(k): v for k, v in ms.items()})
    return best, ms
