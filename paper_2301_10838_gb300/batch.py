"""Batched merge trees over many uneven fields (host-side orchestration).

``Batch`` packs fields into device arenas, prepares the field table in libmt,
picks the launch configuration (tile shape, level buckets, repair CTA size)
with libmt's autotuner (cached per GPU and batch shape class, ``autotune``),
and optionally captures the batched launch in a CUDA graph so that a
repeated batch costs one graph launch. All merge-tree work runs in libmt's
kernels.
"""

from __future__ import annotations

import torch

from . import autotune
from . import binding as B

def shape_class(grids) -> str:
    return autotune.batch_class(grids)


class Batch:
    """A packed batch of fields on one device.

    grids: list of (nz, ny, nx) shapes in arena order.
    """

    def __init__(self, shapes, device="cuda"):
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.grids = [B.Grid(s[2], s[1], s[0]) for s in self.shapes]
        self.sizes = [s[0] * s[1] * s[2] for s in self.shapes]
        self.offsets = [0]
        for n in self.sizes:
            self.offsets.append(self.offsets[-1] + n)
        total = self.offsets[-1]
        self.device = torch.device(device)
        self.arena = torch.empty(total, dtype=torch.float32, device=self.device)
        self.W = torch.empty(total, dtype=torch.int64, device=self.device)
        self.pairs = torch.empty((total, 2), dtype=torch.int32, device=self.device)
        self.npairs = torch.zeros(len(self.shapes), dtype=torch.int64, device=self.device)
        nbytes = B.mt_batch_workspace_bytes(self.grids)
        if nbytes == 0:
            raise ValueError("invalid batch")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.plan = B.mt_batch_prepare(self.arena, self.grids, self.W, self.pairs, self.ws)
        self.cfg = 0  # launch configuration (MT_CFG_* bits)
        self.graph = None

    def field(self, i: int) -> torch.Tensor:
        a, b = self.offsets[i], self.offsets[i + 1]
        return self.arena[a:b].view(self.shapes[i])

    def load(self, fields) -> None:
        for i, f in enumerate(fields):
            self.field(i).copy_(torch.as_tensor(f).reshape(self.shapes[i]), non_blocking=True)

    def tune(self, use_cache: bool = True) -> int:
        """Pick the launch configuration: cached for this GPU and shape class,
        else libmt's autotuner over all MT_CFG_COUNT configurations (which
        needs the fields loaded). Returns it."""
        cls = autotune.batch_class(self.shapes)
        if use_cache:
            hit = autotune.lookup(self.device, cls)
            if hit is not None:
                self.cfg = int(hit["cfg"])
                return self.cfg
        ms, best = B.mt_batch_autotune(self.plan, self.npairs, self.ws)
        self.cfg = best
        self.tuned_ms = ms
        if use_cache:
            autotune.store(self.device, cls, best, ms)
        return best

    def launch(self, stream=None) -> None:
        if self.graph is not None:
            self.graph.replay()
            return
        B.mt_batch_launch(self.plan, self.cfg, self.npairs, self.ws, stream)

    def capture(self) -> None:
        """Capture the batched launch in a CUDA graph (tracing must be off)."""
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            B.mt_batch_launch(self.plan, self.cfg, self.npairs, self.ws, s)  # warm-up outside the graph
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            B.mt_batch_launch(self.plan, self.cfg, self.npairs, self.ws, s)
        self.graph = g

    def results(self, i: int):
        """(triplets, pairs) of field i as device tensor views."""
        a, b = self.offsets[i], self.offsets[i + 1]
        k = int(self.npairs[i])
        return self.W[a:b], self.pairs[a:a + k]
