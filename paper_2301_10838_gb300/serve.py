"""Python front of libmt's request server (continuous batching on one GPU).

``Server`` keeps every submitted request's host tensors alive until its
result is collected; all work runs in libmt (mt_server_*).
"""

from __future__ import annotations

import torch

from . import binding as B


class Server:
    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4, device: int = 0):
        self.h = B.mt_server_create(hbm_budget_bytes, max_slots, device)
        self.live: dict[int, tuple] = {}

    def submit(self, f: torch.Tensor, t: float, want_pairs: bool = True, want_labels: bool = True,
               pairs: torch.Tensor | None = None, labels: torch.Tensor | None = None, pin: bool = True) -> int:
        """f: host float32 (nz, ny, nx). Output tensors are allocated (pinned)
        unless given. Returns the ticket."""
        n = f.numel()
        if want_pairs and pairs is None:
            pairs = torch.empty((n // 2 + 1, 2), dtype=torch.int32, pin_memory=pin)
        if want_labels and labels is None:
            labels = torch.empty(n, dtype=torch.int32, pin_memory=pin)
        ticket = B.mt_server_submit(self.h, f, t, pairs if want_pairs else None, labels if want_labels else None)
        self.live[ticket] = (f, pairs, labels)
        return ticket

    def submit_resident(self, key: int, f: torch.Tensor | None, t: float, shape=None, want_pairs: bool = True,
                        want_labels: bool = True, pairs: torch.Tensor | None = None,
                        labels: torch.Tensor | None = None, pin: bool = True) -> int:
        """Like submit, but the field, its tree and its pairs stay on the
        device under ``key``; a later call with the same key reuses them (f
        may then be None, with ``shape`` = (nz, ny, nx))."""
        nz, ny, nx = (int(v) for v in (f.shape if f is not None else shape))
        n = nx * ny * nz
        if want_pairs and pairs is None:
            pairs = torch.empty((n // 2 + 1, 2), dtype=torch.int32, pin_memory=pin)
        if want_labels and labels is None:
            labels = torch.empty(n, dtype=torch.int32, pin_memory=pin)
        ticket = B.mt_server_submit_resident(self.h, key, f, B.Grid(nx, ny, nz), t,
                                             pairs if want_pairs else None, labels if want_labels else None)
        self.live[ticket] = (f, pairs, labels)
        return ticket

    def evict(self, key: int) -> None:
        B.mt_server_evict(self.h, key)

    def resident(self) -> tuple[int, int]:
        return B.mt_server_resident(self.h)

    def _out(self, ticket, r):
        f, pairs, labels = self.live.pop(ticket)
        if r.status not in (0,):
            raise B.MtError(r.status, "server request")
        k = int(r.npairs)
        return {"npairs": k, "root": int(r.root), "pairs": pairs[:k] if pairs is not None else None,
                "reused": bool(r.reused),
                "labels": labels, "latency_s": r.t_done - r.t_submit, "queue_s": r.t_admit - r.t_submit,
                "t_submit": r.t_submit, "t_done": r.t_done}

    def poll(self, ticket: int):
        r = B.mt_server_poll(self.h, ticket)
        return None if r is None else self._out(ticket, r)

    def wait(self, ticket: int):
        return self._out(ticket, B.mt_server_wait(self.h, ticket))

    def close(self):
        if self.h:
            B.mt_server_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
