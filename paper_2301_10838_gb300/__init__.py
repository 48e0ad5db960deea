"""Triplet merge trees of scalar fields on regular grids, native to GB300.

The compute path is libmt (hand-written CUDA for sm_103a behind the C ABI of
``include/mt.h``); ``binding`` is its thin ctypes binding with the same names.
``fields`` holds the seeded synthetic inputs. Importing the package does not
load libmt; the first ``mt_*`` call does, and raises if it is not built.
"""

from .binding import (  # noqa: F401
    BatchPlan,
    Grid,
    MtError,
    grid_of,
    load,
    mt_batch_autotune,
    mt_batch_build,
    mt_batch_launch,
    mt_batch_prepare,
    mt_batch_workspace_bytes,
    mt_build_triplets,
    mt_components_at,
    mt_persistence_pairs,
    mt_persistence_pairs_noalloc,
    mt_server_create,
    mt_server_destroy,
    mt_server_poll,
    mt_server_submit,
    mt_server_wait,
    mt_status_str,
    mt_kernel_launches,
    mt_sync_status,
    mt_trace_enable,
    mt_trace_read,
    mt_workspace_bytes,
    workspace,
)

__all__ = [
    "BatchPlan",
    "Grid",
    "mt_batch_autotune",
    "mt_batch_build",
    "mt_batch_launch",
    "mt_batch_prepare",
    "mt_batch_workspace_bytes",
    "MtError",
    "grid_of",
    "load",
    "mt_build_triplets",
    "mt_components_at",
    "mt_persistence_pairs",
    "mt_persistence_pairs_noalloc",
    "mt_server_create",
    "mt_server_destroy",
    "mt_server_poll",
    "mt_server_submit",
    "mt_server_wait",
    "mt_status_str",
    "mt_sync_status",
    "mt_trace_enable",
    "mt_trace_read",
    "mt_kernel_launches",
    "mt_workspace_bytes",
    "workspace",
]
