"""GB300-native sparse MTTKRP / CP-ALS over a linearized sparse encoding.

Python binding of the C ABI in ``include/relate.h`` (librelate.so, built
in-tree for sm_103a). The binding only marshals arguments: every step of
the encode / MTTKRP / CP-ALS path runs in the library's CUDA kernels. There
is no CPU fallback: importing the binding without the built library raises.

Device buffers are passed as torch CUDA tensors (their data_ptr), streams as
``torch.cuda.Stream`` or raw handles; host buffers as numpy arrays.
"""
from __future__ import annotations

from .relate import (  # noqa: F401
    RELATE_BF16, RELATE_CONFLICT_ATOMIC, RELATE_CONFLICT_AUTO, RELATE_CONFLICT_PRIVATIZED,
    RELATE_CONFLICT_SEGMENTED, RELATE_F32, RELATE_F64, RelateError, Handle, lib, library_path,
    relate_cpals, relate_decode, relate_encode, relate_footprint, relate_free, relate_get_conflict,
    relate_get_partitions, relate_get_stats, relate_gram, relate_gram_noalloc, relate_last_error, relate_solve_rows,
    relate_get_mode_kr, relate_get_mode_plan, relate_mttkrp, relate_mttkrp_batch, relate_cpals_batch, relate_release_cached_memory,
    relate_set_conflict, relate_set_reduce_hook, relate_shard_range,
    relate_set_cpals_graph, relate_set_mode_kr, relate_set_mode_plan, relate_set_precision, relate_set_stream,
    relate_status_string, relate_sync_status, relate_version,
)
