"""Sharded CP-ALS over torch.distributed: one process per GPU, each holding a
contiguous equal-nnz shard of the sorted nonzero stream.

The MTTKRP of Sec. 2.2 (Fig. 2) is a sum over the nonzeros, so with the
factors replicated on every process each shard computes a partial M_n and
one all-reduce per mode (of I_n x R values) gives every process the full M_n;
||X||^2 is summed once per call. Everything else of CP-ALS (Grams, normal
equations, solve, normalisation, fit) is R x R or row-local and runs
identically everywhere. The library does the sharding
(relate_params_t.shard_rank / shard_count, relate_shard_range) and calls the
reduction through relate_set_reduce_hook; this module supplies the
reduction: an NCCL all-reduce enqueued on the library's stream, or, for a
gloo group, a host round trip.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import relate as rl

_TORCH_OF = {rl.RELATE_F64: "float64", rl.RELATE_F32: "float32"}
_NP_OF = {rl.RELATE_F64: np.float64, rl.RELATE_F32: np.float32}


class _DeviceBuffer:
    """A device buffer described by __cuda_array_interface__ (zero-copy view)."""

    def __init__(self, ptr: int, count: int, dtype: int):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8" if dtype == rl.RELATE_F64 else "<f4",
                                         "data": (int(ptr), False), "version": 2, "strides": None}


def device_view(ptr: int, count: int, dtype: int):
    """A torch CUDA tensor over `count` elements at device address `ptr`."""
    import torch
    return torch.as_tensor(_DeviceBuffer(ptr, count, dtype), device="cuda")


def host_view(ptr: int, count: int, dtype: int) -> np.ndarray:
    """A numpy array over `count` elements at host address `ptr`."""
    ctype = ctypes.c_double if dtype == rl.RELATE_F64 else ctypes.c_float
    return np.ctypeslib.as_array((ctype * int(count)).from_address(int(ptr)))


def torch_reduce_hook(group=None):
    """The all-reduce (sum) of a sharded relate_cpals over a torch.distributed
    group: NCCL enqueues it on the library's stream; another backend (gloo)
    copies the buffer to the host, reduces there and copies it back."""
    import torch
    import torch.distributed as dist

    backend = dist.get_backend(group)

    def fn(buf, count, dtype, stream):
        t = device_view(buf, count, dtype)
        st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
        if backend == "nccl":
            with torch.cuda.stream(st):
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        else:
            st.synchronize()
            host = t.cpu()
            dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
            with torch.cuda.stream(st):
                t.copy_(host, non_blocking=False)
            st.synchronize()
        return 0

    return fn


def host_reduce_hook(group=None):
    """The same reduction for buffers in host memory (gloo): what a CPU
    process of the sharded protocol calls."""
    import torch
    import torch.distributed as dist

    def fn(buf, count, dtype, stream):
        t = torch.from_numpy(host_view(buf, count, dtype))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return 0

    return fn


def sharded_encode(coords, vals, dims, rank: int, world: int, **kw):
    """relate_encode of this process's shard of the sorted stream (every
    process passes the whole tensor)."""
    return rl.relate_encode(coords, vals, dims, shard_rank=rank, shard_count=world, **kw)


def sharded_cpals(h, R: int, iters: int, tol: float, factors, group=None):
    """relate_cpals of a sharded handle with the group's all-reduce: every
    process gets the same factors, lambda and fit."""
    rl.relate_set_reduce_hook(h, torch_reduce_hook(group))
    try:
        return rl.relate_cpals(h, R, iters, tol, factors)
    finally:
        rl.relate_set_reduce_hook(h, None)
