"""Sharded evaluation over several ranks (arXiv:1905.04582, section 2.5: the
pairwise sum split over workers and the partial sums reduced).

The library does the work: each rank's context holds only its range of the
tile-packed Y (``mds_shard_range``: contiguous tiles of equal pair count),
computes its partials {L_r, dL/dsigma_r, sum r_r, dL/dX_r} on the device and,
once the partials of all ranks are gathered, sums them in rank order
(``mds_set_shard``; ``mds_shard_sum`` is the same sum on the host).  This
module only moves bytes: ``torch_allgather`` adapts ``torch.distributed`` to
the library's all-gather callback (NCCL on device buffers, gloo or any other
backend on host buffers).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi


def shard_range(n, n_ranks, rank):
    """Tiles [t0, t1) of rank `rank` (mds_shard_range)."""
    t0, t1 = ctypes.c_int64(), ctypes.c_int64()
    capi.check(capi.lib().mds_shard_range(int(n), int(n_ranks), int(rank), ctypes.byref(t0), ctypes.byref(t1)))
    return t0.value, t1.value


def shard_sum(gathered):
    """The fixed-order sum (rank 0 first) of an (n_ranks, count) array of
    partial vectors, as the library's combine does it (mds_shard_sum)."""
    g = np.ascontiguousarray(gathered, dtype=np.float64)
    out = np.empty(g.shape[1], dtype=np.float64)
    capi.check(capi.lib().mds_shard_sum(int(g.shape[0]), int(g.shape[1]), g.ctypes.data_as(ctypes.c_void_p),
                                        out.ctypes.data_as(ctypes.c_void_p)))
    return out


class _CudaBuf:
    """A device buffer of float64 known by its address (zero-copy view)."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def torch_allgather(group=None):
    """An all-gather for MDS.set_shard over a torch.distributed group: host
    buffers (MDS_HOST) go through CPU tensors (gloo), device buffers
    (MDS_DEVICE) through CUDA tensors (NCCL), gathered in rank order."""
    import torch
    import torch.distributed as dist

    def allgather(send, recv, count, where):
        world = dist.get_world_size(group)
        if where == capi.MDS_HOST:
            s = torch.from_numpy(np.ctypeslib.as_array((ctypes.c_double * count).from_address(send)))
            r = torch.from_numpy(np.ctypeslib.as_array((ctypes.c_double * (count * world)).from_address(recv)))
        else:
            s = torch.as_tensor(_CudaBuf(send, count), device="cuda")
            r = torch.as_tensor(_CudaBuf(recv, count * world), device="cuda")
        parts = list(r.view(world, count).unbind(0))
        dist.all_gather(parts, s, group=group)
        if where != capi.MDS_HOST:
            torch.cuda.synchronize()
        return 0

    return allgather
