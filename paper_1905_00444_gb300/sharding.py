"""Host-side sharding of slices across processes (replicas: one process per GPU).

Slices are independent (Sec. III.A: "no communication between compute nodes"), so each
rank takes a contiguous range of slice ids, computes its partial amplitudes with
qfx_amplitudes(slice_begin, slice_end), and the host adds the partials.  The only
exchange is one gather of B complex128 values per bitstring batch; the sum runs in rank
order, so the result does not depend on the backend's reduction order.
"""
from __future__ import annotations

from typing import Tuple


def partition_slices(n_slices: int, world_size: int, rank: int) -> Tuple[int, int]:
    """Balanced contiguous range [begin, end) of slice ids for `rank` (may be empty)."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world_size / rank")
    base, extra = divmod(n_slices, world_size)
    begin = rank * base + min(rank, extra)
    end = begin + base + (1 if rank < extra else 0)
    return begin, end


def reduce_partials(partial, group=None):
    """Sum a CPU complex128 tensor over all ranks, adding in rank order (deterministic)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return partial
    world = dist.get_world_size(group)
    real = torch.view_as_real(partial.contiguous()).clone()
    bufs = [torch.empty_like(real) for _ in range(world)]
    dist.all_gather(bufs, real, group=group)
    total = bufs[0].clone()
    for b in bufs[1:]:
        total += b
    return torch.view_as_complex(total)
