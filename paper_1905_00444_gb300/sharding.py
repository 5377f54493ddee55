"""Host-side sharding of slices across processes (replicas: one process per GPU).

Slices are independent (Sec. III.A: the paper's compute nodes never exchange data), so each
rank takes a contiguous range of slice ids, computes its partial amplitudes with
qfx_amplitudes(slice_begin, slice_end), and the host adds the partials.  The only
exchange is one gather of B complex128 values per bitstring batch; the sum runs in rank
order, so the result does not depend on the backend's reduction order.  Batches of items
of uneven cost (mixed grids, slices and x1 batches) go to ranks by planned cost (LPT);
each item's rows then come from one rank, and the same rank-order sum assembles them.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence, Tuple


def partition_slices(n_slices: int, world_size: int, rank: int) -> Tuple[int, int]:
    """Balanced contiguous range [begin, end) of slice ids for `rank` (may be empty)."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world_size / rank")
    base, extra = divmod(n_slices, world_size)
    begin = rank * base + min(rank, extra)
    end = begin + base + (1 if rank < extra else 0)
    return begin, end


def item_costs(items) -> List[float]:
    """Planned cost of each batch item (plan, x1, slice_begin, slice_end): Eq. 1 flops of one
    work item times its slices times its x1 bitstrings (slice_end None = every slice)."""
    costs = []
    for plan, x1, sb, se in items:
        se = plan.n_slices if se is None else se
        costs.append(float(plan.stats["flops_per_item"]) * (se - sb) * plan.batch_of(x1))
    return costs


def partition_items(costs: Sequence[float], world_size: int) -> List[List[int]]:
    """Items of uneven cost over ranks by LPT (Graham's longest-processing-time-first rule):
    the items by decreasing cost (ties: lower index first), each to the rank with the least
    load so far (ties: lower rank).  Returns each rank's item indices in increasing order;
    the largest load is at most (4/3 - 1/(3 world_size)) of the best possible."""
    if world_size < 1:
        raise ValueError("bad world_size")
    if any(c < 0 for c in costs):
        raise ValueError("negative cost")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world_size)]
    out: List[List[int]] = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(x) for x in out]


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
