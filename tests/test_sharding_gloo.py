"""Multi-process sharding of slices and batch items (replicas, no data-path collective) on
CPU ranks.

Slices are independent paths (Sec. III.A): each rank takes a contiguous slice range and
computes its partial amplitudes; the host adds the partials in rank order.  On this CPU
test the per-rank partial comes from the oracle's sliced contraction (the GPU path
computes the same quantity with qfx_amplitudes(slice_begin, slice_end)); what is tested
is the partition and the reduction over gloo ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import itertools

import rqc_inputs as ri
from oracle import network
from paper_1905_00444_gb300.sharding import (item_costs, partition_items, partition_slices,
                                             reduce_partials)


def test_partition_covers_every_slice_once():
    for n in (1, 2, 7, 16, 1000):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                b, e = partition_slices(n, world, r)
                assert 0 <= b <= e <= n
                got += list(range(b, e))
            assert got == list(range(n))
            sizes = [partition_slices(n, world, r)[1] - partition_slices(n, world, r)[0] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


CUTS = [(5, 6, 1), (9, 13, 2)]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = ri.rqc(4, 4, 16, seed=3)
    x1 = int(ri.random_bitstrings(16, 1, seed=2)[0])
    open_sites = [15, 14, 13]
    n = network.n_slices(c, CUTS)
    b, e = partition_slices(n, world, rank)
    part = np.zeros(8, dtype=complex)
    if e > b:
        part = network.amplitudes_sliced(c, x1, open_sites, CUTS, range(b, e))
    total = reduce_partials(torch.from_numpy(part))
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), total.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sum_equals_unsliced(tmp_path, world):
    port = _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    c = ri.rqc(4, 4, 16, seed=3)
    x1 = int(ri.random_bitstrings(16, 1, seed=2)[0])
    want = network.amplitudes_open(c, x1, [15, 14, 13])
    results = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for r in results:
        np.testing.assert_allclose(r, want, atol=1e-14)
        np.testing.assert_array_equal(r, results[0])    # every rank holds the same sum


# --- batch items of uneven cost: LPT over ranks ----------------------------------------

def test_lpt_classic_example():
    """Graham's tight case for two ranks: costs 3, 3, 2, 2, 2 give loads 7 and 5 (the best
    split is 6 and 6, and 7/6 is the LPT bound 4/3 - 1/6)."""
    assert partition_items([3, 3, 2, 2, 2], 2) == [[0, 2, 4], [1, 3]]
    assert partition_items([], 3) == [[], [], []]
    assert partition_items([5.0], 4) == [[0], [], [], []]
    with pytest.raises(ValueError):
        partition_items([1.0, -1.0], 2)


def test_lpt_covers_every_item_once_within_grahams_bound():
    rng = np.random.default_rng(11)
    for case in range(200):
        n, m = int(rng.integers(1, 9)), int(rng.integers(1, 5))
        costs = [float(c) for c in rng.integers(1, 50, size=n)]
        parts = partition_items(costs, m)
        assert len(parts) == m and sorted(i for p in parts for i in p) == list(range(n)), case
        assert parts == partition_items(costs, m), case          # deterministic
        span = max(sum(costs[i] for i in p) for p in parts)
        best = min(max(sum(c for c, r in zip(costs, a) if r == k) for k in range(m))
                   for a in itertools.product(range(m), repeat=n))
        assert span <= (4 / 3 - 1 / (3 * m)) * best + 1e-9, case


ITEMS = [(4, 4, 16, 3, 1, 3), (3, 4, 8, 5, 2, 2), (4, 5, 16, 7, 0, 4), (2, 5, 12, 9, 1, 1), (4, 4, 8, 11, 2, 2)]


def _items():
    """(circuit, x1 list, open sites) per item: uneven grids, depths and batch sizes."""
    out = []
    for rows, cols, depth, seed, n_open, n_x1 in ITEMS:
        c = ri.rqc(rows, cols, depth, seed=seed)
        n = rows * cols
        out.append((c, [int(x) for x in ri.random_bitstrings(n, n_x1, seed=seed)],
                    list(range(n - n_open, n))))
    return out


def _item_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1905_00444_gb300 as qfx   # host-only planning: the costs
    items = _items()
    plans = [(qfx.Plan(qfx.Circuit(c), open_sites=o), torch.zeros(len(xs), dtype=torch.int64), 0, None)
             for c, xs, o in items]
    mine = partition_items(item_costs(plans), world)[rank]
    rows = [np.zeros((len(xs), 1 << len(o)), dtype=complex) for _, xs, o in items]
    for i in mine:      # this rank's items; the others stay zero here
        c, xs, o = items[i]
        rows[i] = np.stack([network.amplitudes_open(c, x, o) for x in xs])
    flat = np.concatenate([r.reshape(-1) for r in rows])
    total = reduce_partials(torch.from_numpy(flat))
    np.save(os.path.join(out_dir, f"items{rank}.npy"), total.numpy())
    np.save(os.path.join(out_dir, f"mine{rank}.npy"), np.array(mine, dtype=np.int64))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_items_sharded_by_lpt_over_gloo_ranks(tmp_path):
    """Two ranks take the items LPT assigns them by planned cost (Eq. 1 flops x slices x
    bitstrings); each item's rows come from one rank and the rank-order sum assembles the
    whole batch, equal on every rank to the single-process result."""
    world = 2
    port = _free_port()
    mp.spawn(_item_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    want = np.concatenate([np.stack([network.amplitudes_open(c, x, o) for x in xs]).reshape(-1)
                           for c, xs, o in _items()])
    mine = [set(np.load(tmp_path / f"mine{r}.npy").tolist()) for r in range(world)]
    assert mine[0] and mine[1] and not (mine[0] & mine[1])
    assert mine[0] | mine[1] == set(range(len(ITEMS)))
    for r in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / f"items{r}.npy"), want)
