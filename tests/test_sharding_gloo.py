"""Multi-process sharding of slices (replicas, no data-path collective) on CPU ranks.

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

import rqc_inputs as ri
from oracle import network
from paper_1905_00444_gb300.sharding import partition_slices, reduce_partials


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
