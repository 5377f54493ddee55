"""Batched persistent scheduler (qfx_batch_*): many work items of uneven shapes in one
launch must reproduce the per-item results exactly (same tile bodies, same FP64 order),
match the oracle, not depend on the number of slots, and replay from a CUDA graph."""
import numpy as np
import pytest

import rqc_inputs as ri
from oracle import network

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def mixed_items(qfx):
    specs = [  # (rows, cols, depth, seed, n_open, cuts, n_x1)
        (4, 4, 16, 0, 5, [], 3),
        (5, 5, 24, 1, 4, [(6, 7, 4)], 2),
        (6, 6, 24, 2, 3, [(14, 15, 2)], 2),
        (3, 5, 16, 3, 6, [], 4),
        (2, 2, 3, 4, 2, [], 1),
    ]
    items, circuits = [], []
    for rows, cols, d, seed, no, cuts, nx in specs:
        c = ri.rqc(rows, cols, d, seed=seed)
        plan = qfx.Plan(qfx.Circuit(c), n_open=no, cuts=cuts)
        x1 = torch.tensor(ri.random_bitstrings(rows * cols, nx, seed=seed + 50).view(np.int64),
                          device="cuda")
        items.append((plan, x1, 0, None))
        circuits.append(c)
    return items, circuits


def check_amps(got, want, n, rel):
    """Per amplitude against max(|ref|, 2^(-n/2)), and normwise."""
    floor = 2.0 ** (-n / 2)
    assert np.all(np.abs(got - want) <= rel * np.maximum(np.abs(want), floor))
    assert np.linalg.norm(got - want) <= rel * np.linalg.norm(want)


def per_item(qfx, items):
    outs = []
    for plan, x1, sb, se in items:
        ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device="cuda")
        outs.append(qfx.amplitudes(plan, x1, slice_begin=sb,
                                   slice_end=plan.n_slices if se is None else se,
                                   workspace=ws).cpu().numpy())
    qfx.sync()
    return outs


@pytest.mark.parametrize("slots", [1, 3, 16])
def test_mixed_batch_matches_per_item(qfx, slots):
    items, circuits = mixed_items(qfx)
    want = per_item(qfx, items)
    b = qfx.Batch(items, slots=slots)
    outs = b.run()
    qfx.sync()
    assert b.n_work == sum(x1.numel() * plan.n_slices for plan, x1, _, _ in items)
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)
    # and one item against the oracle
    plan, x1, _, _ = items[2]
    for r, x in enumerate(x1.cpu().numpy().view(np.uint64)):
        ref = network.amplitudes_open(circuits[2], int(x), plan.open_sites)
        check_amps(outs[2][r].cpu().numpy(), ref, circuits[2].n_qubits, 1e-5)


def test_batch_replays_from_cuda_graph(qfx):
    items, _ = mixed_items(qfx)
    want = per_item(qfx, items)
    b = qfx.Batch(items, slots=4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(stream=s)            # warm-up outside capture
    torch.cuda.synchronize()
    for o in b.outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(stream=s)
    for _ in range(2):
        for o in b.outs:
            o.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        qfx.sync()
        for o, w in zip(b.outs, want):
            np.testing.assert_array_equal(o.cpu().numpy(), w)


def test_sampled_paths_of_a_capped_plan(qfx):
    """Path subsampling (Sec. III.C): a seeded sample of slices of a 7x7x(1+24+1) plan cut
    down to a 4 MiB per-item cap, each slice a separate batch item."""
    c = ri.rqc(7, 7, 24, seed=5)
    plan = qfx.Plan(qfx.Circuit(c), n_open=4, max_intermediate_bytes=4 << 20)
    assert plan.n_slices >= 64
    rng = np.random.default_rng(3)
    sample = sorted(set(int(v) for v in rng.integers(0, plan.n_slices, size=64)))
    x1 = torch.tensor(ri.random_bitstrings(49, 1, seed=8).view(np.int64), device="cuda")
    items = [(plan, x1, s, s + 1) for s in sample]
    want = per_item(qfx, items)
    b = qfx.Batch(items, slots=8)
    outs = b.run()
    qfx.sync()
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)


def mixed_tc_items(qfx):
    specs = [  # (rows, cols, depth, seed, n_open, cuts, n_x1, precision)
        (4, 4, 16, 0, 5, [], 3, "bf16x3"),
        (5, 5, 24, 1, 4, [(6, 7, 4)], 2, "bf16x3"),
        (6, 6, 24, 2, 3, [(14, 15, 2)], 2, "tf32x3"),
        (3, 5, 16, 3, 6, [], 4, "bf16x3"),
    ]
    items, circuits = [], []
    for rows, cols, d, seed, no, cuts, nx, prec in specs:
        c = ri.rqc(rows, cols, d, seed=seed)
        plan = qfx.Plan(qfx.Circuit(c), n_open=no, cuts=cuts, precision=prec)
        x1 = torch.tensor(ri.random_bitstrings(rows * cols, nx, seed=seed + 50).view(np.int64),
                          device="cuda")
        items.append((plan, x1, 0, None))
        circuits.append(c)
    return items, circuits


@pytest.mark.parametrize("slots", [1, 3, 16])
def test_split_precision_batch_graph_matches_per_item(qfx, slots):
    """Items with tensor-core steps run as per-item launch sequences over parallel lanes of
    one CUDA graph, the split-precision items whose steps all take FP32 tiles (4x4x16,
    3x5x16) in the persistent kernel recorded in the same graph: outputs equal per-item
    qfx_amplitudes bit for bit, whatever the number of lanes."""
    items, circuits = mixed_tc_items(qfx)
    n_tc = sum(any(s["variant"] >= 10 for s in p.steps) for p, _, _, _ in items)
    assert n_tc == 2
    want = per_item(qfx, items)
    b = qfx.Batch(items, slots=slots)
    assert b.slots == min(slots, n_tc)
    outs = b.run()
    qfx.sync()
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)
    plan, x1, _, _ = items[2]   # TF32x3 item against the oracle, within its stated bound
    for r, x in enumerate(x1.cpu().numpy().view(np.uint64)):
        ref = network.amplitudes_open(circuits[2], int(x), plan.open_sites)
        check_amps(outs[2][r].cpu().numpy(), ref, circuits[2].n_qubits, 3e-5)


def test_split_precision_batch_replays_inside_a_cuda_graph(qfx):
    items, _ = mixed_tc_items(qfx)
    want = per_item(qfx, items)
    b = qfx.Batch(items, slots=4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(stream=s)
    for _ in range(2):
        for o in b.outs:
            o.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        qfx.sync()
        for o, w in zip(b.outs, want):
            np.testing.assert_array_equal(o.cpu().numpy(), w)


def test_small_split_precision_items_in_one_persistent_launch(qfx):
    """Split-precision plans whose step shapes the tensor-core tile does not take (bond
    dimension 4) are FP32-tile items: a batch of them is ONE persistent kernel launch,
    bit-identical to per-item launches of the same plans."""
    items = []
    for rows, cols, seed, no, nx in [(4, 4, 20, 5, 3), (3, 5, 21, 6, 2), (4, 4, 22, 3, 4)]:
        c = ri.rqc(rows, cols, 16, seed=seed)
        plan = qfx.Plan(qfx.Circuit(c), n_open=no, precision="bf16x3")
        assert all(st["variant"] < 10 for st in plan.steps)
        x1 = torch.tensor(ri.random_bitstrings(rows * cols, nx, seed=seed).view(np.int64),
                          device="cuda")
        items.append((plan, x1, 0, None))
    want = per_item(qfx, items)
    b = qfx.Batch(items, slots=4)
    before = qfx.launch_count()
    outs = b.run()
    assert qfx.launch_count() - before == 1
    qfx.sync()
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)


def test_fp32_items_in_a_split_precision_batch(qfx):
    """An FP32 plan mixed with tensor-core plans (it joins the persistent launch beside
    the lanes) keeps its FP32 result."""
    items, _ = mixed_tc_items(qfx)
    c = ri.rqc(4, 5, 16, seed=9)
    plan = qfx.Plan(qfx.Circuit(c), n_open=4)
    x1 = torch.tensor(ri.random_bitstrings(20, 2, seed=3).view(np.int64), device="cuda")
    items.append((plan, x1, 0, None))
    want = per_item(qfx, items)
    b = qfx.Batch(items, slots=2)
    outs = b.run()
    qfx.sync()
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)


def test_large_fp32_items_run_as_launches_beside_the_persistent_kernel(qfx):
    """FP32 items whose steps have at least 512 output tiles (7x7x(1+24+1): 1024) run as
    their own launch sequences in the batch's graph; the small items run in one persistent
    launch recorded in the same graph.  Outputs equal per-item qfx_amplitudes bit for bit,
    also when the batch is replayed from a caller's CUDA graph."""
    items, _ = mixed_items(qfx)
    c = ri.rqc(7, 7, 24, seed=7)
    big = qfx.Plan(qfx.Circuit(c), n_open=5)
    x1 = torch.tensor(ri.random_bitstrings(49, 2, seed=4).view(np.int64), device="cuda")
    items = [items[0], (big, x1, 0, None)] + items[1:] + [(big, x1[1:], 0, None)]
    want = per_item(qfx, items)
    b = qfx.Batch(items, slots=3)
    assert b.n_work == sum(x.numel() * p.n_slices for p, x, _, _ in items)
    outs = b.run()
    qfx.sync()
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(stream=s)
    for o in b.outs:
        o.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    qfx.sync()
    for o, w in zip(b.outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)
