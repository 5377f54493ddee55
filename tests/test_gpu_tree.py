"""Contraction-tree plans (plan family 1, the region plans of Sec. III / Fig. 3): a greedy
tree of TTGT steps with greedy cuts, run by the permute and step kernels.

* Small grids against the FP64 oracle, element by element (1e-5, floor 2^(-n/2)): the
  state vector (every output open), the network route with open sites, capped plans whose
  slices sum to the amplitude, general two-qubit gates, split-K nodes (a long contraction
  into a small result as side-by-side chunks and an FP64 sum).
* The benchmarked 7x7x(1+32+1) workload under the 12 stored vertical cuts: the tree plan
  contracts each slice with a different order and different kernels shapes than the line
  sweep (9.7e12 instead of 2.3e14 flop), and must match the stored FP64 slices.
* 7x7x(1+40+1), the paper's own shape, at an 8 GiB cap (2^20 slices instead of the line
  sweep's 2^59): a slice against its refinement (two finer slices sum to it).
* The tree plan inside a batch and through the allocation-free entry point.
* Split precisions: tensor-core nodes (chunked contractions added into the result) against
  the oracle on small grids and against the stored 7x7x32 slices, within the modes' bounds.
"""
import json
import os

import numpy as np
import pytest

import rqc_inputs as ri
from oracle import network, statevector

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rqc_7x7x32_slices.json")


def check(got, want, n, rel=REL):
    got, want = np.asarray(got).reshape(-1), np.asarray(want).reshape(-1)
    floor = 2.0 ** (-n / 2)
    err = np.abs(got - want)
    assert np.all(err <= rel * np.maximum(np.abs(want), floor)), float(np.max(err / np.maximum(np.abs(want), floor)))
    assert np.linalg.norm(got - want) <= rel * np.linalg.norm(want)


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.uint64).view(np.int64), device="cuda")


def expand(x1, open_sites, j):
    x = int(x1)
    for i, q in enumerate(open_sites):
        x = (x & ~(1 << q)) | (((j >> i) & 1) << q)
    return x


def run(qfx, plan, x1s, slices=None, items=1):
    ws = torch.empty(plan.workspace_bytes(items), dtype=torch.uint8, device="cuda")
    sb, se = slices or (0, plan.n_slices)
    out = qfx.amplitudes(plan, dev(x1s), slice_begin=sb, slice_end=se, workspace=ws)
    qfx.sync()
    return out.cpu().numpy()


def test_4x4x16_all_outputs_open_vs_state_vector(qfx):
    c = ri.rqc(4, 4, 16, seed=0)
    plan = qfx.Plan(qfx.Circuit(c), open_sites=list(range(16)), family="tree")
    out = run(qfx, plan, [0])
    check(out[0], statevector.amplitudes(c), 16)


@pytest.mark.parametrize("shape", [(5, 5, 24), (3, 5, 16), (6, 2, 16), (4, 5, 24)])
def test_shapes_vs_oracle(qfx, shape):
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=rows + cols)
    plan = qfx.Plan(qfx.Circuit(c), n_open=5, family="tree")
    x1s = ri.random_bitstrings(rows * cols, 3, seed=4)
    out = run(qfx, plan, x1s, items=2)
    want = np.array([network.amplitudes_open(c, int(x), plan.open_sites) for x in x1s])
    check(out, want, rows * cols)


def test_capped_tree_plan_slices_sum_to_the_amplitude(qfx):
    c = ri.rqc(6, 6, 24, seed=1)
    x1 = int(ri.random_bitstrings(36, 1, seed=5)[0])
    full = qfx.Plan(qfx.Circuit(c), n_open=6, family="tree")
    cap = full.stats["max_elements"] * 8 // 16
    plan = qfx.Plan(qfx.Circuit(c), n_open=6, max_intermediate_bytes=cap, family="tree")
    assert plan.n_slices > 1 and plan.stats["max_elements"] * 8 <= cap
    want = network.amplitudes_open(c, x1, plan.open_sites)
    check(run(qfx, plan, [x1], items=3)[0], want, 36)
    s = plan.n_slices // 2   # one slice against the oracle's slice
    got = run(qfx, plan, [x1], slices=(s, s + 1))[0]
    ref = network.amplitudes_sliced(c, x1, plan.open_sites, plan.cuts, [s])
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(4, 4, 32, 0), (4, 4, 32, 4), (4, 5, 32, 2)])
def test_split_k_nodes_vs_oracle(qfx, shape):
    # a long contraction into a small result (the root, typically) runs its 1024-long
    # chunks side by side and sums the partial products in FP64
    rows, cols, d, n_open = shape
    c = ri.rqc(rows, cols, d, seed=0)
    plan = qfx.Plan(qfx.Circuit(c), n_open=n_open, family="tree")
    split = [s for s in plan.steps if s["parts"] > 0]
    assert split and all(s["K"] == 1024 * s["parts"] for s in split)
    x1s = ri.random_bitstrings(rows * cols, 2, seed=8)
    out = run(qfx, plan, x1s, items=2)
    if rows * cols <= 16:
        psi = statevector.amplitudes(c)
        want = np.array([[psi[expand(x, plan.open_sites, j)] for j in range(1 << n_open)] for x in x1s])
    else:
        want = np.array([network.amplitudes_open(c, int(x), plan.open_sites) for x in x1s])
    check(out, want, rows * cols)


def test_general_two_qubit_gates(qfx):
    c = ri.rqc(4, 4, 8, seed=3, two_qubit="fsim")
    plan = qfx.Plan(qfx.Circuit(c), n_open=4, family="tree")
    x1s = ri.random_bitstrings(16, 2, seed=6)
    psi = statevector.amplitudes(c)
    want = np.array([[psi[expand(x, plan.open_sites, j)] for j in range(16)] for x in x1s])
    check(run(qfx, plan, x1s), want, 16)


def test_7x7x32_stored_slices_through_a_tree_plan(qfx):
    with open(GOLDEN) as f:
        g = json.load(f)
    c = ri.rqc(7, 7, 32, seed=0)
    plan = qfx.Plan(qfx.Circuit(c), n_open=6, cuts=[tuple(x) for x in g["cuts"]], family="tree")
    assert plan.open_sites == g["open_sites"] and plan.n_slices == int(g["n_slices"])
    top = max(s["norm"] for s in g["slices"])
    for s in g["slices"]:
        if s["norm"] < 1e-9 * top:
            continue
        sid = int(s["slice"])
        want = np.array(s["re"]) + 1j * np.array(s["im"])
        got = run(qfx, plan, [int(g["x1"])], slices=(sid, sid + 1))[0]
        rms = np.linalg.norm(want) / np.sqrt(want.size)
        assert np.all(np.abs(got - want) <= REL * np.maximum(np.abs(want), rms)), sid
        assert np.linalg.norm(got - want) <= REL * np.linalg.norm(want), sid


def _radices(c, cuts):
    legs = network.bond_legs(c)
    return [(1 << sum(network.leg_bits(c.gates[g]) for g in legs[(min(a, b), max(a, b))])) // size
            for a, b, size in cuts]


def _digits(sid, radices):
    out = []
    for r in reversed(radices):
        out.append(sid % r)
        sid //= r
    return out[::-1]


def _sid(digits, radices):
    s = 0
    for d, r in zip(digits, radices):
        s = s * r + d
    return s


def test_7x7x40_at_8_gib_slice_refinement(qfx):
    c = ri.rqc(7, 7, 40, seed=0)
    circ = qfx.Circuit(c)
    plan = qfx.Plan(circ, n_open=6, max_intermediate_bytes=8 << 30, family="tree")
    line = qfx.Plan(circ, n_open=6, max_intermediate_bytes=8 << 30)
    assert plan.n_slices <= 1 << 24 and line.n_slices >= 1 << 50
    assert plan.stats["max_elements"] * 8 <= 8 << 30
    # halve one cut whose finer plan keeps the same cut list within the cap
    for i, (qa, qb, size) in enumerate(plan.cuts):
        if size < 2:
            continue
        cuts = list(plan.cuts)
        cuts[i] = (qa, qb, size // 2)
        finer = qfx.Plan(circ, n_open=6, cuts=cuts, max_intermediate_bytes=8 << 30, family="tree")
        if finer.cuts == cuts:
            break
    else:
        pytest.fail("no cut can be halved within the cap")
    rc, rf = _radices(c, plan.cuts), _radices(c, cuts)
    assert rf[i] == 2 * rc[i] and finer.n_slices == 2 * plan.n_slices
    x1 = int(ri.random_bitstrings(49, 1, seed=2)[0])
    rng = np.random.default_rng(1)
    ws = torch.empty(max(plan.workspace_bytes(1), finer.workspace_bytes(1)), dtype=torch.uint8, device="cuda")
    for _ in range(6):    # first nonzero slice among a few seeded ones
        sid = int(rng.integers(0, plan.n_slices))
        coarse = qfx.amplitudes(plan, dev([x1]), slice_begin=sid, slice_end=sid + 1, workspace=ws).cpu().numpy()
        qfx.sync()
        rms = np.linalg.norm(coarse) / 8
        if rms > 0:
            break
    else:
        pytest.skip("no nonzero slice among the seeded ones")
    d = _digits(sid, rc)
    fine = 0
    for half in (0, 1):
        df = list(d)
        df[i] = 2 * d[i] + half
        f = _sid(df, rf)
        fine = fine + qfx.amplitudes(finer, dev([x1]), slice_begin=f, slice_end=f + 1, workspace=ws).cpu().numpy()
        qfx.sync()
    assert np.all(np.abs(fine - coarse) <= REL * np.maximum(np.abs(coarse), rms))


def test_tree_plan_in_a_batch_and_the_static_entry(qfx):
    c = ri.rqc(5, 5, 24, seed=2)
    tree = qfx.Plan(qfx.Circuit(c), n_open=4, family="tree")
    small = qfx.Plan(qfx.Circuit(ri.rqc(4, 4, 16, seed=1)), n_open=4)
    x1 = dev(ri.random_bitstrings(25, 2, seed=1))
    x2 = dev(ri.random_bitstrings(16, 2, seed=2))
    items = [(tree, x1, 0, None), (small, x2, 0, None)]
    want = [qfx.amplitudes(p, x).cpu().numpy() for p, x, _, _ in items]
    b = qfx.Batch(items, slots=2)
    outs = [o.cpu().numpy() for o in b.run()]
    qfx.sync()
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o, w)
    t2 = qfx.Plan(qfx.Circuit(ri.rqc(4, 5, 16, seed=3)), n_open=4, family="tree")
    assert t2.workspace_bytes(1) <= qfx.qfx.STATIC_SCRATCH_BYTES
    x3 = dev(ri.random_bitstrings(20, 3, seed=3))
    st = qfx.amplitudes_static(t2, x3).cpu().numpy()
    qfx.sync()
    np.testing.assert_array_equal(st, qfx.amplitudes(t2, x3).cpu().numpy())


BOUND = {"bf16x3": 1e-5, "tf32x3": 3e-5}


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_split_precision_tree_plans_vs_oracle(qfx, prec):
    c = ri.rqc(6, 6, 24, seed=4)
    plan = qfx.Plan(qfx.Circuit(c), n_open=6, family="tree", precision=prec)
    assert any(s["variant"] >= 10 for s in plan.steps)
    x1s = ri.random_bitstrings(36, 2, seed=7)
    out = run(qfx, plan, x1s, items=2)
    want = np.array([network.amplitudes_open(c, int(x), plan.open_sites) for x in x1s])
    check(out, want, 36, rel=BOUND[prec])


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_split_precision_tree_plan_on_the_stored_7x7x32_slices(qfx, prec):
    with open(GOLDEN) as f:
        g = json.load(f)
    c = ri.rqc(7, 7, 32, seed=0)
    plan = qfx.Plan(qfx.Circuit(c), n_open=6, cuts=[tuple(x) for x in g["cuts"]], family="tree",
                    precision=prec)
    assert any(s["variant"] >= 10 and s["K"] > 1024 for s in plan.steps)   # chunked tensor-core nodes
    top = max(s["norm"] for s in g["slices"])
    for s in g["slices"]:
        if s["norm"] < 1e-9 * top:
            continue
        sid = int(s["slice"])
        want = np.array(s["re"]) + 1j * np.array(s["im"])
        got = run(qfx, plan, [int(g["x1"])], slices=(sid, sid + 1))[0]
        rms = np.linalg.norm(want) / np.sqrt(want.size)
        assert np.all(np.abs(got - want) <= BOUND[prec] * np.maximum(np.abs(want), rms)), sid
