"""General (non-diagonal) two-qubit gates, kind U4, through the CUDA path, against the
FP64 oracle.

fSim gates with random angles are split on the bond as G = sum_k |o0><i0| (x) B_k (a
leg of two bits per gate); the fold kernel applies the elementary matrix on q0 and the
block B_k on q1.  Tolerances are those of the CZ circuits: FP32 per amplitude
|a - a_ref| <= 1e-5 max(|a_ref|, 2^(-n/2)) and normwise 1e-5; BF16x3 the same bound.
"""
import numpy as np
import pytest

import rqc_inputs as ri
from oracle import network, stabilizer, statevector

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-5


def check(got, want, n, rel=REL):
    got, want = np.asarray(got).reshape(-1), np.asarray(want).reshape(-1)
    bound = rel * np.maximum(np.abs(want), 2.0 ** (-n / 2))
    err = np.abs(got - want)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.linalg.norm(got - want) <= rel * np.linalg.norm(want)


def expand(x1, open_sites, j):
    x = int(x1)
    for i, q in enumerate(open_sites):
        x = (x & ~(1 << q)) | (((j >> i) & 1) << q)
    return x


def gpu_amps(qfx, c, x1s, n_open, cuts=(), slices=None, precision="fp32"):
    plan = qfx.Plan(qfx.Circuit(c), n_open=n_open, cuts=cuts, precision=precision)
    x1 = torch.tensor(np.asarray(x1s, dtype=np.uint64).view(np.int64), device="cuda")
    ws = torch.empty(plan.workspace_bytes(2), dtype=torch.uint8, device="cuda")
    sb, se = (0, plan.n_slices) if slices is None else slices
    out = qfx.amplitudes(plan, x1, slice_begin=sb, slice_end=se, workspace=ws)
    qfx.sync()
    return plan, out.cpu().numpy()


@pytest.mark.parametrize("shape,n_open", [((3, 3, 8), 9), ((4, 4, 8), 4), ((4, 4, 16), 4),
                                          ((4, 5, 12), 3), ((2, 6, 16), 0), ((5, 4, 8), 5)])
def test_fsim_vs_statevector(qfx, shape, n_open):
    c = ri.rqc(*shape, seed=shape[2] + n_open, two_qubit="fsim")
    n = c.n_qubits
    psi = statevector.amplitudes(c)
    x1s = ri.random_bitstrings(n, 3, seed=2)
    plan, out = gpu_amps(qfx, c, x1s, n_open)
    want = np.array([[psi[expand(x1, plan.open_sites, j)] for j in range(1 << n_open)]
                     for x1 in x1s])
    check(out, want, n)


def test_fsim_slices_match_oracle_slice_by_slice(qfx):
    # 4 bond bits per edge; the cuts fix a whole 2-bit leg (size 4) and only the high bit
    # of a leg (size 2 of 16: 3 bits fixed)
    c = ri.rqc(3, 3, 16, seed=7, two_qubit="fsim")
    cuts = [(4, 5, 2), (1, 4, 4)]
    x1 = int(ri.random_bitstrings(9, 1, seed=8)[0])
    plan = qfx.Plan(qfx.Circuit(c), n_open=3, cuts=cuts)
    assert plan.n_slices == network.n_slices(c, cuts) == 8 * 4
    total = 0
    for s in range(plan.n_slices):
        _, out = gpu_amps(qfx, c, [x1], 3, cuts=cuts, slices=(s, s + 1))
        want = network.amplitudes_sliced(c, x1, plan.open_sites, cuts, [s])
        check(out, want, 9)
        total = total + out
    full = network.amplitudes_open(c, x1, plan.open_sites)
    check(total, full, 9)


def test_fsim_batch_matches_per_call(qfx):
    circs = [ri.rqc(4, 4, 16, seed=3, two_qubit="fsim"), ri.rqc(3, 5, 12, seed=4, two_qubit="fsim")]
    items, want = [], []
    for i, c in enumerate(circs):
        plan = qfx.Plan(qfx.Circuit(c), n_open=3, cuts=[(1, 2, 4)] if i else [])
        x1 = torch.tensor(ri.random_bitstrings(c.n_qubits, 3, seed=i).view(np.int64), device="cuda")
        items.append((plan, x1, 0, plan.n_slices))
        ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device="cuda")
        want.append(qfx.amplitudes(plan, x1, workspace=ws).cpu().numpy())
    b = qfx.Batch(items, slots=4)
    outs = b.run()
    qfx.sync()
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)


def test_fsim_tensor_core_steps(qfx):
    c = ri.rqc(4, 5, 16, seed=9, two_qubit="fsim")
    n = c.n_qubits
    psi = statevector.amplitudes(c)
    x1s = ri.random_bitstrings(n, 2, seed=3)
    plan, out = gpu_amps(qfx, c, x1s, 4, precision="bf16x3")
    assert any(s["variant"] >= 10 for s in plan.steps)
    want = np.array([[psi[expand(x1, plan.open_sites, j)] for j in range(16)] for x1 in x1s])
    check(out, want, n)


def test_7x7x16_fsim_clifford_probabilities_exact(qfx):
    """Full size with general gates: every two-qubit gate fSim(pi/2, 0) (Clifford, two bond
    bits), sqrt(X) / sqrt(Y) layers, so chi = 16 and the largest intermediate is 2^32
    elements as at 7x7x(1+32+1) with CZs; exact |amp|^2 per bitstring from the tableau."""
    c = ri.rqc(7, 7, 16, seed=11, gate_set=(ri.SQRT_X, ri.SQRT_Y), two_qubit="fsim_pi2")
    x1 = int(ri.random_bitstrings(49, 1, seed=12)[0])
    plan = qfx.Plan(qfx.Circuit(c), n_open=6)
    assert plan.stats["max_elements"] == 2 ** 32
    xt = torch.tensor(np.array([x1], dtype=np.uint64).view(np.int64), device="cuda")
    ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    out = qfx.amplitudes(plan, xt, workspace=ws)
    qfx.sync()
    got = np.abs(out[0].cpu().numpy())
    del ws
    tab = stabilizer.prepare(c)
    probs = np.array([stabilizer.probability(c, expand(x1, plan.open_sites, j), tab)
                      for j in range(64)])
    assert np.count_nonzero(probs) > 0
    floor = 2.0 ** (-49 / 2)
    assert np.all(np.abs(got - np.sqrt(probs)) <= REL * np.maximum(np.sqrt(probs), floor))
