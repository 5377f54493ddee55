"""Adjoint contraction (qfx_amplitudes_backward, CircuitAmplitudes) against the FP64 oracle.

The oracle's gradient is computed by linearity (each amplitude is linear in each gate's
entries) and is itself pinned to finite differences on the CPU.  The GPU path runs the
forward and reverse sweeps in FP32; gradients must match to 1e-4 relative (normwise over
the compared entries, and per entry with a floor of 1e-3 of the largest entry).
"""
import numpy as np
import pytest

import rqc_inputs as ri
from oracle import gradient, network

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-4


def gates_tensor(c):
    rows = [np.asarray(g.mat).reshape(-1) for g in c.gates]
    return torch.tensor(np.stack(rows), dtype=torch.complex128)


def gpu_grads(qfx, c, x1s, *, n_open=0, open_sites=None, cuts=(), gbar=None, store=0, entries=4):
    plan = qfx.Plan(qfx.Circuit(c), n_open=n_open, open_sites=open_sites, cuts=cuts,
                    adjoint_store_bytes=store)
    x1 = torch.tensor(np.asarray(x1s, dtype=np.uint64).view(np.int64), device="cuda")
    ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    amp = qfx.amplitudes(plan, x1, workspace=ws)
    g = 2 * amp if gbar is None else torch.as_tensor(gbar, device="cuda")
    out = qfx.amplitudes_backward(plan, x1, g, entries=entries)
    qfx.sync()
    return plan, amp.cpu().numpy(), out.cpu().numpy()


def oracle_grads(c, x1s, open_sites, entries, gbar=None):
    """sum over x1 of sum_o gbar[b,o] conj(d amp[b,o] / d G[entry])."""
    out = np.zeros(len(entries), dtype=complex)
    for b, x1 in enumerate(x1s):
        amps = network.amplitudes_open(c, int(x1), open_sites)
        gb = 2 * amps if gbar is None else gbar[b]
        for i, (gi, e) in enumerate(entries):
            d = gradient.amplitude_derivative(c, gi, e, int(x1), open_sites)
            out[i] += np.sum(gb * np.conj(d))
    return out


def compare(got, want, rel=REL):
    got, want = np.asarray(got), np.asarray(want)
    nw = np.linalg.norm(got - want) / np.linalg.norm(want)
    floor = 1e-3 * np.max(np.abs(want))
    per = np.max(np.abs(got - want) / np.maximum(np.abs(want), floor))
    print(f"gradient error: normwise {nw:.2e}, per entry {per:.2e}")
    assert nw <= rel and per <= 10 * rel, (nw, per)


def all_entries(c):
    return [(gi, e) for gi, g in enumerate(c.gates) for e in range(np.asarray(g.mat).size)]


@pytest.mark.parametrize("shape", [(2, 3, 8), (3, 3, 8), (3, 2, 9)])
def test_all_gate_entries_small(qfx, shape):
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=rows * 7 + d, parametrised=True)
    x1s = ri.random_bitstrings(rows * cols, 2, seed=3)
    plan, amp, g = gpu_grads(qfx, c, x1s, n_open=2)
    entries = all_entries(c)
    want = oracle_grads(c, x1s, plan.open_sites, entries)
    got = np.array([g[gi, e] for gi, e in entries])
    compare(got, want)


@pytest.mark.parametrize("shape", [(3, 3, 8), (2, 4, 12)])
def test_general_two_qubit_gates_all_entries(qfx, shape):
    """fSim (U4) gates: all 16 entries per gate, with the block of the gate's q1 event
    mapped back to G[r][c]; single-qubit gates alongside."""
    c = ri.rqc(*shape, seed=shape[2], parametrised=True, two_qubit="fsim")
    x1s = ri.random_bitstrings(c.n_qubits, 2, seed=3)
    plan, amp, g = gpu_grads(qfx, c, x1s, n_open=2, entries=16)
    entries = all_entries(c)
    assert sum(1 for gi, e in entries if e >= 4) > 0
    want = oracle_grads(c, x1s, plan.open_sites, entries)
    got = np.array([g[gi, e] for gi, e in entries])
    compare(got, want)


def test_sixteen_entries_extend_the_four_on_diagonal_gates(qfx):
    c = ri.rqc(3, 4, 16, seed=4, parametrised=True)
    x1s = ri.random_bitstrings(12, 2, seed=2)
    _, _, g4 = gpu_grads(qfx, c, x1s, n_open=2)
    _, _, g16 = gpu_grads(qfx, c, x1s, n_open=2, entries=16)
    assert np.array_equal(g16[:, :4], g4)
    assert not np.any(g16[:, 4:])


def test_general_upstream_gradient(qfx):
    c = ri.rqc(3, 3, 8, seed=5, parametrised=True)
    x1s = ri.random_bitstrings(9, 3, seed=4)
    gbar = ri.random_complex((3, 4), seed=7).astype(np.complex128)
    plan, amp, g = gpu_grads(qfx, c, x1s, n_open=2, gbar=gbar)
    entries = all_entries(c)
    want = oracle_grads(c, x1s, plan.open_sites, entries, gbar=gbar)
    got = np.array([g[gi, e] for gi, e in entries])
    compare(got, want)


def test_rqc_fixed_gates_and_cz_diagonals(qfx):
    # the standard gate set, including gradients of every CZ's diagonal
    c = ri.rqc(3, 4, 16, seed=2)
    x1s = ri.random_bitstrings(12, 1, seed=1)
    plan, amp, g = gpu_grads(qfx, c, x1s, n_open=3)
    entries = all_entries(c)
    want = oracle_grads(c, x1s, plan.open_sites, entries)
    got = np.array([g[gi, e] for gi, e in entries])
    compare(got, want)


def test_gradients_sum_over_slices(qfx):
    c = ri.rqc(3, 4, 16, seed=4, parametrised=True)
    x1s = ri.random_bitstrings(12, 2, seed=2)
    _, _, g0 = gpu_grads(qfx, c, x1s, n_open=2)
    _, _, g1 = gpu_grads(qfx, c, x1s, n_open=2, cuts=[(5, 6, 1), (1, 5, 2)])
    assert np.linalg.norm(g1 - g0) / np.linalg.norm(g0) < 1e-5


@pytest.mark.parametrize("shape", [(3, 4, 16), (5, 4, 16)])
def test_line_checkpoints_match_stored_boundaries(qfx, shape):
    """Keeping every step's output and recomputing each line from its checkpoint run the
    same kernels on the same inputs: the gradients are bit-identical, and the recomputing
    run needs less workspace."""
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=11, parametrised=True)
    x1s = ri.random_bitstrings(rows * cols, 2, seed=5)
    full, _, g_full = gpu_grads(qfx, c, x1s, n_open=3)
    line, _, g_line = gpu_grads(qfx, c, x1s, n_open=3, store=1)
    assert full.backward_workspace_bytes() > line.backward_workspace_bytes()
    assert np.array_equal(g_full, g_line)
    entries = all_entries(c)[:40]
    want = oracle_grads(c, x1s, full.open_sites, entries)
    compare(np.array([g_line[gi, e] for gi, e in entries]), want)


def test_6x6x24_parametrised_128_bitstrings(qfx):
    """Config: 6x6 grid, depth 1+24+1, parametrised single-qubit gates, L = sum over 128
    bitstrings (|x2| = 7) of |amp|^2; 64 seeded gate entries against the oracle."""
    c = ri.rqc(6, 6, 24, seed=0, parametrised=True)
    x1s = ri.random_bitstrings(36, 1, seed=9)
    plan, amp, g = gpu_grads(qfx, c, x1s, n_open=7)
    assert amp.shape == (1, 128)
    rng = np.random.default_rng(0)
    entries = []
    for gi in rng.choice(len(c.gates), size=64, replace=False):
        entries.append((int(gi), int(rng.integers(np.asarray(c.gates[gi].mat).size))))
    want = oracle_grads(c, x1s, plan.open_sites, entries)
    got = np.array([g[gi, e] for gi, e in entries])
    compare(got, want)


def test_6x6x24_finite_differences_through_gpu(qfx):
    """Central differences (step 1e-3, on Re and Im) of the GPU loss agree with the GPU
    adjoint to the precision FP32 amplitudes allow."""
    c = ri.rqc(6, 6, 24, seed=0, parametrised=True)
    x1s = ri.random_bitstrings(36, 1, seed=9)
    plan, amp, g = gpu_grads(qfx, c, x1s, n_open=7)
    x1 = torch.tensor(x1s.view(np.int64), device="cuda")
    h = 1e-3

    def loss(circ):
        p = qfx.Plan(qfx.Circuit(circ), n_open=7)
        a = qfx.amplitudes(p, x1)
        qfx.sync()
        return float(torch.sum(torch.abs(a) ** 2).item())

    rng = np.random.default_rng(1)
    for gi in rng.choice([i for i, gg in enumerate(c.gates) if gg.q1 < 0], size=4, replace=False):
        e = int(rng.integers(4))
        fd = []
        for delta in (h, 1j * h):
            cp, cm = c.copy(), c.copy()
            cp.gates[gi].mat.reshape(-1)[e] += delta
            cm.gates[gi].mat.reshape(-1)[e] -= delta
            fd.append((loss(cp) - loss(cm)) / (2 * h))
        fdv = complex(fd[0], fd[1])
        assert abs(fdv - g[gi, e]) <= 2e-2 * max(abs(g[gi, e]), 1e-3 * np.abs(g).max())


def test_autograd_function(qfx):
    c = ri.rqc(3, 3, 8, seed=1, parametrised=True)
    x1 = torch.tensor(ri.random_bitstrings(9, 2, seed=5).view(np.int64), device="cuda")
    gates = gates_tensor(c).requires_grad_(True)
    amp = qfx.circuit_amplitudes(gates, c, x1, n_open=2)
    loss = torch.sum(torch.abs(amp) ** 2)
    loss.backward()
    plan, _, g = gpu_grads(qfx, c, ri.random_bitstrings(9, 2, seed=5), n_open=2)
    np.testing.assert_allclose(gates.grad.numpy(), g, rtol=1e-12, atol=1e-20)
    # and torch's own gradient check of the convention on one entry: d loss / d Re(G)
    entries = [(3, 1)]
    want = oracle_grads(c, ri.random_bitstrings(9, 2, seed=5), plan.open_sites, entries)
    assert abs(gates.grad[3, 1].item() - want[0]) <= REL * abs(want[0]) + 1e-12
