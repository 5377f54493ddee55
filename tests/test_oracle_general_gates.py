"""Pins of the oracle for general (non-diagonal) two-qubit gates, kind U4.

A U4 gate G (4x4, G[2*o0 + o1, 2*i0 + i1]) becomes a bond leg of dimension 4 through
G = sum_k |o0><i0| (x) B_k, B_k[o1, i1] = G[2*o0 + o1, 2*i0 + i1], k = 2*o0 + i0.
- fSim closed forms: unitary, fSim(0, 0) = I, fSim(0, phi) = diag(1, 1, 1, e^-i phi),
  fSim(pi/2, 0) maps |01> to -i|10>.
- A single U4 gate on |00> of a 1x2 grid: amplitudes = G[:, 0] (network route, whose
  split must reproduce G); with H on both qubits first: G @ (1/2, 1/2, 1/2, 1/2).
- Dense matrix vs gate-by-gate state vector on fSim circuits (two independent routes).
- Network (split legs) vs state vector on fSim circuits: all outputs open, some open,
  closed.
- Slices over cuts that fix whole two-bit legs, or only their high bit, sum to the
  amplitude, and a half cut of a one-gate edge fixes that leg's high bit (o0).
- The stabilizer oracle's word for the Clifford gate fSim(pi/2, 0), multiplied out from
  textbook matrices, is that gate up to a phase; its probabilities on fSim(pi/2, 0)
  circuits match the state vector.
"""
import math

import numpy as np
import pytest

import rqc_inputs as ri
from oracle import dense, network, statevector


def test_fsim_closed_forms():
    for th, ph in [(0.3, 1.1), (math.pi / 2, math.pi / 6), (2.9, 5.0)]:
        g = ri.fsim(th, ph)
        np.testing.assert_allclose(g.conj().T @ g, np.eye(4), atol=1e-15)
    np.testing.assert_allclose(ri.fsim(0, 0), np.eye(4), atol=0)
    np.testing.assert_allclose(ri.fsim(0, 0.7), np.diag([1, 1, 1, np.exp(-0.7j)]), atol=1e-16)
    g = ri.fsim(math.pi / 2, 0)
    e01 = np.zeros(4); e01[1] = 1
    np.testing.assert_allclose(g @ e01, [0, 0, -1j, 0], atol=1e-16)


def one_gate_circuit(G, hadamards=False):
    gates = []
    layer = 0
    if hadamards:
        gates += [ri.Gate(0, 0, -1, ri.H, ri.MAT_H.copy()), ri.Gate(0, 1, -1, ri.H, ri.MAT_H.copy())]
        layer = 1
    gates.append(ri.Gate(layer, 0, 1, ri.U4, G))
    return ri.Circuit(1, 2, gates)


@pytest.mark.parametrize("hadamards", [False, True])
def test_single_general_gate_closed_form(hadamards):
    G = ri.random_complex((4, 4), seed=3).astype(np.complex128)   # any matrix, not unitary
    c = one_gate_circuit(G, hadamards)
    inp = np.full(4, 0.5) if hadamards else np.eye(4)[0]
    want = G @ inp                       # index 2*b(q0) + b(q1)
    # basis index of the state vector: bit q = qubit q, so x = b0 + 2*b1
    got = network.amplitudes_open(c, 0, [0, 1])        # output bit i = open site i
    for x in range(4):
        b0, b1 = x & 1, x >> 1
        assert abs(got[x] - want[2 * b0 + b1]) < 1e-14
    np.testing.assert_allclose(statevector.amplitudes(c)[[0, 1, 2, 3]],
                               [want[0], want[2], want[1], want[3]], atol=1e-14)


@pytest.mark.parametrize("shape", [(3, 3, 8), (2, 4, 12), (3, 2, 10)])
def test_dense_matches_statevector_fsim(shape):
    c = ri.rqc(*shape, seed=4, two_qubit="fsim")
    np.testing.assert_allclose(dense.amplitudes(c), statevector.amplitudes(c), atol=1e-13)


@pytest.mark.parametrize("shape,n_open", [((3, 3, 8), 9), ((3, 4, 8), 4), ((4, 3, 12), 0)])
def test_network_matches_statevector_fsim(shape, n_open):
    c = ri.rqc(*shape, seed=5, two_qubit="fsim")
    n = c.n_qubits
    psi = statevector.amplitudes(c)
    open_sites = list(range(n - n_open, n))
    for x1 in ri.random_bitstrings(n, 2, seed=6):
        got = network.amplitudes_open(c, int(x1), open_sites)
        idx = []
        for j in range(1 << n_open):
            x = int(x1)
            for i, q in enumerate(open_sites):
                x = (x & ~(1 << q)) | (((j >> i) & 1) << q)
            idx.append(x)
        np.testing.assert_allclose(got, psi[idx], atol=1e-13)


@pytest.mark.parametrize("cuts", [[(1, 2, 1)], [(1, 2, 2)], [(4, 5, 2), (1, 4, 4)], [(4, 7, 8)]])
def test_slices_of_two_bit_legs_sum_to_amplitude(cuts):
    c = ri.rqc(3, 3, 16, seed=7, two_qubit="fsim")      # two U4 gates per edge: 4 bond bits
    open_sites = [6, 7, 8]
    x1 = int(ri.random_bitstrings(9, 1, seed=8)[0])
    full = network.amplitudes_open(c, x1, open_sites)
    S = network.n_slices(c, cuts)
    parts = [network.amplitudes_sliced(c, x1, open_sites, cuts, [s]) for s in range(S)]
    np.testing.assert_allclose(np.sum(parts, axis=0), full, atol=1e-13)
    assert all(np.abs(p - full).max() > 1e-8 for p in parts)


def test_half_cut_fixes_high_bit_of_a_two_bit_leg():
    c = ri.rqc(2, 2, 8, seed=1, two_qubit="fsim")
    legs = network.bond_legs(c)[(0, 1)]
    assert len(legs) == 1
    assert network.n_slices(c, [(0, 1, 2)]) == 2
    assert network.slice_fixed_legs(c, [(0, 1, 2)], 1) == {legs[0]: (1, 1)}
    assert network.slice_fixed_legs(c, [(0, 1, 1)], 2) == {legs[0]: 2}


def test_stabilizer_word_is_fsim_pi2():
    """The tableau's gate word for fSim(pi/2, 0), multiplied out from the textbook H,
    S = diag(1, i) and CZ matrices, equals the gate up to a global phase."""
    from oracle import stabilizer
    H, S, I = ri.MAT_H, np.diag([1, 1j]), np.eye(2)
    one = {("h", 0): np.kron(H, I), ("h", 1): np.kron(I, H), ("s", 0): np.kron(S, I),
           ("s", 1): np.kron(I, S), ("cz",): np.diag([1, 1, 1, -1])}   # q0 = high factor
    m = np.eye(4, dtype=np.complex128)
    for op in stabilizer.FSIM_PI2_WORD:
        m = one[op] @ m
    g = ri.fsim(np.pi / 2, 0.0)
    phase = g[0, 0] / m[0, 0]
    assert abs(abs(phase) - 1) < 1e-12
    np.testing.assert_allclose(m * phase, g, atol=1e-12)


@pytest.mark.parametrize("shape", [(3, 3, 8), (4, 4, 12), (2, 5, 10)])
def test_stabilizer_matches_statevector_fsim_pi2(shape):
    from oracle import stabilizer
    c = ri.rqc(*shape, seed=13, gate_set=(ri.SQRT_X, ri.SQRT_Y), two_qubit="fsim_pi2")
    p = np.abs(statevector.amplitudes(c)) ** 2
    tab = stabilizer.prepare(c)
    xs = list(ri.random_bitstrings(c.n_qubits, 24, seed=5)) + [int(np.argmax(p))]
    for x in xs:
        assert abs(stabilizer.probability(c, int(x), tab) - p[int(x)]) < 1e-12
    assert np.count_nonzero(p > 1e-12) > 1      # not a product of basis states


def test_planted_swapped_leg_indices_are_caught(monkeypatch):
    """o0 and i0 exchanged in the split (a plausible slip): the closed form fails."""
    real = network.site_tensor

    def wrong(circuit, q, x_bit, fixed):
        c2 = circuit.copy()
        for g in c2.gates:
            m = np.asarray(g.mat)
            if m.size == 16:
                g.mat = m.reshape(2, 2, 2, 2).transpose(2, 1, 0, 3).reshape(4, 4)   # o0 <-> i0
        return real(c2, q, x_bit, fixed)

    monkeypatch.setattr(network, "site_tensor", wrong)
    with pytest.raises(AssertionError):
        test_single_general_gate_closed_form(True)


def test_random_circuits_network_slices_match_statevector():
    """Seeded random small grids (CZ or fSim), open sites and cuts (whole bonds or their
    high bits, which may split a 2-bit leg): the network route's slices sum to the state
    vector's amplitudes."""
    rng = np.random.default_rng(77)
    for case in range(30):
        rows, cols = int(rng.integers(1, 4)), int(rng.integers(2, 5))
        depth = int(rng.choice([4, 8, 12]))
        c = ri.rqc(rows, cols, depth, seed=100 + case,
                   two_qubit="fsim" if rng.random() < 0.5 else "cz")
        n = c.n_qubits
        psi = statevector.amplitudes(c)
        legs = network.bond_legs(c)
        edges = sorted(legs)
        cuts = []
        for k in rng.permutation(len(edges))[:int(rng.integers(0, 3))]:
            e = edges[k]
            m = sum(network.leg_bits(c.gates[g]) for g in legs[e])
            cuts.append((e[0], e[1], 1 << int(rng.integers(0, m))))
        open_sites = sorted(int(q) for q in rng.permutation(n)[:int(rng.integers(0, min(4, n) + 1))])
        x1 = int(ri.random_bitstrings(n, 1, seed=case)[0])
        S = network.n_slices(c, cuts)
        got = network.amplitudes_sliced(c, x1, open_sites, cuts, range(S))
        idx = []
        for j in range(1 << len(open_sites)):
            x = x1
            for i, q in enumerate(open_sites):
                x = (x & ~(1 << q)) | (((j >> i) & 1) << q)
            idx.append(x)
        np.testing.assert_allclose(got, psi[idx], atol=1e-12, err_msg=f"case {case}")
