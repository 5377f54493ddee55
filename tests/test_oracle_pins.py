"""Pins of the CPU FP64 oracle against closed forms, brute force and independent routes.

None of these runs a GPU.  Each pin is chosen so that a plausible slip in the oracle
(a transposed gate, a dropped CZ, a wrong bit order, a wrong bond split) fails it.
"""
import json
import math
import os

import numpy as np
import pytest

import rqc_inputs as ri
from oracle import dense, gradient, network, primitives, stabilizer, statevector

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KIND = {"H": ri.H, "T": ri.T, "SQRT_X": ri.SQRT_X, "SQRT_Y": ri.SQRT_Y, "CZ": ri.CZ}
FIXED = {ri.H: ri.MAT_H, ri.T: ri.MAT_T, ri.SQRT_X: ri.MAT_SQRT_X, ri.SQRT_Y: ri.MAT_SQRT_Y}


def _golden_circuit(case):
    gates = []
    for layer, kind, q0, q1 in case["gates"]:
        k = KIND[kind]
        mat = ri.DIAG_CZ.copy() if k == ri.CZ else FIXED[k].copy()
        gates.append(ri.Gate(layer, q0, q1, k, mat))
    return ri.Circuit(1, case["n"], gates)


def _golden_cases():
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_closed_forms_all_routes(case):
    c = _golden_circuit(case)
    want = np.array(case["amps_re"]) + 1j * np.array(case["amps_im"])
    np.testing.assert_allclose(dense.amplitudes(c), want, atol=1e-15)
    np.testing.assert_allclose(statevector.amplitudes(c), want, atol=1e-15)
    n = case["n"]
    net = np.array([network.amplitudes_open(c, 0, list(range(n)))]).reshape(-1)
    np.testing.assert_allclose(net, want, atol=1e-15)


def test_gate_matrices_unitary_and_roots():
    for m in (ri.MAT_H, ri.MAT_SQRT_X, ri.MAT_SQRT_Y, ri.MAT_T):
        np.testing.assert_allclose(m @ m.conj().T, np.eye(2), atol=1e-15)
    X = np.array([[0, 1], [1, 0]])
    Y = np.array([[0, -1j], [1j, 0]])
    np.testing.assert_allclose(ri.MAT_SQRT_X @ ri.MAT_SQRT_X, X, atol=1e-15)
    np.testing.assert_allclose(ri.MAT_SQRT_Y @ ri.MAT_SQRT_Y, Y, atol=1e-15)


def test_patterns_cover_each_edge_once():
    for rows, cols in [(4, 4), (7, 7), (5, 6), (2, 3)]:
        seen = []
        for p in range(8):
            es = ri.grid_pattern_edges(rows, cols, p)
            qs = [q for e in es for q in e]
            assert len(qs) == len(set(qs)), "pattern must be a matching"
            seen += es
        c = ri.Circuit(rows, cols, [])
        assert sorted(seen) == sorted(c.edges())


@pytest.mark.parametrize("shape", [(2, 3, 8), (3, 3, 8), (1, 4, 5), (3, 2, 9)])
def test_statevector_matches_dense(shape):
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=rows * 10 + d)
    np.testing.assert_allclose(statevector.amplitudes(c), dense.amplitudes(c), atol=1e-13)


def test_product_state_closed_form():
    c = ri.product_circuit(3, 3, 12, seed=5)
    amps = statevector.amplitudes(c)
    per = []
    for q in range(c.n_qubits):
        v = np.array([1.0, 0.0], dtype=complex)
        for g in sorted([g for g in c.gates if g.q0 == q], key=lambda g: g.layer):
            v = g.mat @ v
        per.append(v)
    for x in range(1 << c.n_qubits):
        want = np.prod([per[q][(x >> q) & 1] for q in range(c.n_qubits)])
        assert abs(amps[x] - want) < 1e-14


def test_identity_cycles_give_delta():
    # depth 0: H then H on every qubit -> amp = delta(x, 0)
    c = ri.rqc(3, 3, 0)
    amps = statevector.amplitudes(c)
    want = np.zeros(1 << 9)
    want[0] = 1.0
    np.testing.assert_allclose(amps, want, atol=1e-15)
    np.testing.assert_allclose(network.amplitudes_open(c, 0, list(range(9))), want, atol=1e-15)


@pytest.mark.parametrize("shape", [(2, 2), (3, 3), (3, 4)])
def test_ghz_closed_form(shape):
    c = ri.ghz_snake(*shape)
    n = c.n_qubits
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[(1 << n) - 1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(statevector.amplitudes(c), want, atol=1e-14)
    np.testing.assert_allclose(network.amplitudes_open(c, 0, list(range(n))), want, atol=1e-14)


def test_clifford_rqc_support():
    c = ri.rqc(4, 4, 16, seed=3, gate_set=(ri.SQRT_X, ri.SQRT_Y))
    p = np.abs(statevector.amplitudes(c)) ** 2
    nz = p[p > 1e-12]
    k = round(-math.log2(nz[0]))
    np.testing.assert_allclose(nz, 2.0 ** -k, rtol=1e-10)
    assert nz.size == 2 ** k
    assert abs(p.sum() - 1) < 1e-12


def test_norm_and_mean_4x4x16():
    c = ri.rqc(4, 4, 16, seed=0)
    p = np.abs(statevector.amplitudes(c)) ** 2
    assert abs(p.sum() - 1.0) < 1e-12                      # sum |amp|^2 = 1
    assert abs(p.mean() - 2.0 ** -16) < 1e-12 * 2.0 ** -16  # mean = 2^-n (Sec. III.E)


@pytest.mark.parametrize("shape", [(2, 2, 8), (2, 3, 16), (3, 3, 8), (3, 4, 8), (4, 3, 9)])
def test_network_matches_statevector_all_open(shape):
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=d + rows)
    n = c.n_qubits
    want = statevector.amplitudes(c)
    got = network.amplitudes_open(c, 0, list(range(n)))
    np.testing.assert_allclose(got, want, atol=1e-13)


def test_network_4x4x16_partial_open_sites():
    c = ri.rqc(4, 4, 16, seed=1)
    psi = statevector.amplitudes(c)
    x1s = ri.random_bitstrings(16, 3, seed=9)
    open_sites = [15, 14, 13, 12, 11]
    for x1 in x1s:
        got = network.amplitudes_open(c, int(x1), open_sites)
        for j in range(1 << len(open_sites)):
            x = int(x1)
            for i, q in enumerate(open_sites):
                x = (x & ~(1 << q)) | (((j >> i) & 1) << q)
            assert abs(got[j] - psi[x]) < 1e-13


def test_network_closed_bitstrings():
    c = ri.rqc(3, 4, 16, seed=2)
    psi = statevector.amplitudes(c)
    xs = ri.random_bitstrings(12, 6, seed=4)
    np.testing.assert_allclose(network.amplitudes(c, xs), psi[xs.astype(np.int64)], atol=1e-13)


def test_slicing_is_exact():
    c = ri.rqc(3, 4, 16, seed=7)
    x1 = int(ri.random_bitstrings(12, 1, seed=3)[0])
    open_sites = [11, 10]
    full = network.amplitudes_open(c, x1, open_sites)
    cuts = [(1, 2, 1), (5, 9, 2)]                     # one whole bond, one bond in halves
    ns = network.n_slices(c, cuts)
    assert ns == 4 * 2
    parts = [network.amplitudes_sliced(c, x1, open_sites, cuts, [s]) for s in range(ns)]
    np.testing.assert_allclose(np.sum(parts, axis=0), full, atol=1e-14)
    # each slice is a genuine fraction: no single slice equals the total
    assert all(np.abs(p - full).max() > 1e-6 for p in parts)


def test_slice_bond_index_convention():
    # slice d of a whole-bond cut fixes leg j (time order) to bit (m-1-j) of d
    c = ri.rqc(2, 2, 16, seed=1)
    legs = network.bond_legs(c)[(0, 1)]
    assert len(legs) == 2
    f = network.slice_fixed_legs(c, [(0, 1, 1)], 2)
    assert f == {legs[0]: 1, legs[1]: 0}
    f = network.slice_fixed_legs(c, [(0, 1, 2)], 1)   # halves: only the first leg fixed
    assert f == {legs[0]: 1}


@pytest.mark.parametrize("shape", [(3, 3, 12), (4, 4, 16), (2, 5, 10)])
def test_stabilizer_matches_statevector(shape):
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=11, gate_set=(ri.SQRT_X, ri.SQRT_Y))
    p = np.abs(statevector.amplitudes(c)) ** 2
    tab = stabilizer.prepare(c)
    xs = list(ri.random_bitstrings(c.n_qubits, 24, seed=5)) + [int(np.argmax(p))]
    for x in xs:
        assert abs(stabilizer.probability(c, int(x), tab) - p[int(x)]) < 1e-12


def test_stabilizer_ghz():
    c = ri.ghz_snake(7, 7)
    tab = stabilizer.prepare(c)
    assert stabilizer.probability(c, 0, tab) == 0.5
    assert stabilizer.probability(c, (1 << 49) - 1, tab) == 0.5
    assert stabilizer.probability(c, 1, tab) == 0.0


def test_gradient_linearity_matches_finite_difference():
    c = ri.rqc(2, 3, 8, seed=4, parametrised=True)
    open_sites = [5, 4]
    x1 = 0b010011
    rng = np.random.default_rng(0)
    entries = []
    for gi in rng.choice(len(c.gates), size=8, replace=False):
        entries.append((int(gi), int(rng.integers(c.gates[gi].mat.size))))
    lin = gradient.grad_entries(c, x1, open_sites, entries)
    for (gi, e), g in zip(entries, lin):
        fd = gradient.finite_difference(c, x1, open_sites, gi, e, h=1e-4)
        assert abs(fd - g) < 1e-7 * max(1.0, abs(g)), (gi, e, fd, g)


def test_gradient_linearity_matches_dense():
    # derivative by linearity equals the dense-matrix derivative of one entry
    c = ri.rqc(2, 2, 4, seed=3)
    gi = next(i for i, g in enumerate(c.gates) if g.q1 >= 0)
    for e in range(4):
        d_lin = gradient.amplitude_derivative(c, gi, e, 0, [0, 1, 2, 3])
        c2 = c.copy()
        m = np.zeros(4, dtype=complex)
        m[e] = 1.0
        c2.gates[gi].mat = m
        np.testing.assert_allclose(d_lin, dense.amplitudes(c2), atol=1e-14)


def test_contract_step_brute_force():
    rng = np.random.default_rng(1)
    P, K, N, Sd = 3, 4, 5, 2
    S = rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))
    B = rng.standard_normal((P, K, Sd)) + 1j * rng.standard_normal((P, K, Sd))
    C = primitives.contract_step(S, B, P, K, N, Sd)
    for p in range(P):
        for n in range(N):
            for s in range(Sd):
                acc = 0j
                for k in range(K):
                    acc += S[k, n] * B[p, k, s]
                assert abs(C[p, n, s] - acc) < 1e-13


def test_permute_brute_force():
    x = np.arange(2 * 3 * 4).astype(complex)
    out = primitives.permute(x, (2, 3, 4), (2, 0, 1))
    assert out.shape == (4, 2, 3)
    for a in range(2):
        for b in range(3):
            for d in range(4):
                assert out[d, a, b] == x[a * 12 + b * 4 + d]


def test_flops_eq1_is_8mnk():
    # v0 = M*K, v1 = K*N, v2 = M*N  ->  8 sqrt(v0 v1 v2) = 8 M N K
    for (m, n, k) in [(256, 256, 256), (1 << 24, 256, 256), (16, 1, 4)]:
        assert primitives.flops_eq1(m * k, k * n, m * n) == pytest.approx(8.0 * m * n * k, rel=1e-12)


# --- planted mistakes: each must be caught by a pin above -----------------------

def test_planted_transposed_gate_is_caught(monkeypatch):
    orig = statevector.apply_1q
    monkeypatch.setattr(statevector, "apply_1q", lambda psi, n, q, g: orig(psi, n, q, g.T))
    c = ri.rqc(2, 3, 8, seed=3)
    assert np.abs(statevector.amplitudes(c) - dense.amplitudes(c)).max() > 1e-3


def test_planted_wrong_cz_split_is_caught(monkeypatch):
    # put the phase on the projector side: a plausible slip in the bond split
    real = network.site_tensor

    def wrong(circuit, q, x_bit, fixed):
        c2 = circuit.copy()
        for g in c2.gates:
            if g.q1 >= 0:
                g.q0, g.q1 = g.q1, g.q0
                g.mat = np.asarray(g.mat).reshape(2, 2).T.reshape(-1) * np.array([1, 1, 1, 1j])
        return real(c2, q, x_bit, fixed)
    monkeypatch.setattr(network, "site_tensor", wrong)
    c = ri.rqc(2, 3, 8, seed=3)
    got = network.amplitudes_open(c, 0, list(range(6)))
    assert np.abs(got - statevector.amplitudes(c)).max() > 1e-3
