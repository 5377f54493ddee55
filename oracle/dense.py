"""Textbook route: the whole circuit as one dense 2^n x 2^n matrix (n <= 10).

Test infrastructure only (see ``oracle/__init__.py``).

amp(x) = <x| U_L ... U_1 U_0 |0^n>, each layer U_l the Kronecker product of its gates
(Sec. II: a circuit is a product of gate tensors; rank-1 projectors fix input and
output).  Basis index i carries qubit q in bit q, so the Kronecker factors run from
qubit n-1 (most significant) down to qubit 0.
"""
from __future__ import annotations

import numpy as np


def gate_matrix(n: int, gate) -> np.ndarray:
    """Dense matrix of one gate acting on n qubits."""
    dim = 1 << n
    if gate.q1 < 0:
        full = np.array([[1.0 + 0j]])
        for q in range(n - 1, -1, -1):
            full = np.kron(full, gate.mat if q == gate.q0 else np.eye(2))
        return full
    idx = np.arange(dim)
    b0 = (idx >> gate.q0) & 1
    b1 = (idx >> gate.q1) & 1
    g = np.asarray(gate.mat)
    if g.size == 4:            # diagonal two-qubit gate, entry d[2*bit(q0) + bit(q1)]
        return np.diag(g[2 * b0 + b1])
    # general two-qubit gate g[2*o0 + o1, 2*i0 + i1]: column i maps to the four rows that
    # differ from i only in bits q0 and q1
    full = np.zeros((dim, dim), dtype=np.complex128)
    base = idx & ~((1 << gate.q0) | (1 << gate.q1))
    for o0 in range(2):
        for o1 in range(2):
            rows = base | (o0 << gate.q0) | (o1 << gate.q1)
            full[rows, idx] = g.reshape(4, 4)[2 * o0 + o1, 2 * b0 + b1]
    return full


def unitary(circuit) -> np.ndarray:
    n = circuit.n_qubits
    assert n <= 10, "dense oracle is for tiny circuits only"
    u = np.eye(1 << n, dtype=np.complex128)
    for layer in range(circuit.n_layers):
        for g in circuit.gates:
            if g.layer == layer:
                u = gate_matrix(n, g) @ u
    return u


def amplitudes(circuit) -> np.ndarray:
    """All 2^n amplitudes <x|U|0^n>, indexed by x."""
    return unitary(circuit)[:, 0].copy()
