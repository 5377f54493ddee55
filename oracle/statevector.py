"""Gate-by-gate complex128 state vector.  Test infrastructure only.

Starts from |0^n> and applies the gates in layer order (the RQC form 1+d+1 of
Table I), giving every amplitude <x|C|0^n> at once.  Basis index bit q = qubit q.
"""
from __future__ import annotations

import numpy as np


def apply_1q(psi: np.ndarray, n: int, q: int, g: np.ndarray) -> np.ndarray:
    v = psi.reshape(1 << (n - 1 - q), 2, 1 << q)
    return np.einsum("ab,xby->xay", g, v).reshape(-1)


def apply_diag_2q(psi: np.ndarray, n: int, q0: int, q1: int, d: np.ndarray) -> np.ndarray:
    idx = np.arange(1 << n, dtype=np.int64)
    sel = 2 * ((idx >> q0) & 1) + ((idx >> q1) & 1)
    return psi * np.asarray(d)[sel]


def apply_2q(psi: np.ndarray, n: int, q0: int, q1: int, g: np.ndarray) -> np.ndarray:
    """General two-qubit gate g[2*o0 + o1, 2*i0 + i1] on qubits (q0, q1)."""
    t = psi.reshape([2] * n)                     # axis a holds qubit n - 1 - a
    a0, a1 = n - 1 - q0, n - 1 - q1
    out = np.tensordot(np.asarray(g).reshape(2, 2, 2, 2), t, axes=([2, 3], [a0, a1]))
    return np.moveaxis(out, [0, 1], [a0, a1]).reshape(-1)


def state(circuit) -> np.ndarray:
    n = circuit.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    order = sorted(range(len(circuit.gates)), key=lambda i: circuit.gates[i].layer)
    for i in order:
        g = circuit.gates[i]
        if g.q1 < 0:
            psi = apply_1q(psi, n, g.q0, g.mat)
        elif np.asarray(g.mat).size == 16:
            psi = apply_2q(psi, n, g.q0, g.q1, g.mat)
        else:
            psi = apply_diag_2q(psi, n, g.q0, g.q1, g.mat)
    return psi


def amplitudes(circuit, bitstrings=None) -> np.ndarray:
    psi = state(circuit)
    if bitstrings is None:
        return psi
    return psi[np.asarray(bitstrings, dtype=np.int64)]
