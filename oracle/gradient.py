"""Gate gradients by linearity.  Test infrastructure only.

Every gate appears once in the circuit, so each amplitude is linear in each gate's
entries: d amp / d G_ij = amp with G replaced by the matrix unit e_i e_j^T (for a
diagonal two-qubit gate, its m-th diagonal entry replaced by the unit vector e_m).
For a real loss L(amp) with upstream gradient gbar_b = dL/dRe(amp_b) + i dL/dIm(amp_b)
(PyTorch's convention), the gradient of gate entry G_ij in the same convention is

    grad_ij = sum_b gbar_b * conj(d amp_b / d G_ij).

For L = sum_b |amp_b|^2, gbar_b = 2 amp_b.  ``finite_difference`` gives the same
quantity by central differences on the real and imaginary part (checking the formula).
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

from . import network


def _with_entry(circuit, gate: int, entry: int, value=None):
    c = circuit.copy()
    m = np.zeros_like(c.gates[gate].mat)
    flat = m.reshape(-1)
    if value is None:
        flat[entry] = 1.0
    else:
        flat[:] = value.reshape(-1)
    c.gates[gate].mat = m
    return c


def amplitude_derivative(circuit, gate: int, entry: int, x1: int, open_sites=()) -> np.ndarray:
    """d amp / d G[entry] for every open-site assignment (entry = flat index into .mat)."""
    return network.amplitudes_open(_with_entry(circuit, gate, entry), x1, open_sites)


def loss_sum_abs2(amps: np.ndarray) -> float:
    return float(np.sum(np.abs(amps) ** 2))


def grad_entries(circuit, x1: int, open_sites: Sequence[int],
                 entries: Sequence[Tuple[int, int]]) -> np.ndarray:
    """PyTorch-convention gradient of L = sum |amp|^2 for the listed (gate, entry) pairs."""
    amps = network.amplitudes_open(circuit, x1, open_sites)
    gbar = 2.0 * amps
    out = []
    for gate, entry in entries:
        d = amplitude_derivative(circuit, gate, entry, x1, open_sites)
        out.append(np.sum(gbar * np.conj(d)))
    return np.array(out)


def finite_difference(circuit, x1: int, open_sites: Sequence[int], gate: int, entry: int,
                      h: float = 1e-3) -> complex:
    """Central differences of L on Re and Im of one gate entry: dL/dRe + i dL/dIm."""
    def loss_at(delta):
        c = circuit.copy()
        c.gates[gate].mat = c.gates[gate].mat.copy()
        c.gates[gate].mat.reshape(-1)[entry] += delta
        return loss_sum_abs2(network.amplitudes_open(c, x1, open_sites))
    dre = (loss_at(h) - loss_at(-h)) / (2 * h)
    dim = (loss_at(1j * h) - loss_at(-1j * h)) / (2 * h)
    return complex(dre, dim)
