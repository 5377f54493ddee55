"""Tensor-network route: time-first folding plus a row-major sweep.  Test infrastructure only.

Sec. III: the circuit is contracted "in time" first, so that every grid site becomes
one tensor and the network becomes a regular 2D grid (Fig. 3).  Two neighbouring
sites share one bond of dimension 2 per diagonal two-qubit gate between them
(Fig. 3 caption; App. A: a diagonal two-qubit gate has only two variables).  The
split used here is the identity

    D(b0, b1) = sum_k  delta(b0, k) * D(k, b1),

i.e. the projector |k><k| on the gate's first qubit q0 and diag(D(k,0), D(k,1)) on
its second qubit q1, with k the bond leg.  A general two-qubit gate G (4x4, entries
G[2*o0 + o1, 2*i0 + i1]) has a leg of dimension 4: writing out its q0 indices,

    G = sum_{o0, i0}  |o0><i0|  (x)  B_(o0,i0),   B_(o0,i0)[o1, i1] = G[2*o0 + o1, 2*i0 + i1],

so q0 applies |o0><i0| and q1 applies B_k for leg value k = 2*o0 + i0 (two bits).
Every leg keeps its own label ('cz', gate_index); a grid bond is the group of legs of
the gates on that edge.

Cuts (Sec. III.A): fixing a set of legs to values gives one slice ("path"); the
amplitude is the sum over all slices.  A bond's index is read with the leg of its
earliest gate as the most significant bits (a two-bit leg reads o0 as its high bit), so
a sub-range cut of size 2^b at offset o fixes that bond's first (m - b) bits to the high
bits of o -- which may fix only the high bit of a two-bit leg.

The sweep absorbs sites in row-major order with ``np.tensordot`` over the labels
they share -- a different order from any column sweep, and no layout tricks.
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

Label = Tuple


def gates_by_qubit(circuit) -> Dict[int, List[int]]:
    """Gate indices acting on each qubit, in layer (time) order."""
    out: Dict[int, List[int]] = {q: [] for q in range(circuit.n_qubits)}
    order = sorted(range(len(circuit.gates)), key=lambda i: circuit.gates[i].layer)
    for i in order:
        g = circuit.gates[i]
        out[g.q0].append(i)
        if g.q1 >= 0:
            out[g.q1].append(i)
    return out


def bond_legs(circuit) -> Dict[Tuple[int, int], List[int]]:
    """Edge (q_lo, q_hi) -> indices of the two-qubit gates on it, in time order."""
    out: Dict[Tuple[int, int], List[int]] = {}
    order = sorted(range(len(circuit.gates)), key=lambda i: circuit.gates[i].layer)
    for i in order:
        g = circuit.gates[i]
        if g.q1 >= 0:
            out.setdefault((min(g.q0, g.q1), max(g.q0, g.q1)), []).append(i)
    return out


def leg_bits(gate) -> int:
    """Bits of a two-qubit gate's leg: 2 for a general 4x4 gate, 1 for a diagonal one."""
    return 2 if np.asarray(gate.mat).size == 16 else 1


def site_tensor(circuit, q: int, x_bit: Optional[int], fixed: Dict[int, object]):
    """Fold the time line of qubit q into one tensor.

    x_bit: output value of the qubit (None keeps the output leg open, labelled ('x', q)).
    fixed: gate index -> leg value for legs fixed by a cut: an int when the whole leg is
    fixed, (value, b) when only its b high bits are.
    Returns (tensor, labels); labels are ('cz', gate_index) or ('x', q).
    """
    t = np.array([1.0, 0.0], dtype=np.complex128)   # |0>, physical leg last
    labels: List[Label] = []
    for gi in gates_by_qubit(circuit)[q]:
        g = circuit.gates[gi]
        if g.q1 < 0:
            t = np.tensordot(t, g.mat, axes=([t.ndim - 1], [1]))
            continue
        w = leg_bits(g)
        op = np.zeros((1 << w, 2, 2), dtype=np.complex128)           # op[k, out, in]
        if w == 1:
            d = np.asarray(g.mat, dtype=np.complex128).reshape(2, 2)  # d[b0, b1]
            for k in range(2):
                if q == g.q0:
                    op[k, k, k] = 1.0
                else:
                    op[k, 0, 0] = d[k, 0]
                    op[k, 1, 1] = d[k, 1]
        else:
            G = np.asarray(g.mat, dtype=np.complex128).reshape(4, 4)
            for o0 in range(2):
                for i0 in range(2):
                    k = 2 * o0 + i0
                    if q == g.q0:
                        op[k, o0, i0] = 1.0
                    else:
                        op[k] = G[2 * o0:2 * o0 + 2, 2 * i0:2 * i0 + 2]
        f = fixed.get(gi)
        if isinstance(f, tuple):                  # high bits fixed: other values drop out
            val, b = f
            for k in range(1 << w):
                if k >> (w - b) != val:
                    op[k] = 0
            f = None
        if f is not None:
            t = np.tensordot(t, op[f], axes=([t.ndim - 1], [1]))
        else:
            t = np.tensordot(t, op, axes=([t.ndim - 1], [2]))        # (..., k, out)
            labels.append(("cz", gi))
    if x_bit is None:
        labels.append(("x", q))
    else:
        t = t[..., x_bit]
    return t, labels


def contract_network(tensors: Sequence[Tuple[np.ndarray, List[Label]]]):
    """Absorb tensors one by one, summing every label the running tensor shares."""
    acc, lab = tensors[0]
    for t, tl in tensors[1:]:
        shared = [l for l in lab if l in tl]
        acc = np.tensordot(acc, t, axes=([lab.index(l) for l in shared],
                                          [tl.index(l) for l in shared]))
        lab = [l for l in lab if l not in shared] + [l for l in tl if l not in shared]
    return acc, lab


def slice_fixed_legs(circuit, cuts: Sequence[Tuple[int, int, int]], slice_id: int) -> Dict[int, object]:
    """Leg values fixed by slice `slice_id` of the cut list.

    cuts: (q_a, q_b, size) per cut bond; size is a power of two dividing the bond
    dimension (size == 1 fixes the whole bond).  The slice id is mixed-radix over
    the cuts with the first cut as the most significant digit.
    """
    legs = bond_legs(circuit)

    def bits(gl):
        return sum(leg_bits(circuit.gates[g]) for g in gl)

    radices = []
    for (a, b, size) in cuts:
        m = bits(legs[(min(a, b), max(a, b))])
        assert size >= 1 and (size & (size - 1)) == 0 and size <= (1 << m)
        radices.append((1 << m) // size)
    digits = []
    rem = slice_id
    for r in reversed(radices):
        digits.append(rem % r)
        rem //= r
    assert rem == 0, "slice id out of range"
    digits.reverse()
    fixed: Dict[int, object] = {}
    for (a, b, size), dgt in zip(cuts, digits):
        gl = legs[(min(a, b), max(a, b))]
        nfix = bits(gl) - (size.bit_length() - 1)
        left = nfix                                # fixed bits still to hand out, MSB first
        for g in gl:
            if left <= 0:
                break
            w = leg_bits(circuit.gates[g])
            take = min(w, left)
            left -= take
            val = (dgt >> left) & ((1 << take) - 1)
            fixed[g] = val if take == w else (val, take)
    return fixed


def n_slices(circuit, cuts) -> int:
    legs = bond_legs(circuit)
    out = 1
    for (a, b, size) in cuts:
        m = sum(leg_bits(circuit.gates[g]) for g in legs[(min(a, b), max(a, b))])
        out *= (1 << m) // size
    return out


def amplitudes_open(circuit, x1: int, open_sites: Sequence[int] = (),
                    fixed: Optional[Dict[int, int]] = None) -> np.ndarray:
    """Amplitudes for every assignment of the open sites, the other qubits taken from x1.

    Output index j has bit i equal to the value of qubit open_sites[i].
    """
    fixed = fixed or {}
    opened = set(open_sites)
    tens = []
    for q in range(circuit.n_qubits):                 # row-major: q = r*cols + c
        xb = None if q in opened else (int(x1) >> q) & 1
        tens.append(site_tensor(circuit, q, xb, fixed))
    acc, lab = contract_network(tens)
    if not open_sites:
        return np.array([complex(acc)])
    axes = [lab.index(("x", q)) for q in reversed(list(open_sites))]
    return np.transpose(acc, axes).reshape(-1).copy()


def amplitudes_sliced(circuit, x1: int, open_sites: Sequence[int], cuts,
                      slice_ids: Iterable[int]) -> np.ndarray:
    """Sum of the listed slices' contributions (all slices = the full amplitude)."""
    out = None
    for sid in slice_ids:
        part = amplitudes_open(circuit, x1, open_sites, slice_fixed_legs(circuit, cuts, sid))
        out = part if out is None else out + part
    return out


def amplitudes(circuit, bitstrings) -> np.ndarray:
    """Closed amplitudes <x|C|0^n> for each bitstring x."""
    return np.array([amplitudes_open(circuit, int(x))[0] for x in bitstrings])
