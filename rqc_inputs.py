"""Seeded synthetic inputs: random quantum circuits (RQCs) on a 2D grid and bitstrings.

This module only *describes* inputs. It holds no contraction, folding, scaling or
amplitude arithmetic, so both the CPU oracle (``oracle/``) and the CUDA path
(``paper_1905_00444_gb300``) may import it without sharing any of the method.

Circuit family (the paper's RQC class, Sec. III, "planar NISQ devices ... CZ gates
between two adjacent qubits"; depth written 1+d+1 as in Table I):

* layer 0: Hadamard on every qubit;
* cycle t = 0..d-1: a CZ layer over the nearest-neighbour pattern P_(t mod 8),
  then one single-qubit gate on every qubit drawn uniformly from {sqrt(X), sqrt(Y), T};
* last layer: Hadamard on every qubit.

The paper defers the exact gate rules to its references, so the eight patterns and
the draw are this project's reading: P0..P3 are the horizontal edges (r,c)-(r,c+1)
with (c mod 2, r mod 2) = (0,0), (1,1), (0,1), (1,0); P4..P7 are the vertical edges
(r,c)-(r+1,c) with (r mod 2, c mod 2) in the same order.  Every pattern is a matching
and the eight together cover every edge exactly once, so each edge carries d/8 CZs.
The single-qubit draw is splitmix64(seed, t, q) mod 3.

Qubit numbering: q = r * cols + c; bit q of a uint64 bitstring is the value of qubit q.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# gate kinds (same numbering as the C ABI's qfx_gate_kind)
H, SQRT_X, SQRT_Y, T, CZ, U1, U2, U4 = 0, 1, 2, 3, 4, 5, 6, 7
KIND_NAMES = {H: "H", SQRT_X: "SQRT_X", SQRT_Y: "SQRT_Y", T: "T", CZ: "CZ", U1: "U1", U2: "U2",
              U4: "U4"}

_S2 = 1.0 / math.sqrt(2.0)
# 2x2 matrices, row = output basis state, column = input basis state
MAT_H = np.array([[_S2, _S2], [_S2, -_S2]], dtype=np.complex128)
MAT_SQRT_X = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
MAT_SQRT_Y = 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)
MAT_T = np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=np.complex128)
MAT_S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
MAT_I = np.eye(2, dtype=np.complex128)
# diagonal of a two-qubit diagonal gate, indexed by 2*bit(q0) + bit(q1)
DIAG_CZ = np.array([1, 1, 1, -1], dtype=np.complex128)

_FIXED = {H: MAT_H, SQRT_X: MAT_SQRT_X, SQRT_Y: MAT_SQRT_Y, T: MAT_T}


@dataclasses.dataclass
class Gate:
    layer: int
    q0: int
    q1: int            # -1 for a single-qubit gate
    kind: int
    mat: np.ndarray    # 2x2 complex for 1q gates; length-4 diagonal for CZ and U2;
                       # 4x4 complex for U4, indexed [2*o0 + o1, 2*i0 + i1]

    @property
    def two_qubit(self) -> bool:
        return self.q1 >= 0


@dataclasses.dataclass
class Circuit:
    rows: int
    cols: int
    gates: List[Gate]
    name: str = ""

    @property
    def n_qubits(self) -> int:
        return self.rows * self.cols

    @property
    def n_layers(self) -> int:
        return 1 + max((g.layer for g in self.gates), default=-1)

    def qubit(self, r: int, c: int) -> int:
        return r * self.cols + c

    def edges(self):
        """All nearest-neighbour edges (q_lo, q_hi), horizontal first."""
        out = []
        for r in range(self.rows):
            for c in range(self.cols - 1):
                out.append((self.qubit(r, c), self.qubit(r, c + 1)))
        for r in range(self.rows - 1):
            for c in range(self.cols):
                out.append((self.qubit(r, c), self.qubit(r + 1, c)))
        return out

    def copy(self) -> "Circuit":
        return Circuit(self.rows, self.cols,
                       [Gate(g.layer, g.q0, g.q1, g.kind, g.mat.copy()) for g in self.gates],
                       self.name)


# ---------------------------------------------------------------------------
# counter-based random numbers (splitmix64, Steele/Lea/Flood 2014)
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One splitmix64 output for state x (the published finaliser of Steele et al.)."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def counter_draw(seed: int, a: int, b: int) -> int:
    """Draw keyed by (seed, a, b): three chained splitmix64 rounds."""
    return splitmix64(splitmix64(splitmix64(seed & _M64) ^ (a & _M64)) ^ (b & _M64))


def grid_pattern_edges(rows: int, cols: int, pattern: int):
    """Edges of CZ pattern P_pattern (0..7) on a rows x cols grid, as (q_lo, q_hi)."""
    order = [(0, 0), (1, 1), (0, 1), (1, 0)]
    out = []
    if pattern < 4:
        pc, pr = order[pattern]
        for r in range(rows):
            for c in range(cols - 1):
                if c % 2 == pc and r % 2 == pr:
                    out.append((r * cols + c, r * cols + c + 1))
    else:
        pr, pc = order[pattern - 4]
        for r in range(rows - 1):
            for c in range(cols):
                if r % 2 == pr and c % 2 == pc:
                    out.append((r * cols + c, (r + 1) * cols + c))
    return out


def fsim(theta: float, phi: float) -> np.ndarray:
    """The fermionic-simulation gate fSim(theta, phi) (a published two-qubit family: an
    XX+YY rotation by theta and a controlled phase e^(-i phi)), 4x4, basis 2*b(q0) + b(q1)."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0], [0, c, -1j * s, 0], [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


def rqc(rows: int, cols: int, depth: int, seed: int = 0,
        gate_set: Sequence[int] = (SQRT_X, SQRT_Y, T), parametrised: bool = False,
        two_qubit: str = "cz") -> Circuit:
    """Random circuit of depth 1+depth+1 on a rows x cols grid (see module docstring).

    gate_set: kinds drawn for the single-qubit layers (uniform, counter-based).
    parametrised: draw G = Rz(a) Ry(b) Rz(c) with angles uniform in [0, 2pi) instead.
    two_qubit: "cz" (diagonal, one bond bit per gate) or "fsim": every two-qubit gate is a
    general (U4) fSim(theta, phi) with theta uniform in [0, pi) and phi in [0, 2pi) drawn
    per gate (two bond bits per gate); "fsim_pi2": every one is fSim(pi/2, 0), a Clifford
    gate (with a Clifford gate_set the circuit has exact stabilizer probabilities).
    """
    n = rows * cols
    gates: List[Gate] = []
    for q in range(n):
        gates.append(Gate(0, q, -1, H, MAT_H.copy()))
    layer = 1
    for t in range(depth):
        for (a, b) in grid_pattern_edges(rows, cols, t % 8):
            if two_qubit == "fsim":
                th = counter_draw(seed, 2000003 * t + a, 0x5F1) / 2.0 ** 64 * math.pi
                ph = counter_draw(seed, 2000003 * t + a, 0x5F2) / 2.0 ** 64 * 2 * math.pi
                gates.append(Gate(layer, a, b, U4, fsim(th, ph)))
            elif two_qubit == "fsim_pi2":
                gates.append(Gate(layer, a, b, U4, fsim(math.pi / 2, 0.0)))
            else:
                gates.append(Gate(layer, a, b, CZ, DIAG_CZ.copy()))
        layer += 1
        for q in range(n):
            if parametrised:
                ang = [counter_draw(seed, 1000003 * t + 7 * q + j, 0xA5A5) / 2.0 ** 64 * 2 * math.pi
                       for j in range(3)]
                gates.append(Gate(layer, q, -1, U1, zyz(*ang)))
            else:
                kind = gate_set[counter_draw(seed, t, q) % len(gate_set)]
                gates.append(Gate(layer, q, -1, kind, _FIXED[kind].copy()))
        layer += 1
    for q in range(n):
        gates.append(Gate(layer, q, -1, H, MAT_H.copy()))
    suffix = "" if two_qubit == "cz" else "_" + two_qubit
    return Circuit(rows, cols, gates, name=f"rqc_{rows}x{cols}x(1+{depth}+1)_s{seed}{suffix}")


def zyz(a: float, b: float, c: float) -> np.ndarray:
    """Rz(a) @ Ry(b) @ Rz(c), the parametrised single-qubit gate."""
    rz = lambda t: np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=np.complex128)
    ry = np.array([[math.cos(b / 2), -math.sin(b / 2)], [math.sin(b / 2), math.cos(b / 2)]],
                  dtype=np.complex128)
    return rz(a) @ ry @ rz(c)


def ghz_snake(rows: int, cols: int) -> Circuit:
    """GHZ preparation: H on qubit 0, then CNOT(prev -> next) along a boustrophedon path,
    each CNOT written as H(target) CZ H(target).  Amplitudes: 1/sqrt(2) on 0^n and 1^n."""
    path = []
    for r in range(rows):
        cs = range(cols) if r % 2 == 0 else range(cols - 1, -1, -1)
        path += [r * cols + c for c in cs]
    gates = [Gate(0, path[0], -1, H, MAT_H.copy())]
    layer = 1
    for a, b in zip(path[:-1], path[1:]):
        gates.append(Gate(layer, b, -1, H, MAT_H.copy()))
        gates.append(Gate(layer + 1, min(a, b), max(a, b), CZ, DIAG_CZ.copy()))
        gates.append(Gate(layer + 2, b, -1, H, MAT_H.copy()))
        layer += 3
    return Circuit(rows, cols, gates, name=f"ghz_{rows}x{cols}")


def product_circuit(rows: int, cols: int, depth: int, seed: int = 0) -> Circuit:
    """An RQC with every CZ removed: a product state (closed form per qubit)."""
    c = rqc(rows, cols, depth, seed)
    c.gates = [g for g in c.gates if not g.two_qubit]
    c.name = f"product_{rows}x{cols}x{depth}_s{seed}"
    return c


def random_bitstrings(n_qubits: int, count: int, seed: int) -> np.ndarray:
    """count uint64 bitstrings with the low n_qubits bits uniform (counter-based)."""
    mask = (1 << n_qubits) - 1 if n_qubits < 64 else _M64
    return np.array([counter_draw(seed, 0xB17, i) & mask for i in range(count)], dtype=np.uint64)


def random_bitstring_words(n_qubits: int, count: int, seed: int) -> np.ndarray:
    """count bitstrings of n_qubits bits as uint64 words [count, ceil(n_qubits / 64)]: qubit q
    is bit q % 64 of word q / 64.  Word w of bitstring i is counter_draw(seed, 0xB17 + w, i),
    masked to the qubits it holds, so one-word bitstrings equal random_bitstrings'."""
    W = (n_qubits + 63) // 64
    out = np.zeros((count, W), dtype=np.uint64)
    for w in range(W):
        bits = min(64, n_qubits - 64 * w)
        mask = (1 << bits) - 1
        out[:, w] = [counter_draw(seed, 0xB17 + w, i) & mask for i in range(count)]
    return out


def words_to_int(words) -> int:
    """The bitstring held by uint64 words (word w holds qubits 64 w .. 64 w + 63)."""
    return sum(int(v) << (64 * w) for w, v in enumerate(np.asarray(words, dtype=np.uint64).reshape(-1)))


def int_to_words(x: int, n_qubits: int) -> np.ndarray:
    """Inverse of words_to_int for an n_qubits bitstring."""
    W = (n_qubits + 63) // 64
    return np.array([(int(x) >> (64 * w)) & _M64 for w in range(W)], dtype=np.uint64)


def sampling_draws(n_qubits: int, n_open: int, count: int, seed: int):
    """Random inputs of `count` fast-sampling batches (one x1 each): x1 (uint64, low n_qubits
    bits uniform), a scan mask (uint64, low n_open bits uniform) and one uniform variate in
    [0, 1) per candidate (float64 [count, 2^n_open])."""
    rng = np.random.default_rng(seed)
    x1 = random_bitstrings(n_qubits, count, seed ^ 0x5A3)
    mask = rng.integers(0, 1 << n_open, size=count, dtype=np.uint64)
    u = rng.random((count, 1 << n_open))
    return x1, mask, u


def random_complex(shape, seed: int, dtype=np.complex64) -> np.ndarray:
    """Seeded complex array with iid N(0,1) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(dtype)


def circuit_to_text(c: Circuit) -> str:
    """The project's text format: header 'grid R C', then one gate per line,
    'layer KIND q0 [q1] v0 ..', with the gate's matrix values (re, im interleaved: the 2x2
    matrix row-major, the 4 diagonal entries of a CZ or U2 gate, or the 4x4 matrix of a U4
    gate row-major)."""
    lines = [f"grid {c.rows} {c.cols}"]
    for g in c.gates:
        vals = " ".join(f"{v.real:.17g} {v.imag:.17g}" for v in np.asarray(g.mat).reshape(-1))
        qs = f"{g.q0} {g.q1}" if g.two_qubit else f"{g.q0}"
        lines.append(f"{g.layer} {KIND_NAMES[g.kind]} {qs} {vals}")
    return "\n".join(lines) + "\n"
