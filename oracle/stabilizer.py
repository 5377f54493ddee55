"""Exact output probabilities of Clifford circuits (Aaronson-Gottesman tableau).
Test infrastructure only.

The paper (Sec. II) notes that circuits without non-Clifford gates are efficiently
simulable by stabilizer methods.  That makes T-free members of the RQC family a
full-size check: at any grid size, every |amp(x)|^2 is 0 or 2^-k, and this module
gives the exact value for each sampled x by measuring the qubits one by one in the
Z basis (random outcome: factor 1/2; determined outcome: factor 1 or 0).

The tableau follows Aaronson & Gottesman, "Improved simulation of stabilizer
circuits", PRA 70, 052328 (2004): rows 0..n-1 destabilisers, n..2n-1 stabilisers.
Global phases are ignored, so sqrt(X) = H S H and sqrt(Y) ~ H Z are exact here.
"""
from __future__ import annotations

import numpy as np

import rqc_inputs as ri


class Tableau:
    def __init__(self, n: int):
        self.n = n
        self.x = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.z = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.r = np.zeros(2 * n + 1, dtype=np.uint8)
        for i in range(n):
            self.x[i, i] = 1
            self.z[n + i, i] = 1

    # --- gates -----------------------------------------------------------
    def h(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.x[:, a], self.z[:, a] = self.z[:, a].copy(), self.x[:, a].copy()

    def s(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.z[:, a] ^= self.x[:, a]

    def cnot(self, a, b):
        self.r ^= self.x[:, a] & self.z[:, b] & (self.x[:, b] ^ self.z[:, a] ^ 1)
        self.x[:, b] ^= self.x[:, a]
        self.z[:, a] ^= self.z[:, b]

    def cz(self, a, b):
        self.h(b)
        self.cnot(a, b)
        self.h(b)

    # --- row arithmetic ----------------------------------------------------
    @staticmethod
    def _g(x1, z1, x2, z2):
        g = np.zeros(x1.shape, dtype=np.int64)
        both = (x1 == 1) & (z1 == 1)
        xo = (x1 == 1) & (z1 == 0)
        zo = (x1 == 0) & (z1 == 1)
        g[both] = z2[both].astype(np.int64) - x2[both].astype(np.int64)
        g[xo] = z2[xo].astype(np.int64) * (2 * x2[xo].astype(np.int64) - 1)
        g[zo] = x2[zo].astype(np.int64) * (1 - 2 * z2[zo].astype(np.int64))
        return g

    def rowsum(self, h, i):
        tot = 2 * int(self.r[h]) + 2 * int(self.r[i]) + int(
            self._g(self.x[i], self.z[i], self.x[h], self.z[h]).sum())
        tot %= 4
        # destabiliser rows (h < n) may pick up a phase of +-i; their sign is never read
        assert h < self.n or tot in (0, 2)
        self.r[h] = 1 if tot == 2 else 0
        self.x[h] ^= self.x[i]
        self.z[h] ^= self.z[i]

    def measure_forced(self, a: int, outcome: int) -> float:
        """Measure qubit a in Z, force the outcome, return its probability."""
        n = self.n
        stab = np.nonzero(self.x[n:2 * n, a])[0]
        if stab.size:
            p = n + int(stab[0])
            for i in range(2 * n):
                if i != p and self.x[i, a]:
                    self.rowsum(i, p)
            self.x[p - n], self.z[p - n], self.r[p - n] = self.x[p].copy(), self.z[p].copy(), self.r[p]
            self.x[p] = 0
            self.z[p] = 0
            self.z[p, a] = 1
            self.r[p] = outcome
            return 0.5
        sc = 2 * n
        self.x[sc] = 0
        self.z[sc] = 0
        self.r[sc] = 0
        for i in range(n):
            if self.x[i, a]:
                self.rowsum(sc, i + n)
        return 1.0 if int(self.r[sc]) == outcome else 0.0


# fSim(pi/2, 0) (|01> -> -i|10>, |10> -> -i|01>) up to a global phase, as a word in the
# tableau's H, S = diag(1, i) and CZ, applied left to right; 0 = the gate's q0, 1 = its q1.
# Found by a breadth-first search over two-qubit Clifford words and checked against the
# matrix by tests/test_oracle_general_gates.py.
FSIM_PI2_WORD = (("h", 0), ("h", 1), ("s", 0), ("h", 0), ("cz",), ("h", 0), ("h", 1), ("s", 1),
                 ("cz",), ("h", 0), ("cz",), ("h", 1))


def _apply(tab: Tableau, g):
    if g.q1 >= 0:
        m = np.asarray(g.mat)
        if m.size == 16 and np.allclose(m, ri.fsim(np.pi / 2, 0.0)):
            qs = (g.q0, g.q1)
            for op in FSIM_PI2_WORD:
                if op[0] == "cz":
                    tab.cz(g.q0, g.q1)
                elif op[0] == "h":
                    tab.h(qs[op[1]])
                else:
                    tab.s(qs[op[1]])
            return
        if m.size != 4 or not np.allclose(m.reshape(-1), ri.DIAG_CZ):
            raise ValueError("stabilizer oracle: only CZ and fSim(pi/2, 0) among two-qubit gates")
        tab.cz(g.q0, g.q1)
        return
    if g.kind == ri.H:
        tab.h(g.q0)
    elif g.kind == ri.SQRT_X:          # H S H
        tab.h(g.q0); tab.s(g.q0); tab.h(g.q0)
    elif g.kind == ri.SQRT_Y:          # Z then H (global phase dropped)
        tab.s(g.q0); tab.s(g.q0); tab.h(g.q0)
    else:
        raise ValueError(f"stabilizer oracle: gate kind {g.kind} is not Clifford")


def prepare(circuit) -> Tableau:
    tab = Tableau(circuit.n_qubits)
    for i in sorted(range(len(circuit.gates)), key=lambda i: circuit.gates[i].layer):
        _apply(tab, circuit.gates[i])
    return tab


def probability(circuit, x: int, tab: Tableau = None) -> float:
    """Exact |<x|C|0^n>|^2 for a Clifford circuit."""
    base = tab if tab is not None else prepare(circuit)
    t = Tableau.__new__(Tableau)
    t.n, t.x, t.z, t.r = base.n, base.x.copy(), base.z.copy(), base.r.copy()
    p = 1.0
    for q in range(circuit.n_qubits):
        p *= t.measure_forced(q, (int(x) >> q) & 1)
        if p == 0.0:
            return 0.0
    return p
