"""Fast sampling with frugal rejection (Sec. III.B) and path-fraction noisy sampling
(Sec. III.C).  Test infrastructure only.

Sec. III.B: the amplitudes of all bitstrings x = x1 u x2 that share one random x1 come
from one contraction, with the |x2| open sites left as output legs.  That batch is the
candidate pool of frugal rejection sampling for one output bitstring; the next output
bitstring starts from a new random x1.  The paper names the method and cites it without
restating it.  The reading taken here:
  - the candidates of a batch are examined in the order x2 = t XOR mask, t = 0, 1, ...,
    with `mask` a uniform random |x2|-bit value per batch;
  - candidate t is accepted when u_t < N p(x) / M, with N = 2^n, p(x) = |amp(x)|^2,
    M > 0 the rejection constant and u_t uniform in [0, 1);
  - the first accepted candidate is the batch's sample; a batch without one gives none.
For Porter-Thomas amplitudes (N p ~ Exp(1)) the acceptance N p / M exceeds 1 with
probability e^-M, so the sample distribution approaches p as M grows, and a batch of B
candidates gives a sample with probability about 1 - (1 - 1/M)^B.

Sec. III.C: summing only a fraction f of the paths (slices) of every amplitude gives
amplitudes of fidelity about f; sampling from them is noisy sampling at fidelity f.

Linear cross-entropy fidelity of samples x_i under the ideal distribution:
F = N * mean_i p(x_i) - 1 (about 1 for samples from p at Porter-Thomas statistics, 0 for
uniform samples).

All arithmetic is FP64.  The acceptance threshold rounds exactly as written:
p = re*re + im*im, then p * (2^n / M), each operation rounded once.
"""
from __future__ import annotations

from typing import Callable, List, Sequence

import numpy as np


def acceptance(amp: complex, n_qubits: int, M: float) -> float:
    """N |amp|^2 / M, rounded as the module docstring states."""
    re, im = float(amp.real), float(amp.imag)
    p = re * re + im * im
    return p * (2.0 ** n_qubits / M)


def frugal_select(amps: np.ndarray, n_qubits: int, M: float, u: np.ndarray, mask: int) -> int:
    """One batch of frugal rejection sampling.

    amps: complex128 [2^k], amplitude of x1 u x2 at index x2 (bit i = open site i).
    u: float64 [2^k], the uniform variate of scan position t.  mask: the batch's scan mask.
    Returns the first accepted x2 in scan order, or -1."""
    for t in range(len(amps)):
        x2 = t ^ int(mask)
        if float(u[t]) < acceptance(amps[x2], n_qubits, M):
            return x2
    return -1


def assemble(x1: int, x2: int, open_sites: Sequence[int]) -> int:
    """The bitstring x1 u x2: x1 with bit open_sites[i] replaced by bit i of x2."""
    x = int(x1)
    for i, q in enumerate(open_sites):
        x = (x & ~(1 << q)) | (((x2 >> i) & 1) << q)
    return x


def frugal_sample(amp_fn: Callable[[int], np.ndarray], n_qubits: int, open_sites: Sequence[int],
                  x1s: Sequence[int], masks: Sequence[int], u: np.ndarray, M: float) -> List[int]:
    """Sec. III.B: one frugal rejection pass per x1 batch; amp_fn(x1) gives the batch's
    2^|x2| amplitudes.  Returns the sampled bitstrings (batches without a sample skipped)."""
    out = []
    for b, x1 in enumerate(x1s):
        x2 = frugal_select(amp_fn(int(x1)), n_qubits, M, u[b], int(masks[b]))
        if x2 >= 0:
            out.append(assemble(int(x1), x2, open_sites))
    return out


def linear_xeb(probs: np.ndarray, n_qubits: int) -> float:
    """F = N * mean p(x_i) - 1 over the ideal probabilities of the samples."""
    return float(2.0 ** n_qubits * np.mean(np.asarray(probs, dtype=np.float64)) - 1.0)
