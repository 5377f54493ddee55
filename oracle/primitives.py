"""Single operations of the contraction, written as their definitions.
Test infrastructure only.

* ``contract_step``: one pairwise contraction in the TTGT form (Sec. III.E):
  C[p, n, s] = sum_k S[k, n] * B[p, k, s], complex128.
* ``permute``: out = in with its axes reordered (the tensor transpose of Sec. III.E).
* ``flops_eq1``: the flop count of Eq. 1, F = 8 sqrt(v0 v1 v2), from the three tensor
  volumes (4 real multiplies and 4 real adds per complex multiply-add).
"""
from __future__ import annotations

import math

import numpy as np


def contract_step(S: np.ndarray, B: np.ndarray, P: int, K: int, N: int, Sd: int) -> np.ndarray:
    s = np.asarray(S, dtype=np.complex128).reshape(K, N)
    b = np.asarray(B, dtype=np.complex128).reshape(P, K, Sd)
    return np.einsum("kn,pks->pns", s, b)


def permute(x: np.ndarray, shape, perm) -> np.ndarray:
    """out has axes (shape[perm[0]], shape[perm[1]], ...), C order."""
    return np.ascontiguousarray(np.transpose(np.asarray(x).reshape(shape), perm))


def flops_eq1(v0: float, v1: float, v2: float) -> float:
    return 8.0 * math.sqrt(float(v0) * float(v1) * float(v2))
