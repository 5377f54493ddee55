"""Writes rqc_11x11x16_amplitudes.json: FP64 oracle amplitudes of a 121-qubit circuit, the
paper's 11x11 grid (Table I) at depth 1+16+1, through oracle.network only (the uncut
row-major sweep, about a minute on 8 cores).  Bitstrings have two uint64 words.

Inputs (all seeded):
  circuit    rqc_inputs.rqc(11, 11, 16, seed=0)
  x1         rqc_inputs.random_bitstring_words(121, 1, seed=5)[0] (words, hex in the file)
  open sites 65, 76, 87, 98, 109, 120 (the planner's default: the last six sites of its
             column sweep; output index j has bit i = value of open site i)

Run:  python tests/golden/make_rqc_11x11_amplitudes.py
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import rqc_inputs as ri  # noqa: E402
from oracle import network  # noqa: E402

OUT = os.path.join(HERE, "rqc_11x11x16_amplitudes.json")
OPEN_SITES = [65, 76, 87, 98, 109, 120]


def main():
    circ = ri.rqc(11, 11, 16, seed=0)
    words = ri.random_bitstring_words(121, 1, seed=5)[0]
    x1 = ri.words_to_int(words)
    t0 = time.perf_counter()
    amps = network.amplitudes_open(circ, x1, OPEN_SITES)
    dt = time.perf_counter() - t0
    with open(OUT, "w") as f:
        json.dump({"_about": "FP64 oracle amplitudes <x|C|0^121> of rqc(11, 11, 16, seed=0) for the "
                             "64 bitstrings x = x1 u x2 over the open sites, written by "
                             "tests/golden/make_rqc_11x11_amplitudes.py through oracle.network.",
                   "rows": 11, "cols": 11, "depth": 16, "seed": 0,
                   "x1_words": [hex(int(w)) for w in words], "open_sites": OPEN_SITES,
                   "re": [float(v) for v in amps.real], "im": [float(v) for v in amps.imag],
                   "oracle_seconds": round(dt, 1)}, f, indent=1)
    print(f"{dt:.1f} s, max |amp| {np.abs(amps).max():.3e}")


if __name__ == "__main__":
    main()
