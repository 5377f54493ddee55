"""Writes rqc_7x7x32_slices.json: FP64 oracle partial amplitudes of the 7x7x(1+32+1)
benchmark circuit for a few slices of a 12-bond cut.  Calls only ``oracle/`` and the
seeded input generator ``rqc_inputs``.

Why slices: the uncut circuit's largest intermediate is 2^32 complex128 values (64 GiB,
more with the temporaries of a pairwise contraction), beyond the memory of the hosts this
runs on.  Cutting the 12 vertical bonds of grid columns 0 and 6 (every bond fixed to one
value, 16^12 = 2^48 slices, Sec. III.A) brings the oracle's row-major sweep down to 2^29
values per tensor.  The column sweep of the GPU path keeps, under the same cuts, every
step of grid columns 1..5 exactly as in the uncut benchmark plan -- all 25 steps of shape
(P, K, N, Sd) with K = N = 256 and P * Sd = 2^24 among them -- so a slice exercises the
benchmarked contraction at full size with T gates, and its partial amplitudes are the
oracle's own definition of that slice (the sum over the fixed legs' values).

Inputs (all seeded):
  circuit    rqc_inputs.rqc(7, 7, 32, seed=0)         (the benchmark circuit)
  x1         rqc_inputs.random_bitstrings(49, 1, seed=1000)[0]  (the benchmark's first x1)
  open sites 13, 20, 27, 34, 41, 48 (column 6, rows 1..6; output bit i = open site i)
  cuts       (r*7 + c, (r+1)*7 + c, size 1) for c in (0, 6), r in 0..5, in that order
  slices     ids drawn by numpy.random.default_rng(4848) in [0, 2^48), in order.  Most
             slices of this cut are exactly zero: between two successive gates of a cut
             bond a qubit's own gates can map one fixed leg value to a state orthogonal to
             the next (a site tensor vanishes), and such constraints also chain through
             neighbouring sites.  Candidates with a vanishing site tensor are skipped
             without contracting; the others are contracted, and the file keeps the first
             --nonzero of them whose norm is within 1e-9 of the largest norm met (an exact
             zero comes out of the FP64 contraction as rounding noise some 15 or more
             orders of magnitude below a nonzero slice).

Run:  python tests/golden/make_rqc_7x7x32_slices.py [--nonzero K]   (about a minute per
contracted candidate on 8 cores; progress is kept in the file between runs).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import rqc_inputs as ri  # noqa: E402
from oracle import network  # noqa: E402

OUT = os.path.join(HERE, "rqc_7x7x32_slices.json")
ROWS = COLS = 7
DEPTH = 32
OPEN_SITES = [13, 20, 27, 34, 41, 48]
CUT_COLUMNS = (0, 6)


def cuts():
    return [(r * COLS + c, (r + 1) * COLS + c, 1) for c in CUT_COLUMNS for r in range(ROWS - 1)]


def candidates(circ, x1, cl):
    """Seeded slice ids none of whose site tensors vanishes, in draw order."""
    rng = np.random.default_rng(4848)
    while True:
        sid = int(rng.integers(0, 1 << 48))
        fixed = network.slice_fixed_legs(circ, cl, sid)
        if all(np.any(network.site_tensor(circ, q, None if q in OPEN_SITES else (x1 >> q) & 1,
                                          fixed)[0] != 0) for q in range(ROWS * COLS)):
            yield sid


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nonzero", type=int, default=3, help="nonzero slices to keep")
    args = ap.parse_args()
    circ = ri.rqc(ROWS, COLS, DEPTH, seed=0)
    x1 = int(ri.random_bitstrings(ROWS * COLS, 1, seed=1000)[0])
    cl = cuts()
    n_sl = network.n_slices(circ, cl)
    assert n_sl == 1 << 48
    data = {"_about": (
        "FP64 partial amplitudes of single slices of the 7x7x(1+32+1) benchmark circuit "
        "(rqc seed 0, x1 = the benchmark's first bitstring), 12 vertical bonds of columns 0 "
        "and 6 cut to single values, written by tests/golden/make_rqc_7x7x32_slices.py "
        "through oracle.network only (Sec. III.A: each slice is the network with the cut "
        "legs fixed; the amplitude is the sum over all slices).  Output index j has bit i "
        "equal to the value of open site i."),
        "rows": ROWS, "cols": COLS, "depth": DEPTH, "seed": 0, "x1": str(x1),
        "open_sites": OPEN_SITES, "cuts": [list(c) for c in cl], "n_slices": str(n_sl),
        "slices": [], "zero_slices": []}
    tried = {}                      # slice id -> (amplitudes, seconds) of every contracted candidate
    if os.path.exists(OUT):
        with open(OUT) as f:
            old = json.load(f)
        if {k: old.get(k) for k in ("x1", "cuts", "open_sites")} == \
                {k: data[k] for k in ("x1", "cuts", "open_sites")}:
            for s in old.get("slices", []) + old.get("zero_slices", []):
                tried[int(s["slice"])] = (np.array(s["re"]) + 1j * np.array(s["im"]), s["oracle_seconds"])

    def entry(sid):
        amps, dt = tried[sid]
        return {"slice": str(sid), "re": [float(v) for v in amps.real],
                "im": [float(v) for v in amps.imag], "norm": float(np.linalg.norm(amps)),
                "oracle_seconds": dt}

    for sid in candidates(circ, x1, cl):
        if sid not in tried:
            t0 = time.perf_counter()
            amps = network.amplitudes_open(circ, x1, OPEN_SITES, network.slice_fixed_legs(circ, cl, sid))
            tried[sid] = (amps, round(time.perf_counter() - t0, 1))
            print(f"slice {sid}: norm {np.linalg.norm(amps):.6e}, {tried[sid][1]} s", flush=True)
        top = max(np.linalg.norm(a) for a, _ in tried.values())
        nonzero = [k for k in tried if np.linalg.norm(tried[k][0]) >= 1e-9 * top]
        data["slices"] = [entry(k) for k in nonzero]
        data["zero_slices"] = [entry(k) for k in tried if k not in nonzero]
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1)
        if len(nonzero) >= args.nonzero:
            break


if __name__ == "__main__":
    main()
