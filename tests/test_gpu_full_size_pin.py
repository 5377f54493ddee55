"""The benchmarked workload itself -- 7x7x(1+32+1), seed 0, T gates, the benchmark's first
x1 and its six open sites -- against FP64 oracle values, element by element.

The uncut oracle needs 2^32 complex128 values per tensor plus a pairwise contraction's
temporaries, more host memory than is available, so the pin is per slice (Sec. III.A):
the 12 vertical bonds of grid columns 0 and 6 are cut to single values and
``tests/golden/make_rqc_7x7x32_slices.py`` stored the oracle's partial amplitudes of a few
seeded slices.  Under that cut the GPU plan keeps every step of columns 1..5 exactly as
in the uncut benchmark plan -- all 25 dominant steps (K = N = 256, P * Sd = 2^24) among
them -- so each slice runs the benchmarked contraction at full size.

Tolerance: per amplitude |a - a_ref| <= bound * max(|a_ref|, rms(a_ref)) and normwise
<= bound, with rms(a_ref) the slice's root-mean-square partial amplitude (the analogue of
the 2^(-n/2) floor of whole amplitudes); bound = 1e-5 for FP32 and each split mode's
stated bound (BF16x3 1e-5, TF32x3 3e-5, BF16x2 2e-4).  Slices whose oracle norm is below
1e-9 of the largest stored one are exact zeros computed as rounding noise and are skipped.
"""
import json
import os

import numpy as np
import pytest

import rqc_inputs as ri

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rqc_7x7x32_slices.json")
BOUND = {"fp32": 1e-5, "bf16x3": 1e-5, "tf32x3": 3e-5, "bf16x2": 2e-4}


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _usable(g):
    top = max(s["norm"] for s in g["slices"])
    return [s for s in g["slices"] if s["norm"] >= 1e-9 * top]


def _plans(qfx, g, precision="fp32"):
    circ = qfx.Circuit(ri.rqc(g["rows"], g["cols"], g["depth"], seed=g["seed"]))
    cuts = [tuple(c) for c in g["cuts"]]
    bench = qfx.Plan(circ, n_open=6, precision=precision)
    pinned = qfx.Plan(circ, n_open=6, cuts=cuts, precision=precision)
    return bench, pinned


def test_golden_inputs_are_the_benchmark_workload():
    """Host only: the stored slices use the benchmark's circuit seed, first x1 and its
    planner-chosen open sites, and enough of them are nonzero to pin anything."""
    g = _golden()
    assert (g["rows"], g["cols"], g["depth"], g["seed"]) == (7, 7, 32, 0)
    assert int(g["x1"]) == int(ri.random_bitstrings(49, 1, seed=1000)[0])
    assert int(g["n_slices"]) == 16 ** 12
    assert len(_usable(g)) >= 3
    for s in g["slices"]:
        assert len(s["re"]) == len(s["im"]) == 64


def test_cut_plan_keeps_the_benchmark_steps():
    """Host only: under the 12 vertical cuts every step of grid columns 1..5 has the shape
    it has in the uncut benchmark plan, and the open sites are the benchmark's."""
    import paper_1905_00444_gb300 as qfx
    g = _golden()
    bench, pinned = _plans(qfx, g)
    assert bench.open_sites == pinned.open_sites == g["open_sites"]
    assert pinned.n_slices == int(g["n_slices"])
    same = 0
    for a, b in zip(bench.steps, pinned.steps):
        assert a["site"] == b["site"]
        if a["site"] % 7 in (1, 2, 3, 4, 5):
            assert (a["P"], a["K"], a["N"], a["NL"], a["Sd"]) == (b["P"], b["K"], b["N"], b["NL"], b["Sd"])
            same += (a["K"], a["N"], a["P"] * a["Sd"]) == (256, 256, 1 << 24)
    assert same == 25


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32x3", "bf16x2"])
def test_7x7x32_slices_vs_oracle(qfx, precision):
    torch = pytest.importorskip("torch")
    g = _golden()
    _, plan = _plans(qfx, g, precision)
    x1 = torch.tensor(np.array([int(g["x1"])], dtype=np.uint64).view(np.int64), device="cuda")
    ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    bound = BOUND[precision]
    for s in _usable(g):
        sid = int(s["slice"])
        want = np.array(s["re"]) + 1j * np.array(s["im"])
        got = qfx.amplitudes(plan, x1, slice_begin=sid, slice_end=sid + 1, workspace=ws)
        qfx.sync()
        got = got.cpu().numpy()[0]
        rms = np.linalg.norm(want) / np.sqrt(want.size)
        err = np.abs(got - want)
        lim = bound * np.maximum(np.abs(want), rms)
        worst = int(np.argmax(err / lim))
        assert np.all(err <= lim), (sid, worst, got[worst], want[worst])
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= bound, sid
