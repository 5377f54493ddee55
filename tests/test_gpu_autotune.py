"""Autotuner: timing writes a cache covering every step shape, and tuned plans produce
the same amplitudes (every variant computes the same products)."""
import json

import numpy as np
import pytest

import rqc_inputs as ri

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autotune_writes_cache_and_keeps_results(qfx, tmp_path):
    c = ri.rqc(6, 6, 24, seed=3)
    plan = qfx.Plan(qfx.Circuit(c), n_open=5)
    cache = str(tmp_path / "tune.json")
    qfx.autotune(plan, cache)
    qfx.sync()
    entries = json.load(open(cache))["entries"]
    keys = {(e["N"], e["K"], e["NL"], e["Sd"]) for e in entries}
    for s in plan.steps[1:]:
        assert (s["N"], s["K"], s["NL"], s["Sd"]) in keys
    tuned = qfx.Plan(qfx.Circuit(c), n_open=5, autotune_cache=cache)
    x1 = torch.tensor(ri.random_bitstrings(36, 2, seed=1).view(np.int64), device="cuda")
    a = qfx.amplitudes(plan, x1).cpu().numpy()
    b = qfx.amplitudes(tuned, x1).cpu().numpy()
    qfx.sync()
    assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    # re-running keeps existing entries (no re-timing) and the file stays valid
    qfx.autotune(tuned, cache)
    assert len(json.load(open(cache))["entries"]) == len(entries)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_autotune_chooses_between_tensor_cores_and_fp32_tiles(qfx, tmp_path, prec):
    """For a split-precision plan the tensor-core kernel is one more timed candidate: the
    cache records the plan's precision with each shape, the tuned plan takes each step
    from the cache (tensor cores or an FP32 tile), and its amplitudes stay within the
    mode's bound of the FP32 plan (FP32 tiles are at least as accurate)."""
    c = ri.rqc(6, 6, 24, seed=4)
    plan = qfx.Plan(qfx.Circuit(c), n_open=5, precision=prec)
    cache = str(tmp_path / "tune_tc.json")
    qfx.autotune(plan, cache)
    qfx.sync()
    code = {"bf16x3": 1, "tf32x3": 2}[prec]
    entries = {(e["N"], e["K"], e["NL"], e["Sd"]): e for e in json.load(open(cache))["entries"]
               if e.get("prec") == code}
    for s in plan.steps[1:]:
        assert (s["N"], s["K"], s["NL"], s["Sd"]) in entries
    tuned = qfx.Plan(qfx.Circuit(c), n_open=5, precision=prec, autotune_cache=cache)
    for s in tuned.steps[1:]:
        e = entries[(s["N"], s["K"], s["NL"], s["Sd"])]
        assert (s["variant"] >= 10) == (e["variant"] >= 10)
    # an FP32 plan of the same circuit ignores the split-precision entries
    fp = qfx.Plan(qfx.Circuit(c), n_open=5, autotune_cache=cache)
    assert all(s["variant"] < 10 for s in fp.steps)
    x1 = torch.tensor(ri.random_bitstrings(36, 2, seed=1).view(np.int64), device="cuda")
    ref = qfx.amplitudes(fp, x1).cpu().numpy()
    got = qfx.amplitudes(tuned, x1).cpu().numpy()
    qfx.sync()
    assert np.linalg.norm(got - ref) <= 3e-5 * np.linalg.norm(ref)
