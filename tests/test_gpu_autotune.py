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
