"""Host-side parts of bench.py: the constants its CPU figures are counted in match the
planner, the oracle legs run, the reference arm prints the contract's line with the same
config as the GPU arm, and the summary of a line holds every part's figures."""
import json
import os
import subprocess
import sys

import numpy as np

import rqc_inputs as ri

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_full_route_constants_match_the_planner():
    import paper_1905_00444_gb300 as qfx
    plan = qfx.Plan(qfx.Circuit(ri.rqc(7, 7, 24, seed=0)), n_open=6)
    assert plan.stats["flops_per_item"] == bench.FLOPS_7x7x24
    assert plan.open_sites == bench.OPEN_7x7
    plan32 = qfx.Plan(qfx.Circuit(ri.rqc(7, 7, 32, seed=0)), n_open=6)
    assert plan32.open_sites == bench.OPEN_7x7


def test_step_sample_counts_the_dominant_step():
    rate, reps, dt = bench.cpu_step_sample(seconds=0.01, cols=1 << 8)
    assert reps >= 1 and dt > 0
    assert rate == 8.0 * 256 * 256 * (1 << 8) * reps / dt / 1e12


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=300, check=True).stdout.strip().splitlines()
    line = json.loads(out[-1])
    assert line["impl"] == "reference" and line["unit"] == "TFLOP/s" and line["value"] > 0
    assert line["config"] == bench.shared_config(bench.WORKLOADS["full"])
    assert line["cpu_baseline"]["cores"] == os.cpu_count()
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_summary_holds_every_part():
    clk = {"sm_mhz": 2070.0}
    mode = {"value": 264.0, "roofline": {"tensor_probe": {"frac": 0.74}}, "max_rel_diff_vs_fp32": 4e-6,
            "clocks": clk}
    line = {"value": 55.2, "roofline": {"frac": 0.70}, "e2e": {"value": 55.1}, "clocks": clk,
            "precision_modes": {"bf16x3": mode},
            "adjoint": {"forward_ms": 1.0, "backward_ms": 3.9, "roofline": {"frac": 0.18},
                        "graph_forward_backward_ms": 4.5},
            "permute": {"cases": [{"frac": 0.75}, {"frac": 0.9}]},
            "batch": {"fp32_persistent": {"value": 41.6}, "fp32_per_item": {"value": 48.2},
                      "bf16x3_graph": {"value": 157.7}, "bf16x3_per_item": {"value": 153.6}},
            "region": {"value": 280.0, "roofline": {"tensor_probe": {"frac": 0.76}},
                       "amplitudes_per_s_at_fidelity_0.006": 6.7},
            "cpu_baseline": {"value": 0.01, "cores": 16, "step_sample": {"value": 0.1}}}
    s = bench.summarize(line)
    assert set(s) == {"fp32", "bf16x3", "adjoint", "permute_frac", "batch_tflops", "region_7x7x40_bf16x3", "cpu"}
    assert s["batch_tflops"]["persistent"] == 41.6 and s["fp32"]["frac"] == 0.7
    assert len(json.dumps(s)) < 1000
    assert np.isclose(s["bf16x3"]["err_vs_fp32"], 4e-6)
