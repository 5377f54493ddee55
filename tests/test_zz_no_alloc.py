"""qfx_amplitudes_static: the entry point for callers that cannot allocate device memory
(a host application whose memory manager owns the device, latency-bound code that cannot
take cudaMalloc's implicit synchronisation, plugins handed only their buffers).  Its
scratch is a 64 MiB array compiled into the library.  This file is collected last on
purpose; it passes alone in a fresh process and after the other tests.

The static path runs the same executor as qfx_amplitudes (same kernels, the same FP64
slice-order sums), so its results must be bit-identical to the workspace path's, whatever
the number of items in flight."""
import numpy as np
import pytest

import rqc_inputs as ri

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case(qfx, rows, cols, depth, seed, n_open, n_x1, cuts=(), precision="fp32"):
    circ = ri.rqc(rows, cols, depth, seed=seed)
    plan = qfx.Plan(qfx.Circuit(circ), n_open=n_open, cuts=cuts, precision=precision)
    x1 = torch.tensor(ri.random_bitstrings(rows * cols, n_x1, seed=seed + 7).view(np.int64),
                      device="cuda")
    return plan, x1


def test_static_scratch_matches_workspace_path(qfx):
    # fresh plans: their first call is the static one (nothing was staged for them before)
    cases = [(_case(qfx, 4, 4, 16, 0, 5, 3), None),
             (_case(qfx, 5, 5, 24, 1, 6, 2, cuts=[(6, 7, 4)]), None),
             (_case(qfx, 5, 5, 24, 1, 6, 2, cuts=[(6, 7, 4)]), (1, 2)),    # one slice of two
             (_case(qfx, 5, 6, 24, 3, 6, 2, precision="bf16x3"), None)]
    assert any(s["variant"] >= 10 for s in cases[3][0][0].steps)        # tensor-core steps
    # two calls in a row through the C ABI, then the first again (the shared array now
    # holds the previous call's tables and tensors)
    got = {}
    for idx in (0, 1, 2, 3, 0):
        (plan, x1), sl = cases[idx]
        sb, se = sl if sl else (0, plan.n_slices)
        out = qfx.amplitudes_static(plan, x1, slice_begin=sb, slice_end=se)
        qfx.sync()
        got.setdefault(idx, []).append(out.cpu().numpy())
    # the existing entry point with a caller workspace (two items in flight)
    for idx, ((plan, x1), sl) in enumerate(cases):
        sb, se = sl if sl else (0, plan.n_slices)
        ws = torch.empty(plan.workspace_bytes(2), dtype=torch.uint8, device="cuda")
        ref = qfx.amplitudes(plan, x1, slice_begin=sb, slice_end=se, workspace=ws)
        qfx.sync()
        for g in got[idx]:
            np.testing.assert_array_equal(g, ref.cpu().numpy())


def test_static_scratch_rejects_large_plans(qfx):
    plan, x1 = _case(qfx, 7, 7, 24, 0, 6, 1)      # needs 2 x 128 MiB of boundary
    assert plan.workspace_bytes(1) > qfx.qfx.STATIC_SCRATCH_BYTES
    with pytest.raises(qfx.QfxError) as e:
        qfx.amplitudes_static(plan, x1)
    assert e.value.status == qfx.qfx.QFX_ENOMEM
    assert "static array holds 67108864" in str(e.value)
