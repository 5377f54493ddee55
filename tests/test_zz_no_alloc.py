"""qfx_amplitudes_static: the entry point for callers that cannot allocate device memory
(a host application whose memory manager owns the device, latency-bound code that cannot
take cudaMalloc's implicit synchronisation, plugins handed only their buffers).  Its
scratch is a 64 MiB array compiled into the library.  This file is collected last on
purpose; it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

import rqc_inputs as ri

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-5


def _close(got, want, n):
    floor = 2.0 ** (-n / 2)
    err = np.abs(got - want)
    assert np.all(err <= REL * np.maximum(np.abs(want), floor))
    assert np.linalg.norm(got - want) <= REL * np.linalg.norm(want)


def _case(qfx, rows, cols, depth, seed, n_open, n_x1, cuts=()):
    circ = ri.rqc(rows, cols, depth, seed=seed)
    plan = qfx.Plan(qfx.Circuit(circ), n_open=n_open, cuts=cuts)
    x1 = torch.tensor(ri.random_bitstrings(rows * cols, n_x1, seed=seed + 7).view(np.int64),
                      device="cuda")
    return plan, x1


def test_static_scratch_matches_workspace_path(qfx):
    cases = [_case(qfx, 4, 4, 16, 0, 5, 3),
             _case(qfx, 5, 5, 24, 1, 6, 2, cuts=[(6, 7, 4)])]
    # reference results through the existing entry point (caller workspace)
    refs = []
    for plan, x1 in cases:
        ws = torch.empty(plan.workspace_bytes(2), dtype=torch.uint8, device="cuda")
        refs.append(qfx.amplitudes(plan, x1, workspace=ws).cpu().numpy())
    qfx.sync()
    # two calls in a row through the C ABI, then the first again (the shared array now
    # holds the second call's tables and tensors)
    for idx in (0, 1, 0):
        plan, x1 = cases[idx]
        got = qfx.amplitudes_static(plan, x1)
        qfx.sync()
        _close(got.cpu().numpy(), refs[idx], plan.stats["n_sites"])


def test_static_scratch_rejects_large_plans(qfx):
    plan, x1 = _case(qfx, 7, 7, 24, 0, 6, 1)      # needs 2 x 128 MiB of boundary
    assert plan.workspace_bytes(1) > qfx.qfx.STATIC_SCRATCH_BYTES
    with pytest.raises(qfx.QfxError) as e:
        qfx.amplitudes_static(plan, x1)
    assert e.value.status == qfx.qfx.QFX_ENOMEM
    assert "static array holds 67108864" in str(e.value)
