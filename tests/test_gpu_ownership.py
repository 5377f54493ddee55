"""Ownership of device memory: the compute entry points allocate nothing.

Each call copies the plan's table image into the caller's workspace; nothing is kept on
the device between calls.  Product circuits of depth 200 on an 8x8 grid have about
1.2 MB of tables each, so a per-plan device upload of four of them would move the
device's free memory (allocations come in 2 MiB pages)."""
import numpy as np
import pytest

import rqc_inputs as ri
from oracle import network

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_first_calls_with_new_plans_allocate_nothing(qfx):
    # seeds whose qubits all keep both amplitudes well away from zero (seed 3 has one
    # that is exactly zero, which FP64 rounding turns into noise of either sign)
    circs = [ri.product_circuit(8, 8, 200, seed=s) for s in (0, 1, 2, 4, 5)]
    plans = [qfx.Plan(qfx.Circuit(c), n_open=2) for c in circs]
    x1v = int(ri.random_bitstrings(64, 1, seed=3)[0])
    x1 = torch.tensor(np.array([x1v], dtype=np.uint64).view(np.int64), device="cuda")
    ws = torch.empty(max(p.workspace_bytes(1) for p in plans), dtype=torch.uint8, device="cuda")
    outs = [torch.empty((1, 4), dtype=torch.complex128, device="cuda") for _ in plans]
    # the first plan loads the library's kernels on this device
    qfx.amplitudes(plans[0], x1, workspace=ws, out=outs[0])
    qfx.sync()
    free0, _ = torch.cuda.mem_get_info()
    for p, o in zip(plans[1:], outs[1:]):
        qfx.amplitudes(p, x1, workspace=ws, out=o)    # first call with each plan
    qfx.sync()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for c, p, o in zip(circs, plans, outs):
        want = network.amplitudes_open(c, x1v, p.open_sites)
        got = o.cpu().numpy()[0]
        assert np.allclose(got, want, rtol=1e-5, atol=1e-5 * np.abs(want).max())


def test_workspace_holds_the_tables(qfx):
    """workspace_min covers the tables: one byte less is refused with QFX_ENOMEM."""
    c = ri.rqc(4, 4, 16, seed=2)
    plan = qfx.Plan(qfx.Circuit(c), n_open=3)
    x1 = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(plan.stats["workspace_min"] - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(qfx.QfxError) as e:
        qfx.amplitudes(plan, x1, workspace=ws)
    assert e.value.status == qfx.qfx.QFX_ENOMEM
