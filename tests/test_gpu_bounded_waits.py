"""Bounded device waits that run out: the batch scheduler's dependency wait and the
permute's copy wait.  Test hooks make one wait impossible to satisfy (a dependency count
no task reaches; copies that are never issued) with a 1 ms limit.  The waiting kernel must
record QFX_ETIMEOUT, every CTA must return, and the context must stay usable: a normal
call afterwards gives the same results as before.  Nothing here faults or hangs the GPU."""
import numpy as np
import pytest

import rqc_inputs as ri

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WAIT_NS = 1_000_000   # 1 ms


def _items(qfx):
    out = []
    for rows, cols, d, seed, no in [(4, 4, 16, 0, 4), (5, 5, 24, 1, 3), (3, 5, 16, 3, 5)]:
        plan = qfx.Plan(qfx.Circuit(ri.rqc(rows, cols, d, seed=seed)), n_open=no)
        x1 = torch.tensor(ri.random_bitstrings(rows * cols, 2, seed=seed + 5).view(np.int64),
                          device="cuda")
        out.append((plan, x1, 0, None))
    return out


def test_batch_dependency_wait_expires(qfx):
    items = _items(qfx)
    good = qfx.Batch(items, slots=2)
    want = [o.cpu().numpy() for o in good.run()]
    qfx.sync()
    bad = qfx.Batch(items, slots=2)
    bad.debug_stall(WAIT_NS)
    bad.run()
    with pytest.raises(qfx.QfxError) as e:
        qfx.sync()
    assert e.value.status == qfx.qfx.QFX_ETIMEOUT
    qfx.sync()                                     # the status word was cleared
    del bad
    again = [o.cpu().numpy() for o in good.run()]  # context still usable
    qfx.sync()
    for a, b in zip(again, want):
        np.testing.assert_array_equal(a, b)


def test_permute_copy_wait_expires(qfx):
    shape, perm = (130, 72), (1, 0)                # a tensor-map transpose
    x = torch.from_numpy(ri.random_complex(130 * 72, seed=4)).cuda()
    want = qfx.permute(x, shape, perm).cpu().numpy()
    qfx.sync()
    qfx.debug_permute_withhold(WAIT_NS)
    qfx.permute(x, shape, perm)
    with pytest.raises(qfx.QfxError) as e:
        qfx.sync()
    assert e.value.status == qfx.qfx.QFX_ETIMEOUT
    got = qfx.permute(x, shape, perm).cpu().numpy()   # the hook covered one call only
    qfx.sync()
    np.testing.assert_array_equal(got, want)


def test_hooks_reject_bad_limits(qfx):
    with pytest.raises(qfx.QfxError):
        qfx.debug_permute_withhold(10)
    b = qfx.Batch(_items(qfx)[:1], slots=1)
    with pytest.raises(qfx.QfxError):
        b.debug_stall(10**12)
