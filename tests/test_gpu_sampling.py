"""Fast sampling with frugal rejection (qfx_frugal_select / frugal_sample) against the
sampling oracle (Sec. III.B, III.C).

- On the same amplitudes, variates and masks, the selected x2 and the assembled
  bitstrings are bit-identical to the oracle's.  Both sides decide in FP64 with the
  same rounding (p = re*re + im*im, then p * (2^n / M)).
- End to end, the GPU's FP32 amplitudes and the oracle's FP64 ones may put an acceptance
  on the other side of a variate.  A batch is compared only where every variate up to the
  later of the two choices lies farther from its acceptance than the FP32 parity bound
  allows (|a - a_ref| <= 2e-5 max(a, sqrt(a / M)), from the per-amplitude bound
  1e-5 max(|amp|, 2^(-n/2))); at least 95% of the batches must be comparable.
"""
import numpy as np
import pytest

import rqc_inputs as ri
from oracle import network, sampling, statevector

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to(dtype).to("cuda")


def oracle_select(amps, x1s, masks, u, n, M, open_sites):
    x2 = np.array([sampling.frugal_select(amps[b], n, M, u[b], int(masks[b]))
                   for b in range(len(x1s))], dtype=np.int64)
    bits = np.array([sampling.assemble(int(x1s[b]), int(x2[b]), open_sites) if x2[b] >= 0
                     else int(x1s[b]) for b in range(len(x1s))], dtype=np.uint64)
    return x2, bits


@pytest.mark.parametrize("n_open,n_batch", [(0, 5), (1, 7), (4, 37), (6, 64), (9, 33), (12, 3)])
def test_select_matches_oracle_bitwise(qfx, n_open, n_batch):
    rows, cols = 4, 4
    n = rows * cols
    c = ri.rqc(rows, cols, 8, seed=1)
    plan = qfx.Plan(qfx.Circuit(c), n_open=n_open)
    open_sites = plan.open_sites
    per = 1 << n_open
    x1s, masks, u = ri.sampling_draws(n, n_open, n_batch, seed=100 + n_open)
    # |amp|^2 ~ Exp(1) / N (Porter-Thomas scale), M = 10: acceptance ~ 0.1 per candidate
    amps = ri.random_complex((n_batch, per), seed=7 + n_open).astype(np.complex128)
    amps *= np.sqrt(0.5 / 2.0 ** n)
    if per > 256:
        amps[0, [t ^ int(masks[0]) for t in range(300)]] = 0   # first acceptance past the first 256-candidate scan
    amps[-1, :] *= 1e-6                                          # (almost surely) no sample
    M = 10.0
    want_x2, want_bits = oracle_select(amps, x1s, masks, u, n, M, open_sites)
    x2, bits = qfx.frugal_select(plan, dev(x1s.view(np.int64)), dev(amps), dev(u),
                                 dev(masks.view(np.int64)), M)
    qfx.sync()
    np.testing.assert_array_equal(x2.cpu().numpy(), want_x2)
    np.testing.assert_array_equal(bits.cpu().numpy().view(np.uint64), want_bits)
    if per > 256:
        assert want_x2[0] >= 0 and (int(want_x2[0]) ^ int(masks[0])) >= 300


def test_select_threshold_ties_are_rejected(qfx):
    # amp = 1/8: |amp|^2 = 2^-6, n = 16, M = 2048: acceptance = 2^16 * 2^-6 / 2^11 = 0.5
    # exactly; a variate on the threshold is rejected, one just below it accepted
    c = ri.rqc(4, 4, 8, seed=1)
    plan = qfx.Plan(qfx.Circuit(c), n_open=1)
    amps = np.full((2, 2), 0.125 + 0j)
    u = np.array([[0.5, 0.5], [np.nextafter(0.5, 0.0), 0.5]])
    masks = np.zeros(2, dtype=np.uint64)
    x1s = np.zeros(2, dtype=np.uint64)
    assert sampling.acceptance(amps[0, 0], 16, 2048.0) == 0.5
    x2, _ = qfx.frugal_select(plan, dev(x1s.view(np.int64)), dev(amps), dev(u),
                              dev(masks.view(np.int64)), 2048.0)
    qfx.sync()
    assert x2.cpu().tolist() == [-1, 0]


def comparable(a_ref, u, masks, x2_a, x2_b, M):
    """Batches whose decisions cannot flip within the FP32 parity bound."""
    ok = []
    for b in range(len(masks)):
        ts = [int(x) ^ int(masks[b]) for x in (x2_a[b], x2_b[b]) if x >= 0]
        last = max(ts) if len(ts) == 2 else a_ref.shape[1] - 1
        t = np.arange(last + 1)
        a = a_ref[b, t ^ int(masks[b])]
        margin = 2e-5 * np.maximum(a, np.sqrt(a / M)) + 1e-12
        ok.append(bool(np.all(np.abs(u[b, t] - a) > margin)))
    return np.array(ok)


def test_frugal_sample_4x4x16_matches_state_vector(qfx):
    c = ri.rqc(4, 4, 16, seed=3)
    n = c.n_qubits
    psi = statevector.amplitudes(c)
    plan = qfx.Plan(qfx.Circuit(c), n_open=4)
    open_sites = plan.open_sites
    x1s, masks, u = ri.sampling_draws(n, 4, 256, seed=21)
    M = 10.0
    ref = np.array([[psi[sampling.assemble(int(x1), x2, open_sites)] for x2 in range(16)]
                    for x1 in x1s])
    want_x2, want_bits = oracle_select(ref, x1s, masks, u, n, M, open_sites)
    x2, bits, amps = qfx.frugal_sample(plan, dev(x1s.view(np.int64)), dev(u),
                                       dev(masks.view(np.int64)), M)
    qfx.sync()
    x2, bits = x2.cpu().numpy(), bits.cpu().numpy().view(np.uint64)
    a_ref = (2.0 ** n) * np.abs(ref) ** 2 / M
    ok = comparable(a_ref, u, masks, x2, want_x2, M)
    assert ok.mean() >= 0.95
    np.testing.assert_array_equal(x2[ok], want_x2[ok])
    np.testing.assert_array_equal(bits[ok], want_bits[ok])
    assert (x2 >= 0).mean() > 0.7          # 1 - 0.9^16 = 0.81 expected


def test_noisy_sampling_quarter_of_the_slices(qfx):
    # two cut bonds of 4 values each on 4x4x16 (16 paths); the first 4 slices
    c = ri.rqc(4, 4, 16, seed=3)
    n = c.n_qubits
    cuts = [(5, 9, 1), (6, 10, 1)]
    plan = qfx.Plan(qfx.Circuit(c), n_open=4, cuts=cuts)
    assert plan.n_slices == 16
    open_sites = plan.open_sites
    x1s, masks, u = ri.sampling_draws(n, 4, 48, seed=22)
    M = 10.0 * 0.25
    ref = np.array([network.amplitudes_sliced(c, int(x1), open_sites, cuts, range(4))
                    for x1 in x1s])
    want_x2, want_bits = oracle_select(ref, x1s, masks, u, n, M, open_sites)
    x2, bits, amps = qfx.frugal_sample(plan, dev(x1s.view(np.int64)), dev(u),
                                       dev(masks.view(np.int64)), M, slice_begin=0, slice_end=4)
    qfx.sync()
    x2, bits = x2.cpu().numpy(), bits.cpu().numpy().view(np.uint64)
    a_ref = (2.0 ** n) * np.abs(ref) ** 2 / M
    ok = comparable(a_ref, u, masks, x2, want_x2, M)
    assert ok.mean() >= 0.95
    np.testing.assert_array_equal(x2[ok], want_x2[ok])
    np.testing.assert_array_equal(bits[ok], want_bits[ok])
