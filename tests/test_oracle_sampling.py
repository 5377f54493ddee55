"""Pins of the sampling oracle (Sec. III.B fast sampling with frugal rejection, Sec. III.C
noisy sampling from a fraction of the paths).  CPU only.

- Closed forms: zero variates accept the first nonzero candidate in scan order; an
  acceptance of at least 1 takes scan position 0 (x2 = mask); the comparison is strict at
  an exactly representable threshold; no acceptance gives -1.
- The sample distribution of one batch, over random masks and variates, matches the
  distribution enumerated over all masks (Monte Carlo against an exact sum).
- Samples from the exact state vector of a 4x4x(1+24+1) RQC have the linear
  cross-entropy fidelity N sum p^2 - 1 of the ideal distribution; uniform bitstrings
  have 0.
- Amplitudes summed over a quarter of the paths of a 4x4x(1+24+1) RQC with two cut bonds
  (64 paths) sample at fidelity about 1/4.  The paths come from state vectors of the
  circuit with each cut CZ replaced by one term of its split, and one of them is checked
  against the tensor-network oracle's slice.
- Planted mistakes (a non-strict threshold, an ignored scan mask, a missing 2^n in the
  acceptance) each fail one of these pins.
"""
import copy

import numpy as np
import pytest

import rqc_inputs as ri
from oracle import network, sampling, statevector


def test_zero_variates_accept_first_nonzero_candidate():
    amps = np.zeros(16, dtype=np.complex128)
    amps[[3, 9, 12]] = [1e-3, 0.2j, 0.5]
    u = np.zeros(16)
    for mask in range(16):
        order = [t ^ mask for t in range(16)]
        want = next(x for x in order if amps[x] != 0)
        assert sampling.frugal_select(amps, 10, 10.0, u, mask) == want


def test_certain_acceptance_takes_scan_position_zero():
    amps = np.full(8, 0.5 + 0.5j)          # 2^4 * 0.5 / M = 8 / M >= 1 for M <= 8
    u = np.full(8, np.nextafter(1.0, 0.0))
    for mask in range(8):
        assert sampling.frugal_select(amps, 4, 8.0, u, mask) == mask


def test_threshold_is_strict_and_exact():
    # n = 2, |amp|^2 = 1/4, M = 2: acceptance = 4 * 0.25 / 2 = 0.5 exactly
    amps = np.array([0.5, 0.0], dtype=np.complex128)
    assert sampling.acceptance(amps[0], 2, 2.0) == 0.5
    assert sampling.frugal_select(amps, 2, 2.0, np.array([0.5, 0.0]), 0) == -1
    assert sampling.frugal_select(amps, 2, 2.0, np.array([np.nextafter(0.5, 0.0), 0.0]), 0) == 0


def test_no_acceptance_gives_minus_one():
    amps = ri.random_complex(32, seed=4).astype(np.complex128) * 1e-6
    u = np.full(32, 0.5)
    assert sampling.frugal_select(amps, 8, 1e3, u, 7) == -1


def test_assemble_replaces_open_bits():
    assert sampling.assemble(0b101101, 0b10, [0, 3]) == 0b101100 | (1 << 3)
    assert sampling.assemble(0, 0b111, [5, 1, 9]) == (1 << 5) | (1 << 1) | (1 << 9)
    assert sampling.assemble((1 << 40) - 1, 0, [39, 0]) == ((1 << 40) - 1) & ~(1 << 39) & ~1


def test_batch_distribution_matches_enumeration_over_masks():
    # target acceptances for 8 candidates (n = 6, M = 4: a = 16 |amp|^2)
    a = np.array([0.1, 0.3, 0.0, 0.9, 0.2, 1.5, 0.05, 0.4])
    amps = np.sqrt(a / 16.0).astype(np.complex128)
    n, M, k = 6, 4.0, 3
    # exact: P(y) = mean over masks of prod_{earlier t} (1 - min(1, a)) * min(1, a_y)
    c = np.minimum(1.0, a)
    exact = np.zeros(9)                      # index 8 = no sample
    for mask in range(8):
        keep = 1.0
        for t in range(8):
            y = t ^ mask
            exact[y] += keep * c[y] / 8
            keep *= 1.0 - c[y]
        exact[8] += keep / 8
    rng = np.random.default_rng(11)
    trials = 60000
    counts = np.zeros(9)
    masks = rng.integers(0, 8, size=trials)
    us = rng.random((trials, 8))
    for i in range(trials):
        y = sampling.frugal_select(amps, n, M, us[i], int(masks[i]))
        counts[8 if y < 0 else y] += 1
    freq = counts / trials
    sigma = np.sqrt(np.maximum(exact * (1 - exact), 1e-12) / trials)
    assert np.all(np.abs(freq - exact) <= 5 * sigma + 1e-12), (freq, exact)
    assert counts[2] == 0                    # zero amplitude is never sampled


@pytest.fixture(scope="module")
def rqc_4x4x24():
    c = ri.rqc(4, 4, 24, seed=0)
    return c, statevector.state(c)


def _xeb_sigma(p_samples, n):
    v = (2.0 ** n) * np.asarray(p_samples)
    return float(np.std(v) / np.sqrt(len(v)))


def test_ideal_samples_have_ideal_xeb(rqc_4x4x24):
    c, psi = rqc_4x4x24
    n = c.n_qubits
    p = np.abs(psi) ** 2
    open_sites = [12, 13, 14, 15]
    x1s, masks, u = ri.sampling_draws(n, 4, 3000, seed=5)

    def amp_fn(x1):
        return psi[[sampling.assemble(x1, x2, open_sites) for x2 in range(16)]]

    smp = sampling.frugal_sample(amp_fn, n, open_sites, x1s, masks, u, 10.0)
    # acceptance per batch 1 - (1 - 1/M)^16 for Porter-Thomas amplitudes
    assert abs(len(smp) / 3000 - (1 - 0.9 ** 16)) < 0.04
    assert all((s & ~((1 << n) - 1)) == 0 for s in smp)
    ideal = (2.0 ** n) * np.sum(p * p) - 1
    got = sampling.linear_xeb(p[smp], n)
    assert abs(got - ideal) < 4 * _xeb_sigma(p[smp], n), (got, ideal)
    uni = x1s.astype(np.int64)
    assert abs(sampling.linear_xeb(p[uni], n)) < 4 * _xeb_sigma(p[uni], n)


def _path_state(c, cuts, sid):
    """State vector of path `sid`: each cut CZ replaced by the term of its split that the
    slice fixes, delta(b_lo, k) D(k, b_hi)."""
    c2 = copy.deepcopy(c)
    for gi, k in network.slice_fixed_legs(c, cuts, sid).items():
        d = np.asarray(c2.gates[gi].mat).reshape(-1)
        t = np.zeros(4, dtype=np.complex128)
        t[2 * k], t[2 * k + 1] = d[2 * k], d[2 * k + 1]
        c2.gates[gi].mat = t
    return statevector.state(c2)


def test_quarter_of_the_paths_samples_at_fidelity_a_quarter(rqc_4x4x24):
    c, psi = rqc_4x4x24
    n = c.n_qubits
    cuts = [(5, 9, 1), (6, 10, 1)]
    S = network.n_slices(c, cuts)
    assert S == 64
    open_sites = [12, 13, 14, 15]
    part = [_path_state(c, cuts, sid) for sid in range(S // 4)]
    # the path construction agrees with the network oracle's slice
    sl = network.amplitudes_sliced(c, 0b0000101100110101, open_sites, cuts, [3])
    want = part[3][[sampling.assemble(0b0000101100110101, x2, open_sites) for x2 in range(16)]]
    np.testing.assert_allclose(sl, want, atol=1e-13)
    amp_f = np.sum(part, axis=0)
    norm = float(np.sum(np.abs(amp_f) ** 2))
    assert abs(norm - 0.25) < 0.02
    p = np.abs(psi) ** 2
    q = np.abs(amp_f) ** 2 / norm
    xeb_q = (2.0 ** n) * np.sum(p * q) - 1
    assert abs(xeb_q - 0.25) < 0.03
    x1s, masks, u = ri.sampling_draws(n, 4, 3000, seed=6)

    def amp_fn(x1):
        return amp_f[[sampling.assemble(x1, x2, open_sites) for x2 in range(16)]]

    smp = sampling.frugal_sample(amp_fn, n, open_sites, x1s, masks, u, 10.0 * 0.25)
    got = sampling.linear_xeb(p[smp], n)
    assert abs(got - xeb_q) < 4 * _xeb_sigma(p[smp], n), (got, xeb_q)


# --- planted mistakes: each must be caught by a pin above ---------------------------

def _select_with(accept_cmp, use_mask=True):
    def select(amps, n, M, u, mask):
        for t in range(len(amps)):
            x2 = t ^ int(mask) if use_mask else t
            if accept_cmp(float(u[t]), sampling.acceptance(amps[x2], n, M)):
                return x2
        return -1
    return select


def test_planted_non_strict_threshold_is_caught(monkeypatch):
    monkeypatch.setattr(sampling, "frugal_select", _select_with(lambda u, a: u <= a))
    with pytest.raises(AssertionError):
        test_threshold_is_strict_and_exact()


def test_planted_ignored_scan_mask_is_caught(monkeypatch):
    monkeypatch.setattr(sampling, "frugal_select", _select_with(lambda u, a: u < a, use_mask=False))
    with pytest.raises(AssertionError):
        test_zero_variates_accept_first_nonzero_candidate()


def test_planted_missing_dimension_factor_is_caught(monkeypatch):
    # acceptance |amp|^2 / M instead of 2^n |amp|^2 / M
    monkeypatch.setattr(sampling, "acceptance",
                        lambda amp, n, M: (amp.real ** 2 + amp.imag ** 2) / M)
    with pytest.raises(AssertionError):
        test_batch_distribution_matches_enumeration_over_masks()
