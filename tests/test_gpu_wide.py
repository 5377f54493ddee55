"""More than 64 qubits: the paper's 11x11 grid (121 qubits, Table I), bitstrings of two
uint64 words, amplitudes of order 2^-60 (mean |amp|^2 = 2^-121; the per-site power-of-two
scale of Sec. III.E keeps the FP32 contraction away from underflow).

* 11x11x(1+8+1) against the FP64 oracle computed here, 11x11x(1+16+1) against stored
  oracle values (tests/golden/make_rqc_11x11_amplitudes.py), element by element at 1e-5
  with the 2^(-n/2) floor.
* A T-free 11x11x(1+16+1) circuit: |amp|^2 from the stabilizer tableau, exactly.
* 11x11x(1+24+1), the paper's shape, at a 64 GiB cap (2^31 slices): no oracle reaches it,
  so a slice is checked by refinement (halving its last cut gives two slices that sum to
  it, Sec. III.A) and the split precisions against FP32 on it.
* Fast sampling, the batch scheduler and the adjoint with two-word bitstrings.
"""
import json
import os

import numpy as np
import pytest

import rqc_inputs as ri
from oracle import gradient, network, sampling, stabilizer

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rqc_11x11x16_amplitudes.json")


def dev_words(words):
    return torch.tensor(np.ascontiguousarray(words, dtype=np.uint64).view(np.int64), device="cuda")


def expand(x1, open_sites, j):
    x = int(x1)
    for i, q in enumerate(open_sites):
        x = (x & ~(1 << q)) | (((j >> i) & 1) << q)
    return x


def check(got, want, n, rel=REL):
    floor = 2.0 ** (-n / 2)
    err = np.abs(got - want)
    assert np.all(err <= rel * np.maximum(np.abs(want), floor)), float(np.max(err / np.maximum(np.abs(want), floor)))
    assert np.linalg.norm(got - want) <= rel * np.linalg.norm(want)


def test_11x11x8_vs_oracle(qfx):
    c = ri.rqc(11, 11, 8, seed=0)
    plan = qfx.Plan(qfx.Circuit(c), n_open=6)
    assert plan.x1_words == 2
    words = ri.random_bitstring_words(121, 3, seed=2)
    out = qfx.amplitudes(plan, dev_words(words), workspace=torch.empty(
        plan.workspace_bytes(3), dtype=torch.uint8, device="cuda"))
    qfx.sync()
    want = np.array([network.amplitudes_open(c, ri.words_to_int(w), plan.open_sites) for w in words])
    assert out.shape == (3, 64)
    check(out.cpu().numpy(), want, 121)


def test_11x11x16_vs_stored_oracle(qfx):
    with open(GOLDEN) as f:
        g = json.load(f)
    c = ri.rqc(g["rows"], g["cols"], g["depth"], seed=g["seed"])
    plan = qfx.Plan(qfx.Circuit(c), n_open=6)
    assert plan.open_sites == g["open_sites"]
    words = np.array([int(w, 16) for w in g["x1_words"]], dtype=np.uint64)
    out = qfx.amplitudes(plan, dev_words(words[None, :]))
    qfx.sync()
    check(out.cpu().numpy()[0], np.array(g["re"]) + 1j * np.array(g["im"]), 121)


def test_11x11x16_clifford_probabilities_exact(qfx):
    c = ri.rqc(11, 11, 16, seed=4, gate_set=(ri.SQRT_X, ri.SQRT_Y))
    plan = qfx.Plan(qfx.Circuit(c), n_open=6)
    words = ri.random_bitstring_words(121, 1, seed=7)
    out = qfx.amplitudes(plan, dev_words(words))
    qfx.sync()
    x1 = ri.words_to_int(words[0])
    tab = stabilizer.prepare(c)
    probs = np.array([stabilizer.probability(c, expand(x1, plan.open_sites, j), tab) for j in range(64)])
    got = np.abs(out.cpu().numpy()[0])
    floor = 2.0 ** (-121 / 2)
    assert np.any(probs > 0)
    assert np.all(np.abs(got - np.sqrt(probs)) <= REL * np.maximum(np.sqrt(probs), floor))


def test_11x11x24_slice_refinement_and_split_modes(qfx):
    c = ri.rqc(11, 11, 24, seed=0)
    circ = qfx.Circuit(c)
    plan = qfx.Plan(circ, n_open=6, max_intermediate_bytes=64 << 30)
    assert plan.n_slices == 1 << 31 and plan.stats["max_elements"] == 1 << 33
    qa, qb, size = plan.cuts[-1]
    assert size >= 2
    finer = qfx.Plan(circ, n_open=6, cuts=plan.cuts[:-1] + [(qa, qb, size // 2)])
    assert finer.n_slices == 2 * plan.n_slices
    w = ri.random_bitstring_words(121, 1, seed=11)
    words, x1v = dev_words(w), ri.words_to_int(w[0])
    # most slices of these cuts are exactly zero (a fixed leg of the first gate of a bond
    # after sqrt(Y)|+> = |1>, for example, removes a whole site tensor); candidates whose
    # site tensors all survive are tried in seeded order until one is nonzero on the GPU
    rng = np.random.default_rng(3)
    cands = []
    while len(cands) < 8:
        sid = int(rng.integers(0, plan.n_slices))
        fixed = network.slice_fixed_legs(c, plan.cuts, sid)
        if all(np.any(network.site_tensor(c, q, None if q in plan.open_sites else (x1v >> q) & 1,
                                          fixed)[0] != 0) for q in range(121)):
            cands.append(sid)
    ws = torch.empty(max(plan.workspace_bytes(1), finer.workspace_bytes(1)), dtype=torch.uint8,
                     device="cuda")
    for sid in cands:
        coarse = qfx.amplitudes(plan, words, slice_begin=sid, slice_end=sid + 1, workspace=ws).cpu().numpy()
        qfx.sync()
        rms = np.linalg.norm(coarse) / np.sqrt(coarse.size)
        if rms > 0:
            break
    else:
        pytest.fail("no nonzero slice among the candidates")
    fine = qfx.amplitudes(finer, words, slice_begin=2 * sid, slice_end=2 * sid + 2, workspace=ws).cpu().numpy()
    qfx.sync()
    assert np.all(np.abs(fine - coarse) <= REL * np.maximum(np.abs(coarse), rms))
    del ws
    torch.cuda.empty_cache()
    for prec, bound in (("bf16x3", 1e-5), ("tf32x3", 3e-5)):
        p = qfx.Plan(circ, n_open=6, max_intermediate_bytes=64 << 30, precision=prec)
        assert p.cuts == plan.cuts
        ws = torch.empty(p.workspace_bytes(1), dtype=torch.uint8, device="cuda")
        got = qfx.amplitudes(p, words, slice_begin=sid, slice_end=sid + 1, workspace=ws).cpu().numpy()
        qfx.sync()
        del ws
        torch.cuda.empty_cache()
        assert np.all(np.abs(got - coarse) <= bound * np.maximum(np.abs(coarse), rms)), prec


def test_frugal_select_two_word_bitstrings(qfx):
    c = ri.rqc(11, 11, 8, seed=1)
    plan = qfx.Plan(qfx.Circuit(c), n_open=5)
    nb = 6
    words = ri.random_bitstring_words(121, nb, seed=8)
    _, masks, u = ri.sampling_draws(121, 5, nb, seed=9)
    x1 = dev_words(words)
    amps = qfx.amplitudes(plan, x1, workspace=torch.empty(plan.workspace_bytes(2), dtype=torch.uint8,
                                                          device="cuda"))
    x2, bits = qfx.frugal_select(plan, x1, amps, torch.from_numpy(u).cuda(),
                                 torch.from_numpy(masks.view(np.int64)).cuda(), 10.0)
    qfx.sync()
    assert bits.shape == (nb, 2)
    a = amps.cpu().numpy()
    for b in range(nb):
        want = sampling.frugal_select(a[b], 121, 10.0, u[b], int(masks[b]))
        assert int(x2[b]) == want
        x1i = ri.words_to_int(words[b])
        full = x1i if want < 0 else sampling.assemble(x1i, want, plan.open_sites)
        assert ri.words_to_int(bits[b].cpu().numpy().view(np.uint64)) == full


def test_batch_with_two_word_bitstrings(qfx):
    items = []
    for rows, cols, d, seed, nx, words in ((11, 11, 8, 0, 3, True), (4, 4, 16, 1, 2, False)):
        plan = qfx.Plan(qfx.Circuit(ri.rqc(rows, cols, d, seed=seed)), n_open=4)
        if words:
            x1 = dev_words(ri.random_bitstring_words(rows * cols, nx, seed=seed + 3))
        else:
            x1 = torch.tensor(ri.random_bitstrings(rows * cols, nx, seed=seed + 3).view(np.int64), device="cuda")
        items.append((plan, x1, 0, None))
    b = qfx.Batch(items, slots=2)
    outs = [o.cpu().numpy() for o in b.run()]
    for (plan, x1, _, _), o in zip(items, outs):
        want = qfx.amplitudes(plan, x1).cpu().numpy()
        np.testing.assert_array_equal(o, want)
    qfx.sync()


def test_adjoint_two_word_bitstrings(qfx):
    c = ri.rqc(9, 8, 4, seed=2, parametrised=True)      # 72 qubits
    plan = qfx.Plan(qfx.Circuit(c), n_open=3)
    words = ri.random_bitstring_words(72, 1, seed=6)
    x1 = dev_words(words)
    amp = qfx.amplitudes(plan, x1)
    g = qfx.amplitudes_backward(plan, x1, 2 * amp).cpu().numpy()
    qfx.sync()
    rng = np.random.default_rng(5)
    pick = [(int(gi), int(e)) for gi, e in zip(rng.integers(0, len(c.gates), 24), rng.integers(0, 4, 24))]
    want = gradient.grad_entries(c, ri.words_to_int(words[0]), plan.open_sites, pick)
    got = np.array([g[gi, e] for gi, e in pick])
    assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)
