"""CUDA path (through the C ABI) against the CPU FP64 oracle, element by element.

Tolerance (FP32 path): per amplitude |a - a_ref| <= 1e-5 * max(|a_ref|, 2^(-n/2)) and
normwise ||a - a_ref|| / ||a_ref|| <= 1e-5.  2^(-n/2) is the RMS amplitude (mean
|amp|^2 = 2^-n, Sec. III.E), the floor below which Porter-Thomas amplitudes near zero
make a per-amplitude relative error meaningless.
"""
import math

import numpy as np
import pytest

import rqc_inputs as ri
from oracle import network, primitives, stabilizer, statevector

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-5


def check_amps(got, want, n, rel=REL):
    got = np.asarray(got).reshape(-1)
    want = np.asarray(want).reshape(-1)
    floor = 2.0 ** (-n / 2)
    err = np.abs(got - want)
    bound = rel * np.maximum(np.abs(want), floor)
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"amp {worst}: got {got[worst]}, want {want[worst]}"
    nw = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
    assert nw <= rel, f"normwise error {nw}"
    return nw


def run(qfx, circ, x1s, *, open_sites=None, n_open=0, cuts=(), slices=None, ws_items=1,
        cap=0):
    plan = qfx.Plan(qfx.Circuit(circ), open_sites=open_sites, n_open=n_open, cuts=cuts,
                    max_intermediate_bytes=cap)
    x1 = torch.tensor(np.asarray(x1s, dtype=np.uint64).view(np.int64), device="cuda")
    ws = torch.empty(plan.workspace_bytes(ws_items), dtype=torch.uint8, device="cuda")
    sb, se = (0, plan.n_slices) if slices is None else slices
    out = qfx.amplitudes(plan, x1, slice_begin=sb, slice_end=se, workspace=ws)
    qfx.sync()
    return plan, out.cpu().numpy()


def expand(x1, open_sites, j):
    x = int(x1)
    for i, q in enumerate(open_sites):
        x = (x & ~(1 << q)) | (((j >> i) & 1) << q)
    return x


# --- config: 4x4, depth 1+16+1, all 2^16 amplitudes ---------------------------------

def test_4x4x16_all_amplitudes_open(qfx):
    c = ri.rqc(4, 4, 16, seed=0)
    psi = statevector.amplitudes(c)
    plan, out = run(qfx, c, [0], open_sites=list(range(16)))
    assert out.shape == (1, 1 << 16)
    check_amps(out[0], psi, 16)
    assert abs(np.sum(np.abs(out) ** 2) - 1.0) < 1e-6          # sum |amp|^2 = 1


def test_4x4x16_all_amplitudes_closed_batched(qfx):
    c = ri.rqc(4, 4, 16, seed=0)
    psi = statevector.amplitudes(c)
    xs = np.arange(1 << 16, dtype=np.uint64)
    plan, out = run(qfx, c, xs, ws_items=4096)
    check_amps(out[:, 0], psi, 16)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_4x4x16_fast_sampling_batches(qfx, seed):
    c = ri.rqc(4, 4, 16, seed=seed)
    psi = statevector.amplitudes(c)
    x1s = ri.random_bitstrings(16, 5, seed=seed)
    plan, out = run(qfx, c, x1s, n_open=5, ws_items=3)
    want = np.array([[psi[expand(x, plan.open_sites, j)] for j in range(32)] for x in x1s])
    check_amps(out, want, 16)


def test_4x4x16_open_sites_anywhere(qfx):
    c = ri.rqc(4, 4, 16, seed=4)
    psi = statevector.amplitudes(c)
    open_sites = [5, 0, 15, 10, 3]            # interior, first site, last site, mixed order
    x1s = ri.random_bitstrings(16, 3, seed=8)
    plan, out = run(qfx, c, x1s, open_sites=open_sites)
    want = np.array([[psi[expand(x, open_sites, j)] for j in range(32)] for x in x1s])
    check_amps(out, want, 16)


# --- shapes: non-square grids, lines, one site, shallow circuits ---------------------

@pytest.mark.parametrize("shape", [(3, 5, 16), (5, 3, 16), (2, 6, 24), (1, 7, 8), (6, 1, 8),
                                   (1, 1, 4), (2, 2, 3), (4, 5, 24), (3, 3, 40), (4, 4, 40)])
def test_shapes_vs_statevector(qfx, shape):
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=rows + cols + d)
    n = rows * cols
    psi = statevector.amplitudes(c)
    no = min(n, 6)
    x1s = ri.random_bitstrings(n, 4, seed=2)
    plan, out = run(qfx, c, x1s, n_open=no, ws_items=2)
    want = np.array([[psi[expand(x, plan.open_sites, j)] for j in range(1 << no)] for x in x1s])
    check_amps(out, want, n)


def test_identity_circuit_exact(qfx):
    c = ri.rqc(3, 4, 0)                        # H then H: amp = delta(x, 0)
    plan, out = run(qfx, c, [0, 5], n_open=12)  # all sites open: x1 is ignored
    want = np.zeros((2, 1 << 12))
    want[:, 0] = 1.0
    np.testing.assert_array_equal(out, want)
    plan, out = run(qfx, c, [0, 5, 16], n_open=3)
    want = np.zeros((3, 8))
    want[0, 0] = 1.0                           # x1 = 5 and 16 have closed bits set
    np.testing.assert_array_equal(out, want)


def test_ghz_exact(qfx):
    c = ri.ghz_snake(4, 4)
    plan, out = run(qfx, c, [0], open_sites=list(range(16)))
    want = np.zeros(1 << 16)
    want[0] = want[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(out[0], want, atol=1e-7)


# --- slicing (Sec. III.A) ------------------------------------------------------------

def test_slices_match_oracle_slice_by_slice(qfx):
    c = ri.rqc(4, 4, 16, seed=6)
    cuts = [(5, 6, 1), (9, 13, 2), (2, 3, 2)]
    x1 = int(ri.random_bitstrings(16, 1, seed=1)[0])
    plan = qfx.Plan(qfx.Circuit(c), n_open=4, cuts=cuts)
    assert plan.cuts == cuts
    ns = plan.n_slices
    assert ns == network.n_slices(c, cuts) == 4 * 2 * 2
    parts = []
    for s in range(ns):
        _, out = run(qfx, c, [x1], open_sites=plan.open_sites, cuts=cuts, slices=(s, s + 1))
        want = network.amplitudes_sliced(c, x1, plan.open_sites, cuts, [s])
        np.testing.assert_allclose(out[0], want, atol=1e-5 * 2 ** -8, rtol=1e-5)
        parts.append(out[0])
    full = network.amplitudes_open(c, x1, plan.open_sites)
    _, tot = run(qfx, c, [x1], open_sites=plan.open_sites, cuts=cuts, ws_items=5)
    check_amps(tot[0], full, 16)
    np.testing.assert_allclose(np.sum(parts, axis=0), tot[0], atol=1e-12)


def test_capped_plan_equals_uncapped(qfx):
    c = ri.rqc(5, 5, 24, seed=2)
    x1s = ri.random_bitstrings(25, 2, seed=3)
    p0, full = run(qfx, c, x1s, n_open=4)
    cap = p0.stats["max_elements"] * 8 // 8
    p1, capped = run(qfx, c, x1s, n_open=4, cap=cap, ws_items=7)
    assert p1.n_slices > 1 and p1.stats["max_elements"] * 8 <= cap
    want = np.array([network.amplitudes_open(c, int(x), p0.open_sites) for x in x1s])
    check_amps(full, want, 25)
    check_amps(capped, want, 25)


# --- paper-like shapes against the oracle's network contraction ---------------------

def test_5x5x24_vs_oracle(qfx):
    c = ri.rqc(5, 5, 24, seed=0)
    x1s = ri.random_bitstrings(25, 3, seed=7)
    plan, out = run(qfx, c, x1s, n_open=6, ws_items=3)
    want = np.array([network.amplitudes_open(c, int(x), plan.open_sites) for x in x1s])
    check_amps(out, want, 25)


def test_6x6x24_vs_oracle(qfx):
    c = ri.rqc(6, 6, 24, seed=1)
    x1 = int(ri.random_bitstrings(36, 1, seed=5)[0])
    plan, out = run(qfx, c, [x1], n_open=7)
    want = network.amplitudes_open(c, x1, plan.open_sites)
    check_amps(out[0], want, 36)


def test_7x7x24_vs_oracle(qfx):
    c = ri.rqc(7, 7, 24, seed=3)
    x1 = int(ri.random_bitstrings(49, 1, seed=6)[0])
    plan, out = run(qfx, c, [x1], n_open=6)
    want = network.amplitudes_open(c, x1, plan.open_sites)
    check_amps(out[0], want, 49)


# --- full size 7x7x(1+32+1), the measured workload: properties that hold at any size ----

def _full_plan(qfx, circ, cuts=()):
    return qfx.Plan(qfx.Circuit(circ), n_open=6, cuts=cuts)


def test_7x7x32_clifford_probabilities_exact(qfx):
    """T-free member of the family: |amp|^2 in {0, 2^-k}, exact value per bitstring from
    the stabilizer tableau; the GPU path runs the full 7x7x32 contraction unchanged."""
    c = ri.rqc(7, 7, 32, seed=11, gate_set=(ri.SQRT_X, ri.SQRT_Y))
    x1 = int(ri.random_bitstrings(49, 1, seed=12)[0])
    plan, out = run(qfx, c, [x1], n_open=6)
    tab = stabilizer.prepare(c)
    probs = np.array([stabilizer.probability(c, expand(x1, plan.open_sites, j), tab)
                      for j in range(64)])
    got = np.abs(out[0])
    floor = 2.0 ** (-49 / 2)
    assert np.all(np.abs(got - np.sqrt(probs)) <= REL * np.maximum(np.sqrt(probs), floor))


def test_7x7x32_slicing_invariance(qfx):
    """Sum over the slices of a sub-range cut equals the uncut contraction (Sec. III.A)."""
    c = ri.rqc(7, 7, 32, seed=0)
    x1 = int(ri.random_bitstrings(49, 1, seed=1)[0])
    _, full = run(qfx, c, [x1], n_open=6)
    _, sliced = run(qfx, c, [x1], n_open=6, cuts=[(24, 31, 8)])     # 2 slices
    nrm = np.linalg.norm(full)
    assert np.linalg.norm(sliced - full) / nrm <= REL
    floor = 2.0 ** (-49 / 2)
    assert np.all(np.abs(sliced - full) <= REL * np.maximum(np.abs(full), floor))


def test_7x7x32_one_full_bond_cut_16_slices(qfx):
    """The benchmarked circuit with one horizontal bond of the middle grid column,
    (3,3)-(3,4), cut to single values: 16 slices whose FP64 sum equals the uncut
    contraction (Sec. III.A), every slice the full-size FP32 path."""
    c = ri.rqc(7, 7, 32, seed=0)
    x1 = int(ri.random_bitstrings(49, 1, seed=1)[0])
    _, full = run(qfx, c, [x1], n_open=6)
    plan, sliced = run(qfx, c, [x1], n_open=6, cuts=[(24, 25, 1)])
    assert plan.n_slices == 16
    nrm = np.linalg.norm(full)
    assert np.linalg.norm(sliced - full) / nrm <= REL
    floor = 2.0 ** (-49 / 2)
    assert np.all(np.abs(sliced - full) <= REL * np.maximum(np.abs(full), floor))


# --- single operations: contraction step and permute --------------------------------

FILL = {0: 20, 1: 20, 2: 21, 3: 22, 4: 23, 5: 25, 6: 25, 7: 26, 8: 27, 9: 28}


@pytest.mark.parametrize("variant", list(range(10)) + [20, 21, 22, 23, 25, 26, 27, 28])
@pytest.mark.parametrize("shape", [(3, 37, 130, 130, 6), (2, 9, 70, 35, 34), (5, 16, 16, 16, 1),
                                   (1, 1, 3, 3, 10), (7, 130, 8, 4, 2), (1, 300, 33, 33, 1)])
def test_contract_step_variants(qfx, variant, shape):
    P, K, N, NL, Sd = shape
    if (variant < 5 or 20 <= variant < 25) and Sd % 2:
        pytest.skip("JMODE variants need even Sd")
    S = ri.random_complex((K, N), seed=1)
    B = ri.random_complex((P, K, Sd), seed=2)
    want = primitives.contract_step(S, B, P, K, N, Sd)            # [p][n][s]
    NH = N // NL
    want = want.reshape(P, NH, NL, Sd).transpose(1, 0, 2, 3)       # [nh][p][nl][s]
    dS = torch.from_numpy(S.reshape(-1)).cuda()
    dB = torch.from_numpy(B.reshape(-1)).cuda()
    out = qfx.contract_step(dS, dB, P, K, N, NL, Sd, variant=variant)
    qfx.sync()
    got = out.cpu().numpy().reshape(NH, P, NL, Sd)
    # element by element against each output's own scale sum_k |S||B|, and normwise
    scale = primitives.contract_step(np.abs(S), np.abs(B), P, K, N, Sd).real
    scale = scale.reshape(P, NH, NL, Sd).transpose(1, 0, 2, 3)
    assert np.all(np.abs(got - want) <= 1e-6 * scale)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-6, err


@pytest.mark.parametrize("shape", [(8, 64, 64, 64, 4096), (3, 37, 130, 130, 6), (4096, 64, 16, 8, 1),
                                   (2, 9, 70, 35, 34)])
def test_fill_variants_bit_identical(qfx, shape):
    # the fill tiles (4 x 4 outputs per thread) sum every output's k terms in the order of
    # the tiles they stand in for, so per-step launches may swap them in freely
    P, K, N, NL, Sd = shape
    S = torch.from_numpy(ri.random_complex(K * N, seed=4)).cuda()
    B = torch.from_numpy(ri.random_complex(P * K * Sd, seed=5)).cuda()
    for v, f in FILL.items():
        if v < 5 and Sd % 2:
            continue
        a = qfx.contract_step(S, B, P, K, N, NL, Sd, variant=v).cpu().numpy()
        b = qfx.contract_step(S, B, P, K, N, NL, Sd, variant=f).cpu().numpy()
        np.testing.assert_array_equal(a, b)
    auto = qfx.contract_step(S, B, P, K, N, NL, Sd).cpu().numpy()
    np.testing.assert_array_equal(auto, a)
    qfx.sync()


@pytest.mark.parametrize("case", [((4, 5, 6), (2, 0, 1)), ((33, 65), (1, 0)),
                                  ((2, 3, 4, 5, 6), (4, 2, 0, 3, 1)), ((7, 8, 9), (0, 2, 1)),
                                  ((64, 3, 64), (2, 1, 0)), ((5, 1, 7), (1, 2, 0)),
                                  ((2,) * 10, tuple(reversed(range(10)))), ((100,), (0,)),
                                  ((8, 8, 8), (0, 1, 2)), ((16,) * 5, (4, 3, 2, 1, 0)),
                                  ((64, 64, 16), (1, 0, 2)), ((3, 5, 7, 9), (2, 0, 3, 1)),
                                  ((5, 7, 3), (1, 0, 2)), ((33, 17, 40), (2, 1, 0)),
                                  ((16, 16, 16, 16, 16), (0, 1, 3, 2, 4)),
                                  # tensor-map path: two input runs, edge tiles, no batch
                                  # axis, a batch axis of 2
                                  ((6, 16, 5, 18, 32), (3, 0, 4, 2, 1)), ((48, 20, 100), (2, 1, 0)),
                                  ((130, 72), (1, 0)), ((16, 2, 16), (2, 1, 0)),
                                  # rows of 2, 3 and 4 elements (row offsets per thread run)
                                  ((7, 3, 2), (1, 0, 2)), ((5, 6, 3), (1, 0, 2)),
                                  ((9, 5, 4), (1, 0, 2)), ((33, 129, 2), (1, 0, 2)),
                                  # tiled transpose whose a side spans several output axes
                                  ((3, 40, 16, 2, 16), (0, 2, 4, 1, 3)),
                                  ((5, 2, 2, 2, 16), (4, 0, 3, 2, 1)),
                                  ((2, 24, 2, 2), (1, 3, 0, 2))])
def test_permute_vs_numpy(qfx, case):
    shape, perm = case
    x = ri.random_complex(int(np.prod(shape)), seed=3)
    want = primitives.permute(x, shape, perm).reshape(-1)
    out = qfx.permute(torch.from_numpy(x).cuda(), shape, perm)
    qfx.sync()
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_workspace_too_small_is_enomem(qfx):
    c = ri.rqc(3, 3, 8, seed=0)
    plan = qfx.Plan(qfx.Circuit(c), n_open=2)
    x1 = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(plan.workspace_bytes(1) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(qfx.QfxError) as e:
        qfx.amplitudes(plan, x1, workspace=ws)
    assert e.value.status == qfx.qfx.QFX_ENOMEM


def test_results_independent_of_concurrency(qfx):
    c = ri.rqc(4, 5, 16, seed=9)
    x1s = ri.random_bitstrings(20, 6, seed=2)
    cuts = [(6, 7, 2)]
    outs = [run(qfx, c, x1s, n_open=3, cuts=cuts, ws_items=w)[1] for w in (1, 4, 12)]
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])    # same order of FP64 adds -> same bits
