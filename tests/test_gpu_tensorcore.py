"""Tensor-core (tcgen05) contraction steps in the split precisions, against the oracle.

Bounds: BF16x3 (x = h + m + l, six cross products) and TF32x3 (x = b + s, three cross
products) both split with error at or below 2^-21 per product, but the tensor core's FP32
accumulation loses a little at every MMA added into an accumulator.  The default tile
keeps the hi x hi products in their own accumulators (two additions per k-step), which
meets the FP32 path's 1e-5 amplitude bar in BF16x3 (measured 4.4e-6 at 7x7x(1+32+1)).
TF32x3 is limited by its two-term split (about 2^-21 per product): stated bound 3e-5
(measured 1.4e-5 at 7x7x(1+32+1)).  Fast accumulation (one accumulator pair, all
term products in it; measured 3.4e-6 per K = 256 step and 5e-5 at 7x7x(1+32+1)) has a
stated amplitude bound of 1e-4.  BF16x2 (x = h + m, products hm, mh, hh) drops terms near
2^-16 relative (measured 4.5e-6 per step, 3e-5 to 5e-5 per amplitude up to 7x7x(1+32+1)):
stated bounds 2e-5 per step and 2e-4 per amplitude.
"""
import numpy as np
import pytest

import rqc_inputs as ri
from oracle import network, primitives, stabilizer

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOUND = {"bf16x3": 1e-5, "tf32x3": 3e-5, "bf16x2": 2e-4}
FAST_BOUND = 1e-4
STEP_BOUND = {"bf16x3": 1e-6, "tf32x3": 3e-6, "bf16x2": 2e-5}
FAST_STEP_BOUND = 1e-5


def step_ref(S, B, P, K, N, NL, Sd):
    want = primitives.contract_step(S, B, P, K, N, Sd)
    return want.reshape(P, N // NL, NL, Sd).transpose(1, 0, 2, 3)


def check_step(got, want, S, B, P, K, N, NL, Sd, bound):
    """Element by element: |got - want| <= bound * sum_k |S[k][n]| |B[p][k][s]| for every
    output (the element's own scale, so outputs near zero are judged fairly), and the
    normwise error below bound."""
    scale = step_ref(np.abs(S), np.abs(B), P, K, N, NL, Sd).real
    err = np.abs(got - want)
    worst = float(np.max(err / scale))
    assert worst <= bound, ("element", worst)
    nw = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    assert nw <= bound, ("normwise", nw)
    return worst, nw


@pytest.mark.parametrize("fast", [False, True])
@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16x2"])
@pytest.mark.parametrize("shape", [(1, 256, 256, 256, 1024), (16, 256, 256, 256, 16),
                                   (3, 64, 64, 32, 64), (2000, 16, 16, 16, 1),
                                   (1, 32, 48, 48, 300), (5, 256, 32, 16, 40),
                                   (2, 48, 112, 112, 200), (1, 16, 240, 48, 136),
                                   (77, 32, 32, 32, 2), (3, 48, 64, 64, 128),
                                   (2, 32, 512, 512, 128), (1, 16, 1024, 256, 256), (40, 32, 768, 384, 4)])
def test_step_vs_oracle(qfx, prec, shape, fast):
    P, K, N, NL, Sd = shape
    S = ri.random_complex((K, N), seed=3)
    B = ri.random_complex((P, K, Sd), seed=4)
    want = step_ref(S, B, P, K, N, NL, Sd)
    out = qfx.contract_step(torch.from_numpy(S.reshape(-1)).cuda(),
                            torch.from_numpy(B.reshape(-1)).cuda(), P, K, N, NL, Sd,
                            precision=prec, variant=12 if fast else -1)
    qfx.sync()
    got = out.cpu().numpy().reshape(want.shape)
    worst, nw = check_step(got, want, S, B, P, K, N, NL, Sd,
                           max(FAST_STEP_BOUND if fast else 0.0, STEP_BOUND[prec]))
    print(f"step {prec} fast={fast} {shape}: element {worst:.2e}, normwise {nw:.2e}")


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16x2"])
def test_step_matches_fp32_path(qfx, prec):
    P, K, N, NL, Sd = 4, 256, 256, 256, 512
    S = torch.from_numpy(ri.random_complex((K * N,), seed=5)).cuda()
    B = torch.from_numpy(ri.random_complex((P * K * Sd,), seed=6)).cuda()
    a = qfx.contract_step(S, B, P, K, N, NL, Sd, precision=prec)
    b = qfx.contract_step(S, B, P, K, N, NL, Sd)
    qfx.sync()
    Sh, Bh = S.cpu().numpy().reshape(K, N), B.cpu().numpy().reshape(P, K, Sd)
    check_step(a.cpu().numpy().reshape(N // NL, P, NL, Sd), b.cpu().numpy().reshape(N // NL, P, NL, Sd),
               Sh, Bh, P, K, N, NL, Sd, STEP_BOUND[prec])


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16x2"])
@pytest.mark.parametrize("shape", [(1, 64, 64, 64, 4096), (8, 64, 64, 64, 512), (64, 64, 64, 64, 64),
                                   (512, 64, 64, 64, 8), (4, 64, 16, 8, 512), (16, 64, 16, 8, 8),
                                   (77, 32, 32, 32, 2), (3, 48, 64, 64, 128), (9, 32, 256, 64, 16),
                                   (4096, 64, 64, 64, 8)])
def test_tensor_map_rows_match_register_rows(qfx, prec, shape):
    """The default tile stages the FP32 rows of B by tensor-map copies (variant -1) or by
    per-thread loads (variant 13): the same values reach the same MMAs, so the results
    agree bit for bit, including ragged p tails the copies fill with zeros.  Repeated:
    CTAs that run several tiles reuse each staging buffer many times, and a missing
    proxy fence between the producers' reads and the next copy showed up only in some
    launches."""
    P, K, N, NL, Sd = shape
    S = torch.from_numpy(ri.random_complex((K * N,), seed=11)).cuda()
    B = torch.from_numpy(ri.random_complex((P * K * Sd,), seed=12)).cuda()
    b = qfx.contract_step(S, B, P, K, N, NL, Sd, precision=prec, variant=13)
    for _ in range(6):
        a = qfx.contract_step(S, B, P, K, N, NL, Sd, precision=prec)
        qfx.sync()
        assert torch.equal(a, b)


@pytest.mark.parametrize("shape", [(1, 8, 64, 64, 4096), (2, 8, 16, 8, 4096), (512, 8, 64, 64, 1),
                                   (40, 8, 32, 32, 4)])
def test_tf32_single_kstage_steps(qfx, shape):
    """K = 8 is one TF32 k-stage per tile (each tile's only stage is also its last)."""
    P, K, N, NL, Sd = shape
    S = ri.random_complex((K, N), seed=13)
    B = ri.random_complex((P, K, Sd), seed=14)
    want = step_ref(S, B, P, K, N, NL, Sd)
    for v in (-1, 13):
        out = qfx.contract_step(torch.from_numpy(S.reshape(-1)).cuda(),
                                torch.from_numpy(B.reshape(-1)).cuda(), P, K, N, NL, Sd,
                                precision="tf32x3", variant=v)
        qfx.sync()
        got = out.cpu().numpy().reshape(want.shape)
        check_step(got, want, S, B, P, K, N, NL, Sd, STEP_BOUND["tf32x3"])


def run(qfx, circ, x1s, prec, n_open, ws_items=1, fast=False):
    plan = qfx.Plan(qfx.Circuit(circ), n_open=n_open, precision=prec, fast_accumulation=fast)
    x1 = torch.tensor(np.asarray(x1s, dtype=np.uint64).view(np.int64), device="cuda")
    ws = torch.empty(plan.workspace_bytes(ws_items), dtype=torch.uint8, device="cuda")
    out = qfx.amplitudes(plan, x1, workspace=ws)
    qfx.sync()
    return plan, out.cpu().numpy()


def errors(got, want, n):
    got, want = got.reshape(-1), want.reshape(-1)
    floor = 2.0 ** (-n / 2)
    per = np.max(np.abs(got - want) / np.maximum(np.abs(want), floor))
    nw = np.linalg.norm(got - want) / np.linalg.norm(want)
    return per, nw


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16x2"])
@pytest.mark.parametrize("shape", [(5, 5, 24), (6, 6, 24), (7, 7, 24)])
def test_amplitudes_vs_oracle(qfx, prec, shape):
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=rows)
    n = rows * cols
    x1 = int(ri.random_bitstrings(n, 1, seed=9)[0])
    plan, out = run(qfx, c, [x1], prec, 6)
    assert any(s["variant"] >= 10 for s in plan.steps)
    want = network.amplitudes_open(c, x1, plan.open_sites)
    per, nw = errors(out[0], want, n)
    print(f"{prec} {shape}: per-amplitude {per:.2e}, normwise {nw:.2e}")
    assert per <= BOUND[prec] and nw <= BOUND[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16x2"])
def test_7x7x32_clifford_exact(qfx, prec):
    c = ri.rqc(7, 7, 32, seed=11, gate_set=(ri.SQRT_X, ri.SQRT_Y))
    x1 = int(ri.random_bitstrings(49, 1, seed=12)[0])
    plan, out = run(qfx, c, [x1], prec, 6)
    tab = stabilizer.prepare(c)
    probs = []
    for j in range(64):
        x = x1
        for i, q in enumerate(plan.open_sites):
            x = (x & ~(1 << q)) | (((j >> i) & 1) << q)
        probs.append(stabilizer.probability(c, x, tab))
    amp = np.sqrt(np.array(probs))
    floor = 2.0 ** (-49 / 2)
    assert np.all(np.abs(np.abs(out[0]) - amp) <= BOUND[prec] * np.maximum(amp, floor))


def test_7x7x32_split_modes_agree_with_fp32(qfx):
    c = ri.rqc(7, 7, 32, seed=0)
    x1 = int(ri.random_bitstrings(49, 1, seed=1)[0])
    _, ref = run(qfx, c, [x1], "fp32", 6)
    floor = 2.0 ** (-49 / 2)
    for prec, fast in (("bf16x3", False), ("tf32x3", False), ("bf16x2", False), ("bf16x3", True)):
        _, out = run(qfx, c, [x1], prec, 6, fast=fast)
        per = np.max(np.abs(out - ref) / np.maximum(np.abs(ref), floor))
        print(f"7x7x32 {prec} fast={fast} vs fp32: {per:.2e}")
        assert per <= (FAST_BOUND if fast else BOUND[prec])


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16x2"])
def test_batched_items_and_slices(qfx, prec):
    # several (slice, x1) items per launch, uneven shapes, through the tensor-core path
    c = ri.rqc(6, 6, 24, seed=2)
    x1s = ri.random_bitstrings(36, 3, seed=4)
    cuts = [(14, 15, 4)]
    plan = qfx.Plan(qfx.Circuit(c), n_open=5, cuts=cuts, precision=prec)
    x1 = torch.tensor(x1s.view(np.int64), device="cuda")
    ws = torch.empty(plan.workspace_bytes(4), dtype=torch.uint8, device="cuda")
    out = qfx.amplitudes(plan, x1, workspace=ws)
    qfx.sync()
    for b, x in enumerate(x1s):
        want = network.amplitudes_open(c, int(x), plan.open_sites)
        per, nw = errors(out[b].cpu().numpy(), want, 36)
        assert per <= BOUND[prec] and nw <= BOUND[prec], (per, nw)


def test_bounded_wait_expires_and_context_survives(qfx):
    """Variant 99 withholds the S stream: the kernel's waits run out after about 1 s,
    it records the timeout and returns; the host sees QFX_ETIMEOUT and the GPU keeps
    working."""
    P, K, N, NL, Sd = 1, 64, 64, 64, 128          # a single CTA
    S = torch.from_numpy(ri.random_complex((K * N,), seed=1)).cuda()
    B = torch.from_numpy(ri.random_complex((P * K * Sd,), seed=2)).cuda()
    qfx.contract_step(S, B, P, K, N, NL, Sd, precision="bf16x3", variant=99)
    with pytest.raises(qfx.QfxError) as e:
        qfx.sync()
    assert e.value.status == qfx.qfx.QFX_ETIMEOUT
    out = qfx.contract_step(S, B, P, K, N, NL, Sd, precision="bf16x3")
    qfx.sync()                                     # status was cleared; normal run is fine
    Sh, Bh = S.cpu().numpy().reshape(K, N), B.cpu().numpy().reshape(P, K, Sd)
    want = step_ref(Sh, Bh, P, K, N, NL, Sd)
    got = out.cpu().numpy().reshape(want.shape)
    check_step(got, want, Sh, Bh, P, K, N, NL, Sd, STEP_BOUND["bf16x3"])


def test_tensor_peak_probe(qfx):
    """The tensor-core peak probe: BF16 and TF32 figures below the pipe's ceiling (152 SMs x
    8192 dense BF16 flop per clock at <= 2.07 GHz = 2.58 PFLOP/s; TF32 half of that), and
    TF32 about half of BF16 per flop (the nominal ratio)."""
    bf = qfx.tensor_peak("bf16x3", 1 << 14)
    tf = qfx.tensor_peak("tf32x3", 1 << 14)
    qfx.sync()
    print(f"probe: bf16 {bf:.0f} TFLOP/s, tf32 {tf:.0f} TFLOP/s")
    assert 500 < bf < 2700 and 250 < tf < 1350
    assert 0.35 < tf / bf < 0.65
    with pytest.raises(qfx.QfxError):
        qfx.tensor_peak("fp32")
