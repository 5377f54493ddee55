"""Host-side tests of libqfx through its C ABI: loading, exported symbols, circuit
validation, the planner's shapes and flop counts (Eq. 1), cut handling, argument checks.
No GPU work is launched here."""
import ctypes as C
import math

import numpy as np
import pytest

import rqc_inputs as ri
from oracle import primitives

qfx = pytest.importorskip("paper_1905_00444_gb300")
q = qfx.qfx


def test_library_exports_every_header_symbol():
    syms = q.header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(q.lib, s), f"libqfx.so does not export {s}"


def test_version_and_no_launches_on_host():
    assert "sm_103a" in qfx.version()
    ri_c = ri.rqc(3, 3, 8, seed=0)
    p = qfx.Plan(qfx.Circuit(ri_c), n_open=2)
    assert p.stats["n_steps"] == 9
    assert qfx.launch_count() == 0


@pytest.mark.parametrize("bad", [
    dict(q0=9), dict(q1=5, kind=ri.CZ),           # out of range / not neighbours (0-5 on 3x3)
    dict(layer=-1), dict(kind=ri.CZ),             # kind/arity mismatch (1q gate labelled CZ)
])
def test_circuit_validation_rejects(bad):
    c = ri.rqc(3, 3, 2, seed=0)
    g = c.gates[0]
    for k, v in bad.items():
        setattr(g, k, v)
    if g.q1 >= 0 and g.mat.size != 4:
        g.mat = ri.DIAG_CZ.copy()
    with pytest.raises(qfx.QfxError) as e:
        qfx.Circuit(c)
    assert e.value.status == q.QFX_EINVAL


def test_layer_disjointness_checked():
    c = ri.rqc(2, 2, 0)
    c.gates.append(ri.Gate(0, 0, -1, ri.H, ri.MAT_H.copy()))   # qubit 0 twice in layer 0
    with pytest.raises(qfx.QfxError):
        qfx.Circuit(c)


def test_text_format_roundtrip_plan_identical():
    c = ri.rqc(3, 4, 16, seed=5)
    a = qfx.Plan(qfx.Circuit(c), n_open=3)
    b = qfx.Plan(qfx.Circuit(text=ri.circuit_to_text(c)), n_open=3)
    assert a.stats == b.stats and a.steps == b.steps


def test_text_format_errors_name_the_line():
    with pytest.raises(qfx.QfxError, match="line 2"):
        qfx.Circuit(text="grid 2 2\n0 H 0 1 0\n")
    with pytest.raises(qfx.QfxError, match="unknown kind"):
        qfx.Circuit(text="grid 2 2\n0 FOO 0 1 0 0 0 0 0 0 0\n")


def test_general_two_qubit_gates_validated():
    c = ri.rqc(3, 3, 8, seed=0, two_qubit="fsim")
    g = next(g for g in c.gates if g.kind == ri.U4)
    g.q1 = -1                                        # U4 on one qubit
    with pytest.raises(qfx.QfxError, match="arity"):
        qfx.Circuit(c)
    c = ri.rqc(3, 3, 8, seed=0, two_qubit="fsim")
    g = next(g for g in c.gates if g.kind == ri.U4)
    g.mat = g.mat.copy()
    g.mat[3, 2] = np.nan
    with pytest.raises(qfx.QfxError, match="non-finite"):
        qfx.Circuit(c)
    with pytest.raises(qfx.QfxError, match="need 32 matrix values"):
        qfx.Circuit(text="grid 1 2\n0 U4 0 1 " + " ".join(["0"] * 8) + "\n")


def test_general_gate_text_roundtrip_and_bond_bits():
    c = ri.rqc(4, 4, 16, seed=2, two_qubit="fsim")
    a = qfx.Plan(qfx.Circuit(c), n_open=3)
    b = qfx.Plan(qfx.Circuit(text=ri.circuit_to_text(c)), n_open=3)
    assert a.stats == b.stats and a.steps == b.steps
    # every edge carries two fSim gates in 16 cycles: 2 x 2 bits, bond dimension 16, the
    # same shapes as the CZ circuit of depth 32
    cz = qfx.Plan(qfx.Circuit(ri.rqc(4, 4, 32, seed=2)), n_open=3)
    assert [(s["P"], s["K"], s["N"], s["Sd"]) for s in a.steps] == \
        [(s["P"], s["K"], s["N"], s["Sd"]) for s in cz.steps]
    # a half cut of a 4-bit bond: 2 slices
    h = qfx.Plan(qfx.Circuit(c), n_open=3, cuts=[(5, 6, 8)])
    assert h.n_slices == 2


def test_bond_bit_limit_counts_two_bits_per_general_gate():
    gates = [ri.Gate(l, 0, 1, ri.U4, ri.fsim(0.3, 0.2)) for l in range(21)]   # 42 bits
    with pytest.raises(qfx.QfxError, match="40 bond bits"):
        qfx.Plan(qfx.Circuit(ri.Circuit(1, 2, gates)), n_open=1)
    forty = qfx.Circuit(ri.Circuit(1, 2, gates[:20]))                        # 40 bits: fine,
    qfx.Plan(forty, n_open=1, cuts=[(0, 1, 1 << 20)])                          # once cut


def test_backward_rejects_general_gates_before_any_launch():
    p = qfx.Plan(qfx.Circuit(ri.rqc(2, 2, 8, seed=0, two_qubit="fsim")), n_open=1)
    fake = C.c_void_p(1 << 20)
    st = q.lib.qfx_amplitudes_backward(p._h, fake, 1, 0, 1, fake, fake, fake, 1 << 30, None)
    assert st == q.QFX_EUNSUPPORTED
    assert qfx.launch_count() == 0


@pytest.mark.parametrize("shape", [(4, 4, 16), (5, 5, 24), (6, 6, 24), (7, 7, 32), (8, 8, 32),
                                   (3, 5, 8), (5, 3, 8), (2, 7, 16), (1, 6, 8)])
def test_plan_steps_obey_eq1(shape):
    rows, cols, d = shape
    c = ri.rqc(rows, cols, d, seed=0)
    p = qfx.Plan(qfx.Circuit(c), n_open=min(4, rows * cols))
    total = 0.0
    for s in p.steps[1:]:
        P, K, N, Sd = s["P"], s["K"], s["N"], s["Sd"]
        v0, v1, v2 = P * K * Sd, K * N, P * N * Sd        # input boundary, site, output
        assert s["flops"] == pytest.approx(primitives.flops_eq1(v0, v1, v2), rel=1e-12)
        assert s["N"] % s["NL"] == 0
        total += s["flops"]
    assert p.stats["flops_per_item"] == pytest.approx(total, rel=1e-12)
    assert sorted(s["site"] for s in p.steps) == list(range(rows * cols))
    # sweep runs along the shorter dimension
    chi = 2 ** (d // 8)
    L = min(rows, cols)
    if rows > 1 and cols > 1 and d % 8 == 0:
        assert p.stats["max_elements"] <= chi ** (L + 1) * 2 ** 4


def test_plan_7x7x32_matches_hand_count():
    # chi = 16, lines of 7: 25 interior kink steps of 8*16^10 flops each dominate
    c = ri.rqc(7, 7, 32, seed=0)
    p = qfx.Plan(qfx.Circuit(c), n_open=6)
    assert p.stats["max_elements"] == 2 ** 32
    big = [s for s in p.steps if s["flops"] == 8 * 16 ** 10]
    assert len(big) == 25
    for s in big:
        assert (s["K"], s["N"], s["P"] * s["Sd"]) == (256, 256, 2 ** 24)
    assert p.stats["flops_per_item"] == pytest.approx(2.2558e14, rel=1e-3)
    assert p.open_sites == [13, 20, 27, 34, 41, 48]


def test_forced_cut_slices_and_cap():
    c = ri.rqc(4, 4, 16, seed=0)
    full = qfx.Plan(qfx.Circuit(c), n_open=2)
    cut = qfx.Plan(qfx.Circuit(c), n_open=2, cuts=[(5, 6, 1), (9, 13, 2)])
    assert cut.n_slices == 4 * 2
    assert cut.cuts == [(5, 6, 1), (9, 13, 2)]
    cap = full.stats["max_elements"] * 8 // 4
    capped = qfx.Plan(qfx.Circuit(c), n_open=2, max_intermediate_bytes=cap)
    assert capped.stats["max_elements"] * 8 <= cap
    assert capped.n_slices > 1


@pytest.mark.parametrize("shape", [(3, 4, 16), (5, 4, 16), (6, 6, 24)])
def test_adjoint_boundary_storage_threshold(shape):
    """The backward keeps all n step outputs when n x (one intermediate, 256-byte rounded)
    fits adjoint_store_bytes, else one per line plus one line's worth: the workspaces differ
    by exactly (n - lines - line_len) boundaries, lines + line_len = rows + cols."""
    rows, cols, d = shape
    c = qfx.Circuit(ri.rqc(rows, cols, d, seed=1))
    base = qfx.Plan(c, n_open=3)
    n = rows * cols
    B = -(-base.stats["max_elements"] * 8 // 256) * 256
    at = qfx.Plan(c, n_open=3, adjoint_store_bytes=n * B)
    below = qfx.Plan(c, n_open=3, adjoint_store_bytes=n * B - 1)
    assert base.backward_workspace_bytes() == at.backward_workspace_bytes()
    assert at.backward_workspace_bytes() - below.backward_workspace_bytes() == \
        (n - rows - cols) * B


@pytest.mark.parametrize("cuts", [[(0, 5, 1)], [(1, 2, 3)], [(1, 2, 8)], [(1, 2, 1), (2, 1, 1)]])
def test_bad_cuts_rejected(cuts):
    c = ri.rqc(4, 4, 16, seed=0)
    with pytest.raises(qfx.QfxError):
        qfx.Plan(qfx.Circuit(c), cuts=cuts)


def test_oversized_plans_refused_without_overflow():
    """Deep circuits make tensor sizes (products of bond dimensions up to 2^40) exceed
    int64; the planner saturates them and refuses plans above 2^50 elements, and bonds
    that keep more than 2^30 values after their cuts."""
    c = ri.rqc(8, 8, 128, seed=0)                   # bond 2^16 per edge: boundary 2^144
    with pytest.raises(qfx.QfxError, match="2\\^50") as e:
        qfx.Plan(qfx.Circuit(c), n_open=4)
    assert e.value.status == q.QFX_EPLAN
    with pytest.raises(qfx.QfxError) as e:
        qfx.Plan(qfx.Circuit(c), n_open=4, max_intermediate_bytes=1 << 30)
    assert e.value.status == q.QFX_EPLAN
    wide = ri.Circuit(1, 2, [ri.Gate(l, 0, 1, ri.CZ, ri.DIAG_CZ.copy()) for l in range(33)])
    with pytest.raises(qfx.QfxError, match="2\\^30"):
        qfx.Plan(qfx.Circuit(wide), n_open=1)
    p = qfx.Plan(qfx.Circuit(wide), n_open=1, cuts=[(0, 1, 1 << 20)])
    assert p.n_slices == 1 << 13 and p.stats["max_elements"] <= 2 << 20


def test_impossible_cap_is_eplan():
    c = ri.rqc(3, 3, 8, seed=0)
    with pytest.raises(qfx.QfxError) as e:
        qfx.Plan(qfx.Circuit(c), n_open=4, max_intermediate_bytes=8)
    assert e.value.status == q.QFX_EPLAN


def test_open_site_validation():
    c = ri.rqc(3, 3, 8, seed=0)
    with pytest.raises(qfx.QfxError):
        qfx.Plan(qfx.Circuit(c), open_sites=[1, 1])
    with pytest.raises(qfx.QfxError):
        qfx.Plan(qfx.Circuit(c), open_sites=[9])
    p = qfx.Plan(qfx.Circuit(c), open_sites=[4, 0, 8])
    assert p.open_sites == [4, 0, 8]


def test_amplitudes_argument_checks_before_any_launch():
    c = ri.rqc(2, 2, 8, seed=0)
    p = qfx.Plan(qfx.Circuit(c), n_open=1)
    f = q.lib.qfx_amplitudes
    assert f(p._h, None, 1, 0, 1, None, 0, None, None) == q.QFX_EINVAL
    fake = C.c_void_p(1 << 20)
    assert f(p._h, fake, 0, 0, 1, fake, 1 << 20, fake, None) == q.QFX_EINVAL      # n_batch
    assert f(p._h, fake, 1, 0, 2, fake, 1 << 20, fake, None) == q.QFX_EINVAL      # slices
    assert f(p._h, fake, 1, 0, 1, C.c_void_p((1 << 20) + 8), 1 << 20, fake, None) == q.QFX_EINVAL
    assert f(p._h, fake, 1, 0, 1, fake, 16, fake, None) == q.QFX_ENOMEM
    assert qfx.launch_count() == 0


def test_frugal_select_argument_checks_before_any_launch():
    c = ri.rqc(2, 2, 8, seed=0)
    p = qfx.Plan(qfx.Circuit(c), n_open=2)
    f = q.lib.qfx_frugal_select
    fake = C.c_void_p(1 << 20)
    assert f(p._h, None, 0, None, None, None, 10.0, None, None, None) == q.QFX_OK   # empty
    assert f(None, fake, 1, fake, fake, fake, 10.0, fake, None, None) == q.QFX_EINVAL
    assert f(p._h, fake, -1, fake, fake, fake, 10.0, fake, None, None) == q.QFX_EINVAL
    for M in (0.0, -1.0, math.inf, math.nan):
        assert f(p._h, fake, 1, fake, fake, fake, M, fake, None, None) == q.QFX_EINVAL
    assert f(p._h, fake, 1, None, fake, fake, 10.0, fake, None, None) == q.QFX_EINVAL
    assert f(p._h, fake, 1, fake, fake, fake, 10.0, None, None, None) == q.QFX_EINVAL
    assert f(p._h, fake, 1, C.c_void_p((1 << 20) + 8), fake, fake, 10.0, fake, None,
             None) == q.QFX_EINVAL                                                  # alignment
    assert qfx.launch_count() == 0


def test_permute_and_step_argument_checks():
    fake = C.c_void_p(1 << 20)
    sh = (C.c_int64 * 3)(2, 3, 4)
    bad = (C.c_int32 * 3)(0, 0, 1)
    assert q.lib.qfx_permute(fake, fake, 3, sh, bad, None) == q.QFX_EINVAL
    assert q.lib.qfx_contract_step(fake, fake, fake, 1, 1, 3, 2, 1, 0, -1, None, 0, None) == q.QFX_EINVAL
    assert q.lib.qfx_contract_step(fake, fake, fake, 1, 1, 2, 2, 3, 0, 0, None, 0, None) == q.QFX_EINVAL
    # tensor-core precision without scratch
    assert q.lib.qfx_contract_step(fake, fake, fake, 1, 256, 256, 256, 256, 1, -1, None, 0,
                                   None) == q.QFX_ENOMEM
    assert q.lib.qfx_step_scratch_bytes(256, 256, 1) == 16 * 9 * 256 * 32
    assert q.lib.qfx_step_scratch_bytes(256, 256, 2) == 32 * 6 * 256 * 32
    assert q.lib.qfx_step_scratch_bytes(256, 256, 0) == 0


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_tensor_core_plan_variants(prec):
    c = ri.rqc(7, 7, 32, seed=0)
    p = qfx.Plan(qfx.Circuit(c), n_open=6, precision=prec)
    tc = [s for s in p.steps if s["variant"] >= 10]
    big = [s for s in p.steps if s["flops"] == 8 * 16 ** 10]
    assert all(s["variant"] == (10 if prec == "bf16x3" else 11) for s in big)
    share = sum(s["flops"] for s in tc) / p.stats["flops_per_item"]
    assert share > 0.97
    # the site image region makes the tensor-core item larger than the FP32 one
    p32 = qfx.Plan(qfx.Circuit(c), n_open=6)
    assert p.stats["item_bytes"] > p32.stats["item_bytes"]


def test_autotune_cache_is_applied(tmp_path):
    c = ri.rqc(4, 4, 16, seed=0)
    base = qfx.Plan(qfx.Circuit(c), n_open=3)
    s = next(st for st in base.steps[1:] if st["Sd"] % 2 == 0 and st["N"] >= 16)
    other = 2 if s["variant"] != 2 else 1
    cache = tmp_path / "tune.json"
    cache.write_text('{"qfx_autotune": 1, "entries": [\n'
                     f'  {{"N": {s["N"]}, "K": {s["K"]}, "NL": {s["NL"]}, "Sd": {s["Sd"]}, '
                     f'"variant": {other}, "ms": 0.5}}\n]}}\n')
    tuned = qfx.Plan(qfx.Circuit(c), n_open=3, autotune_cache=str(cache))
    for a, b in zip(base.steps, tuned.steps):
        same = (a["N"], a["K"], a["NL"], a["Sd"]) == (s["N"], s["K"], s["NL"], s["Sd"])
        assert b["variant"] == (other if same else a["variant"])
    # a missing or unreadable cache leaves the defaults
    p2 = qfx.Plan(qfx.Circuit(c), n_open=3, autotune_cache=str(tmp_path / "missing.json"))
    assert [st["variant"] for st in p2.steps] == [st["variant"] for st in base.steps]


def test_autograd_circuit_rows_of_sixteen_entries():
    """The autograd wrapper rebuilds the template from [n, 16] rows: 2x2 from the first 4
    of a single-qubit gate, the diagonal from the first 4 of a CZ, the 4x4 of a U4 gate;
    rows of 4 cannot carry a U4 gate.  The rebuilt circuit plans like the template."""
    from paper_1905_00444_gb300.autograd import _circuit_with
    c = ri.rqc(3, 3, 8, seed=2, two_qubit="fsim")
    k = next(i for i, g in enumerate(c.gates) if g.kind == ri.U4)      # one CZ among the fSims
    c.gates[k] = ri.Gate(c.gates[k].layer, c.gates[k].q0, c.gates[k].q1, ri.CZ, ri.DIAG_CZ.copy())
    rows = np.zeros((len(c.gates), 16), dtype=np.complex128)
    for i, g in enumerate(c.gates):
        flat = np.asarray(g.mat).reshape(-1)
        rows[i, :flat.size] = flat
    c2 = _circuit_with(c, rows)
    for a, b in zip(c.gates, c2.gates):
        np.testing.assert_array_equal(np.asarray(a.mat).reshape(-1), np.asarray(b.mat).reshape(-1))
        assert np.asarray(a.mat).shape == np.asarray(b.mat).shape
    p1 = qfx.Plan(qfx.Circuit(c), n_open=2)
    p2 = qfx.Plan(qfx.Circuit(c2), n_open=2)
    assert p1.steps == p2.steps
    with pytest.raises(ValueError):
        _circuit_with(c, rows[:, :4])


def test_binding_refuses_host_and_short_tensors_before_any_launch():
    """Host pointers or undersized buffers would reach the kernels as wild addresses: the
    binding checks device, layout, dtype and size first (all on CPU here, so every call
    must refuse)."""
    torch = pytest.importorskip("torch")
    p = qfx.Plan(qfx.Circuit(ri.rqc(2, 2, 8, seed=0)), n_open=1)
    x1 = torch.zeros(2, dtype=torch.int64)
    with pytest.raises(ValueError, match="CUDA"):
        qfx.amplitudes(p, x1)
    with pytest.raises(ValueError, match="CUDA"):
        qfx.amplitudes_static(p, x1)
    with pytest.raises(ValueError, match="CUDA"):
        qfx.amplitudes_backward(p, x1, torch.zeros((2, 2), dtype=torch.complex128))
    with pytest.raises(ValueError, match="CUDA"):
        qfx.frugal_select(p, x1, torch.zeros((2, 2), dtype=torch.complex128),
                          torch.zeros((2, 2), dtype=torch.float64), torch.zeros(2, dtype=torch.int64))
    S = torch.zeros(16, dtype=torch.complex64)
    with pytest.raises(ValueError, match="CUDA"):
        qfx.contract_step(S, S, 1, 4, 4, 4, 1)
    with pytest.raises(ValueError, match="CUDA"):
        qfx.permute(S, (4, 4), (1, 0))
    assert qfx.launch_count() == 0


def test_planner_invariants_on_random_circuits():
    """Seeded random grids, depths, gate kinds, open sites, forced cuts and caps: every plan
    chains its steps (each step reads exactly what the previous one wrote), ends with the
    2^|x2| outputs, counts Eq. 1 per step, covers every site once, has as many slices as
    its cuts' radices multiply to (2^bits per bond, two bits per U4 gate) and meets its
    cap."""
    rng = np.random.default_rng(2024)
    for case in range(150):
        rows, cols = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        if rows * cols < 2:
            cols = 2
        depth = int(rng.choice([0, 4, 8, 12, 16]))
        kind = "fsim" if rng.random() < 0.4 else "cz"
        c = ri.rqc(rows, cols, depth, seed=case, two_qubit=kind)
        n = rows * cols
        n_open = int(rng.integers(0, min(6, n) + 1))
        bits = {}
        for g in c.gates:
            if g.q1 >= 0:
                e = (min(g.q0, g.q1), max(g.q0, g.q1))
                bits[e] = bits.get(e, 0) + (2 if g.kind == ri.U4 else 1)
        cuts = []
        for e in rng.permutation(sorted(bits))[:int(rng.integers(0, 3))]:
            m = bits[tuple(e)]
            cuts.append((int(e[0]), int(e[1]), 1 << int(rng.integers(0, m + 1))))
        base = qfx.Plan(qfx.Circuit(c), n_open=n_open, cuts=cuts)
        cap = 0
        if rng.random() < 0.3 and base.stats["max_elements"] > 64:
            # a quarter of the uncapped peak, but not below the 2^|x2| outputs, which no
            # cut can shrink
            cap = max(base.stats["max_elements"] * 8 // 4, 8 << n_open)
        p = qfx.Plan(qfx.Circuit(c), n_open=n_open, cuts=cuts, max_intermediate_bytes=cap)
        st = p.steps
        assert sorted(s["site"] for s in st) == list(range(n)), case
        assert (st[0]["P"], st[0]["K"], st[0]["Sd"], st[0]["flops"]) == (1, 1, 1, 0), case
        prev_out = st[0]["N"]
        total = 0.0
        for s in st[1:]:
            assert s["P"] * s["K"] * s["Sd"] == prev_out, case
            assert s["N"] % s["NL"] == 0 and s["N"] // s["NL"] in (1, 2), case
            assert s["flops"] == 8.0 * s["P"] * s["K"] * s["N"] * s["Sd"], case
            prev_out = s["P"] * s["N"] * s["Sd"]
            total += s["flops"]
        assert prev_out == 1 << n_open, case
        assert p.stats["flops_per_item"] == pytest.approx(total, rel=1e-12), case
        assert p.stats["max_elements"] == max(s["P"] * s["N"] * s["Sd"] for s in st[1:]), case
        assert p.cuts[:len(cuts)] == cuts, case
        want_slices = 1
        for (a, b, size) in p.cuts:
            want_slices *= (1 << bits[(min(a, b), max(a, b))]) // size
        assert p.n_slices == want_slices, case
        if cap:
            assert p.stats["max_elements"] * 8 <= cap, case


def test_more_than_64_qubits_use_word_bitstrings():
    """Grids up to 144 qubits; a bitstring spans ceil(n / 64) words (Table I's 11x11)."""
    for rows, cols, words in ((11, 11, 2), (12, 12, 3), (8, 8, 1), (13, 5, 2)):
        p = qfx.Plan(qfx.Circuit(ri.rqc(rows, cols, 8, seed=0)), n_open=4)
        assert p.x1_words == words == p.stats["x1_words"]
    with pytest.raises(qfx.QfxError) as e:
        qfx.Circuit(ri.rqc(13, 12, 2, seed=0))
    assert e.value.status == q.QFX_EINVAL and "144" in str(e.value)


def test_word_bitstring_helpers():
    a = ri.random_bitstrings(49, 4, seed=3)
    w = ri.random_bitstring_words(49, 4, seed=3)
    assert w.shape == (4, 1) and np.array_equal(a, w[:, 0])
    w = ri.random_bitstring_words(121, 5, seed=1)
    assert w.shape == (5, 2) and np.all(w[:, 1] < (1 << 57))
    for row in w:
        x = ri.words_to_int(row)
        assert x < 2 ** 121 and np.array_equal(ri.int_to_words(x, 121), row)


def test_tree_plans_steps_cap_and_slices():
    """Plan family 1: Eq. 1 per step, the cap met, an output order over the open sites, and
    far fewer slices than the line sweep for the paper's 7x7x(1+40+1) at 8 GiB."""
    c = qfx.Circuit(ri.rqc(7, 7, 40, seed=0))
    tree = qfx.Plan(c, n_open=6, max_intermediate_bytes=8 << 30, family="tree")
    line = qfx.Plan(c, n_open=6, max_intermediate_bytes=8 << 30)
    assert tree.stats["max_elements"] * 8 <= 8 << 30
    assert tree.n_slices <= 1 << 24 < (1 << 50) <= line.n_slices
    total = 0.0
    for s in tree.steps:
        assert s["flops"] == 8.0 * s["P"] * s["K"] * s["N"] * s["Sd"]
        total += s["flops"]
    assert total == tree.stats["flops_per_item"]
    assert tree.stats["n_steps"] == 48                # n - 1 pairwise contractions
    assert tree.open_sites == line.open_sites
    tc = qfx.Plan(c, n_open=6, max_intermediate_bytes=8 << 30, family="tree", precision="bf16x3")
    assert tc.cuts == tree.cuts and all(s["variant"] >= 10 for s in tc.steps if s["N"] >= 128 and not s["parts"])
    assert all(s["parts"] == 0 for s in line.steps)


def test_tree_plan_split_k_root():
    """Region plans at 8 GiB: the roots contract long K into 64 outputs; they run as
    side-by-side 1024-long chunks (FP32, whatever the plan's precision) whose partial
    products fit the item's scratch."""
    for rows, cols, depth in ((7, 7, 40), (8, 8, 32)):
        c = qfx.Circuit(ri.rqc(rows, cols, depth, seed=0))
        for prec in ("fp32", "bf16x3"):
            tree = qfx.Plan(c, n_open=6, max_intermediate_bytes=8 << 30, family="tree", precision=prec)
            root = tree.steps[-1]
            assert root["N"] * root["Sd"] == 64 and root["K"] >= 4096 and root["parts"] == root["K"] // 1024
            assert root["variant"] < 10
            parts = 0
            for s in tree.steps:
                if s["parts"]:
                    assert s["K"] == 1024 * s["parts"] and s["P"] * s["N"] * s["Sd"] <= 1 << 18
                    parts = max(parts, s["parts"] * s["P"] * s["N"] * s["Sd"])
            assert tree.workspace_bytes(1) >= parts * 8 + tree.stats["max_elements"] * 8


def test_tree_plan_forced_cuts_keep_the_slice_numbering():
    g = ri.rqc(7, 7, 32, seed=0)
    cuts = [(r * 7 + c, (r + 1) * 7 + c, 1) for c in (0, 6) for r in range(6)]
    tree = qfx.Plan(qfx.Circuit(g), n_open=6, cuts=cuts, family="tree")
    line = qfx.Plan(qfx.Circuit(g), n_open=6, cuts=cuts)
    assert tree.cuts == line.cuts == cuts and tree.n_slices == line.n_slices == 16 ** 12
    assert tree.stats["flops_per_item"] < line.stats["flops_per_item"] / 10


def test_batch_workspace_follows_the_persistent_and_lane_split():
    """Host only: qfx_batch_workspace_bytes reads only the plans and ranges.  Split-precision
    items whose steps all take FP32 tiles (bond dimension 4) size a persistent batch, like
    their FP32 twins (same tables and blocks); an item with tensor-core steps (5x5x24,
    K = N = 64) adds one graph lane per slot."""
    def ws(plans, slots):
        arr = (q.BatchItem * len(plans))(*[q.BatchItem(p._h.value, None, 1, 0, p.n_slices, None)
                                            for p in plans])
        return int(q.lib.qfx_batch_workspace_bytes(arr, len(plans), slots))

    small = [ri.rqc(4, 4, 16, seed=s) for s in (20, 22)]
    fp32 = [qfx.Plan(qfx.Circuit(c), n_open=3) for c in small]
    bf16 = [qfx.Plan(qfx.Circuit(c), n_open=3, precision="bf16x3") for c in small]
    assert all(st["variant"] < 10 for p in bf16 for st in p.steps)
    assert ws(bf16, 4) == ws(fp32, 4) > 0
    big = qfx.Plan(qfx.Circuit(ri.rqc(5, 5, 24, seed=1)), n_open=4, precision="bf16x3")
    assert any(st["variant"] >= 10 for st in big.steps)
    one, two = ws(bf16 + [big], 1), ws(bf16 + [big], 2)
    lane = two - one
    assert big.stats["item_bytes"] <= lane <= big.workspace_bytes(1)
    assert ws(bf16 + [big], 3) - two == lane


def test_tree_planner_invariants_on_random_circuits():
    """Plan family 1 on seeded random grids, depths, gate kinds, open sites, forced cuts and
    caps: n - 1 pairwise contractions, Eq. 1 per node, a root of 2^|x2| outputs, long
    contractions in 1024-long chunks (in place, P = 1) or split-K parts, the forced cuts
    first and in order (as given without a cap; a cap may narrow them further), as many
    slices as the cuts' radices multiply to, and the cap met."""
    rng = np.random.default_rng(77)
    for case in range(60):
        rows, cols = int(rng.integers(2, 6)), int(rng.integers(2, 6))
        depth = int(rng.choice([4, 8, 16, 24]))
        kind = "fsim" if rng.random() < 0.3 else "cz"
        c = ri.rqc(rows, cols, depth, seed=500 + case, two_qubit=kind)
        n = rows * cols
        n_open = int(rng.integers(0, min(6, n) + 1))
        bits = {}
        for g in c.gates:
            if g.q1 >= 0:
                e = (min(g.q0, g.q1), max(g.q0, g.q1))
                bits[e] = bits.get(e, 0) + (2 if g.kind == ri.U4 else 1)
        cuts = []
        for e in rng.permutation(sorted(bits))[:int(rng.integers(0, 3))]:
            m = bits[tuple(e)]
            cuts.append((int(e[0]), int(e[1]), 1 << int(rng.integers(0, m + 1))))
        base = qfx.Plan(qfx.Circuit(c), n_open=n_open, cuts=cuts, family="tree")
        cap = 0
        if rng.random() < 0.4 and base.stats["max_elements"] > 64:
            cap = max(base.stats["max_elements"] * 8 // 4, 8 << n_open)
        p = qfx.Plan(qfx.Circuit(c), n_open=n_open, cuts=cuts, max_intermediate_bytes=cap,
                     family="tree")
        st = p.steps
        assert p.stats["n_steps"] == len(st) == n - 1, case
        assert [s["site"] for s in st] == list(range(n, 2 * n - 1)), case   # node result ids
        total = 0.0
        for s in st:
            assert min(s["P"], s["K"], s["N"], s["Sd"]) >= 1, case
            assert s["flops"] == 8.0 * s["P"] * s["K"] * s["N"] * s["Sd"], case
            if s["parts"]:
                assert s["K"] == 1024 * s["parts"] and s["variant"] < 10, case
            elif s["K"] > 1024:
                assert s["P"] == 1 and s["K"] % 1024 == 0, case
            total += s["flops"]
        root = st[-1]
        assert root["P"] * root["N"] * root["Sd"] == 1 << n_open, case
        assert p.stats["flops_per_item"] == pytest.approx(total, rel=1e-12), case
        for (qa, qb, size), got in zip(cuts, p.cuts):
            assert got[:2] == (qa, qb) and got[2] <= size and size % got[2] == 0, case
        if not cap:
            assert p.cuts == cuts, case
        want_slices = 1
        for (a, b, size) in p.cuts:
            want_slices *= (1 << bits[(min(a, b), max(a, b))]) // size
        assert p.n_slices == want_slices, case
        if cap:
            assert p.stats["max_elements"] * 8 <= cap, case
