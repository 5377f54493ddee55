"""ctypes binding of libqfx (include/qfx.h).  Argument marshalling only: every step of
the contraction runs in the library's CUDA kernels; PyTorch supplies device memory and
streams.  If the library cannot be loaded this module raises on import -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Iterable, List, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqfx.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "qfx.h")

QFX_OK, QFX_EINVAL, QFX_ENOMEM, QFX_ECUDA, QFX_ETIMEOUT, QFX_EUNSUPPORTED, QFX_EPLAN = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "EUNSUPPORTED", "EPLAN"]
PRECISIONS = {"fp32": 0, "bf16x3": 1, "tf32x3": 2, "bf16x2": 3}


class QfxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"qfx {name}: {msg}")


class Gate(C.Structure):
    _fields_ = [("layer", C.c_int32), ("q0", C.c_int32), ("q1", C.c_int32), ("kind", C.c_int32),
                ("mat", C.c_double * 32)]


class Cut(C.Structure):
    _fields_ = [("qa", C.c_int32), ("qb", C.c_int32), ("size", C.c_int32)]


class PlanOpts(C.Structure):
    _fields_ = [("max_intermediate_bytes", C.c_uint64), ("open_sites", C.POINTER(C.c_int32)),
                ("n_open", C.c_int32), ("forced_cuts", C.POINTER(Cut)),
                ("n_forced_cuts", C.c_int32), ("precision", C.c_int32),
                ("plan_family", C.c_int32), ("tc_flags", C.c_int32),
                ("autotune_cache", C.c_char_p), ("adjoint_store_bytes", C.c_uint64)]


class PlanStats(C.Structure):
    _fields_ = [("n_slices", C.c_int64), ("n_steps", C.c_int32), ("n_open", C.c_int32),
                ("n_cuts", C.c_int32), ("n_sites", C.c_int32), ("flops_per_item", C.c_double),
                ("bytes_per_item", C.c_double), ("max_elements", C.c_int64),
                ("item_bytes", C.c_uint64), ("workspace_min", C.c_uint64),
                ("largest_step", C.c_int32), ("precision", C.c_int32), ("x1_words", C.c_int32)]


class StepInfo(C.Structure):
    _fields_ = [("site", C.c_int32), ("variant", C.c_int32), ("P", C.c_int64), ("K", C.c_int64),
                ("N", C.c_int64), ("NL", C.c_int64), ("Sd", C.c_int64), ("flops", C.c_double),
                ("bytes", C.c_double), ("parts", C.c_int32), ("reserved", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("x1", C.c_void_p), ("n_batch", C.c_int64),
                ("slice_begin", C.c_int64), ("slice_end", C.c_int64), ("out", C.c_void_p)]


class KernelTime(C.Structure):
    _fields_ = [("step", C.c_int32), ("variant", C.c_int32), ("kind", C.c_int32),
                ("ms", C.c_float), ("flops", C.c_double), ("bytes", C.c_double)]


def _declare(lib):
    vp, i32, i64, u64, st = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_int
    sig = {
        "qfx_circuit_create": (st, [i32, i32, C.POINTER(Gate), i64, C.POINTER(vp)]),
        "qfx_circuit_from_text": (st, [C.c_char_p, C.POINTER(vp)]),
        "qfx_circuit_destroy": (None, [vp]),
        "qfx_plan_create": (st, [vp, C.POINTER(PlanOpts), C.POINTER(vp)]),
        "qfx_plan_destroy": (None, [vp]),
        "qfx_plan_info": (st, [vp, C.POINTER(PlanStats)]),
        "qfx_workspace_bytes": (u64, [vp, i64]),
        "qfx_plan_step": (st, [vp, i32, C.POINTER(StepInfo)]),
        "qfx_plan_cut": (st, [vp, i32, C.POINTER(Cut)]),
        "qfx_plan_open_sites": (st, [vp, C.POINTER(i32)]),
        "qfx_plan_upload": (st, [vp]),
        "qfx_amplitudes": (st, [vp, vp, i64, i64, i64, vp, C.c_size_t, vp, vp]),
        "qfx_amplitudes_static": (st, [vp, vp, i64, i64, i64, vp, vp]),
        "qfx_amplitudes_backward": (st, [vp, vp, i64, i64, i64, vp, vp, vp, C.c_size_t, vp]),
        "qfx_amplitudes_backward_full": (st, [vp, vp, i64, i64, i64, vp, vp, vp, C.c_size_t, vp]),
        "qfx_backward_workspace_bytes": (u64, [vp]),
        "qfx_batch_workspace_bytes": (u64, [C.POINTER(BatchItem), i32, i64]),
        "qfx_batch_prepare": (st, [C.POINTER(BatchItem), i32, vp, C.c_size_t, C.POINTER(vp), vp]),
        "qfx_batch_run": (st, [vp, vp]),
        "qfx_batch_info": (st, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]),
        "qfx_batch_destroy": (None, [vp]),
        "qfx_sync": (st, [vp]),
        "qfx_contract_step": (st, [vp, vp, vp, i64, i64, i64, i64, i64, i32, i32, vp, C.c_size_t, vp]),
        "qfx_tensor_peak": (st, [i32, i64, C.POINTER(C.c_double), vp]),
        "qfx_step_scratch_bytes": (u64, [i64, i64, i32]),
        "qfx_permute": (st, [vp, vp, i32, C.POINTER(i64), C.POINTER(i32), vp]),
        "qfx_frugal_select": (st, [vp, vp, i64, vp, vp, vp, C.c_double, vp, vp, vp]),
        "qfx_profile_enable": (st, [i32]),
        "qfx_profile_collect": (st, [C.POINTER(KernelTime), i32, C.POINTER(i32)]),
        "qfx_autotune": (st, [vp, C.c_char_p, vp, C.c_size_t, vp]),
        "qfx_launch_count": (u64, []),
        "qfx_debug_permute_withhold": (st, [i64]),
        "qfx_debug_batch_stall": (st, [vp, i64]),
        "qfx_last_error": (C.c_char_p, []),
        "qfx_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libqfx.so is not built ({LIB_PATH}); run paper_1905_00444_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    _declare(lib)
    return lib


lib = _load()


def _check(status: int):
    if status != QFX_OK:
        raise QfxError(status, lib.qfx_last_error().decode(errors="replace"))


def header_symbols() -> List[str]:
    """Every function declared in include/qfx.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(qfx_[a-z0-9_]+)\s*\(", text)))


def version() -> str:
    return lib.qfx_version().decode()


def launch_count() -> int:
    return int(lib.qfx_launch_count())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Circuit:
    """Validated circuit owned by the library.  `src` has .rows, .cols and .gates, each
    gate with .layer, .q0, .q1, .kind and .mat (2x2 complex; 4 diagonal entries for CZ
    and U2; 4x4 complex for U4)."""

    def __init__(self, src=None, *, text: Optional[str] = None):
        h = C.c_void_p()
        if text is not None:
            _check(lib.qfx_circuit_from_text(text.encode(), C.byref(h)))
            self.rows = self.cols = None
            self.n_gates = sum(1 for ln in text.splitlines()
                               if ln.split("#")[0].strip() and not ln.strip().startswith("grid"))
        else:
            arr = (Gate * max(1, len(src.gates)))()
            for i, g in enumerate(src.gates):
                arr[i].layer, arr[i].q0, arr[i].q1, arr[i].kind = g.layer, g.q0, g.q1, g.kind
                flat = list(g.mat.reshape(-1))
                for j, v in enumerate(flat):
                    arr[i].mat[2 * j] = float(v.real)
                    arr[i].mat[2 * j + 1] = float(v.imag)
            _check(lib.qfx_circuit_create(src.rows, src.cols, arr, len(src.gates), C.byref(h)))
            self.rows, self.cols = src.rows, src.cols
            self.n_gates = len(src.gates)
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib.qfx_circuit_destroy(self._h)
            self._h = None


class Plan:
    """Contraction plan (order, x2 open sites, cuts, workspace layout)."""

    def __init__(self, circuit: Circuit, *, open_sites: Optional[Sequence[int]] = None,
                 n_open: int = 0, max_intermediate_bytes: int = 0,
                 cuts: Iterable = (), precision: str = "fp32", fast_accumulation: bool = False,
                 autotune_cache: Optional[str] = None, tensor_maps: bool = True,
                 adjoint_store_bytes: int = 0, family: str = "line"):
        opts = PlanOpts()
        opts.max_intermediate_bytes = int(max_intermediate_bytes)
        self._open_arr = None
        if open_sites is not None:
            self._open_arr = (C.c_int32 * max(1, len(open_sites)))(*open_sites)
            opts.open_sites = C.cast(self._open_arr, C.POINTER(C.c_int32))
            opts.n_open = len(open_sites)
        else:
            opts.n_open = n_open
        cuts = list(cuts)
        self._cut_arr = (Cut * max(1, len(cuts)))(*[Cut(a, b, s) for (a, b, s) in cuts])
        opts.forced_cuts = C.cast(self._cut_arr, C.POINTER(Cut))
        opts.n_forced_cuts = len(cuts)
        opts.precision = PRECISIONS[precision]
        opts.tc_flags = (1 if fast_accumulation else 0) | (0 if tensor_maps else 4)
        opts.autotune_cache = autotune_cache.encode() if autotune_cache else None
        opts.adjoint_store_bytes = int(adjoint_store_bytes)
        opts.plan_family = {"line": 0, "tree": 1}[family]
        h = C.c_void_p()
        _check(lib.qfx_plan_create(circuit._h, C.byref(opts), C.byref(h)))
        self._h = h
        self._circuit = circuit
        self.stats_n_gates = circuit.n_gates
        st = PlanStats()
        _check(lib.qfx_plan_info(h, C.byref(st)))
        self.stats = {f: getattr(st, f) for f, _ in PlanStats._fields_}
        self.steps = []
        for i in range(st.n_steps):
            si = StepInfo()
            _check(lib.qfx_plan_step(h, i, C.byref(si)))
            self.steps.append({f: getattr(si, f) for f, _ in StepInfo._fields_})
        self.cuts = []
        for i in range(st.n_cuts):
            c = Cut()
            _check(lib.qfx_plan_cut(h, i, C.byref(c)))
            self.cuts.append((c.qa, c.qb, c.size))
        arr = (C.c_int32 * max(1, st.n_open))()
        _check(lib.qfx_plan_open_sites(h, arr))
        self.open_sites = [arr[i] for i in range(st.n_open)]
        self.x1_words = st.x1_words

    def batch_of(self, x1) -> int:
        """Bitstrings in x1 (x1_words uint64 words each)."""
        n = x1.numel()
        if n % self.x1_words:
            raise ValueError(f"x1 holds {n} words; bitstrings of this plan have {self.x1_words} each")
        return n // self.x1_words

    @property
    def n_slices(self) -> int:
        return self.stats["n_slices"]

    def workspace_bytes(self, n_concurrent: int = 1) -> int:
        return int(lib.qfx_workspace_bytes(self._h, n_concurrent))

    def backward_workspace_bytes(self) -> int:
        """Workspace amplitudes_backward needs (all step outputs, or one per grid line)."""
        return int(lib.qfx_backward_workspace_bytes(self._h))

    def upload(self):
        _check(lib.qfx_plan_upload(self._h))

    def __del__(self):
        if getattr(self, "_h", None):
            lib.qfx_plan_destroy(self._h)
            self._h = None


def _need(t, name, *, dtype=None, size=None, numel=None, device=None):
    """Refuses what the library would read or write out of bounds: a host tensor, a
    non-contiguous one, another dtype or element size, fewer elements than the call uses,
    or another device than the call's."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
    if size is not None and t.element_size() != size:
        raise ValueError(f"{name} must have {size}-byte elements")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements; the call needs {numel}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}; the call runs on {device}")
    return t


def amplitudes(plan: Plan, x1, *, slice_begin: int = 0, slice_end: Optional[int] = None,
               workspace=None, out=None, stream=None):
    """Amplitudes [n_batch, 2^n_open] (torch complex128 on x1's device).

    x1: torch int64/uint64 CUDA tensor of bitstrings, plan.x1_words words each (one word
    up to 64 qubits).  workspace: torch uint8 CUDA tensor (default: room for one work item)."""
    import torch
    _need(x1, "x1", size=8)
    n_batch = plan.batch_of(x1)
    if slice_end is None:
        slice_end = plan.n_slices
    if workspace is None:
        workspace = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device=x1.device)
    _need(workspace, "workspace", dtype=torch.uint8, device=x1.device)
    if out is None:
        out = torch.empty((n_batch, 1 << len(plan.open_sites)), dtype=torch.complex128,
                          device=x1.device)
    _need(out, "out", dtype=torch.complex128, numel=n_batch << len(plan.open_sites),
          device=x1.device)
    _check(lib.qfx_amplitudes(plan._h, x1.data_ptr(), n_batch, slice_begin, slice_end,
                              workspace.data_ptr(), workspace.numel(), out.data_ptr(),
                              _stream_ptr(stream)))
    return out


def amplitudes_backward(plan: Plan, x1, grad_out, *, slice_begin: int = 0,
                        slice_end: Optional[int] = None, workspace=None, stream=None,
                        entries: int = 4):
    """Gradients [n_gates, entries] (complex128) of a real loss with respect to every gate's
    matrix entries, given grad_out = dL/dRe(amp) + i dL/dIm(amp) [n_batch, 2^n_open].
    entries = 4 (single-qubit and diagonal gates) or 16 (any gates, U4 included: entry
    4*r + c of a U4 gate is G[r][c]; other gates fill their first 4)."""
    import torch
    _need(x1, "x1", size=8)
    if slice_end is None:
        slice_end = plan.n_slices
    if workspace is None:
        workspace = torch.empty(plan.backward_workspace_bytes(), dtype=torch.uint8,
                                device=x1.device)
    _need(workspace, "workspace", dtype=torch.uint8, device=x1.device)
    if entries not in (4, 16):
        raise ValueError("entries must be 4 or 16")
    grad_out = grad_out.to(device=x1.device, dtype=torch.complex128).contiguous()
    n_batch = plan.batch_of(x1)
    _need(grad_out, "grad_out", numel=n_batch << len(plan.open_sites))
    out = torch.empty((plan.stats_n_gates, entries), dtype=torch.complex128, device=x1.device)
    f = lib.qfx_amplitudes_backward if entries == 4 else lib.qfx_amplitudes_backward_full
    _check(f(plan._h, x1.data_ptr(), n_batch, slice_begin, slice_end, grad_out.data_ptr(),
             out.data_ptr(), workspace.data_ptr(), workspace.numel(), _stream_ptr(stream)))
    return out


def frugal_select(plan: Plan, x1, amps, u, scan_mask, M: float = 10.0, *, stream=None):
    """Frugal rejection sampling over fast-sampling batches (Sec. III.B), one sample per x1.

    amps: complex128 [n_batch, 2^n_open] from amplitudes(plan, x1, ...); u: float64
    [n_batch, 2^n_open] uniforms in [0, 1); scan_mask: int64/uint64 [n_batch].  Returns
    (x2 int64 [n_batch], -1 where no candidate was accepted; bitstrings int64 [n_batch]
    (or [n_batch, x1_words] above 64 qubits), x1 with the open-site bits set from x2)."""
    import torch
    _need(x1, "x1", size=8)
    n_batch = plan.batch_of(x1)
    per = 1 << len(plan.open_sites)
    _need(amps, "amps", dtype=torch.complex128, numel=n_batch * per, device=x1.device)
    _need(u, "u", dtype=torch.float64, numel=n_batch * per, device=x1.device)
    _need(scan_mask, "scan_mask", size=8, numel=n_batch, device=x1.device)
    if tuple(amps.shape) != (n_batch, per) or tuple(u.shape) != (n_batch, per):
        raise ValueError("amps and u must be [n_batch, 2^n_open]")
    x2 = torch.empty(n_batch, dtype=torch.int64, device=x1.device)
    bits = torch.empty(n_batch if plan.x1_words == 1 else (n_batch, plan.x1_words),
                       dtype=torch.int64, device=x1.device)
    _check(lib.qfx_frugal_select(plan._h, x1.data_ptr(), n_batch, amps.data_ptr(), u.data_ptr(),
                                 scan_mask.data_ptr(), float(M), x2.data_ptr(), bits.data_ptr(),
                                 _stream_ptr(stream)))
    return x2, bits


def frugal_sample(plan: Plan, x1, u, scan_mask, M: float = 10.0, *, slice_begin: int = 0,
                  slice_end: Optional[int] = None, workspace=None, stream=None):
    """Fast sampling (Sec. III.B): the 2^n_open amplitudes of every x1 batch in one
    contraction call, then one frugal rejection pass per batch, all on the device.  A slice
    range covering a fraction f of the slices samples at fidelity about f (Sec. III.C); the
    caller then passes M * f.  Returns (x2, bitstrings, amps) as frugal_select does, plus
    the amplitudes."""
    amps = amplitudes(plan, x1, slice_begin=slice_begin, slice_end=slice_end,
                      workspace=workspace, stream=stream)
    x2, bits = frugal_select(plan, x1, amps, u, scan_mask, M, stream=stream)
    return x2, bits, amps


class Batch:
    """Many (plan, x1 batch, slice range) items in one CUDA graph: small items whose steps
    all take FP32 tiles in one persistent launch, items with tensor-core steps, large items
    and tree plans as per-item launch sequences over parallel lanes (`slots` of them).

    items: list of (plan, x1 tensor, slice_begin, slice_end); outputs are allocated here
    (complex128 [n_batch, 2^n_open] each) and refreshed by every run()."""

    def __init__(self, items, *, slots: int = 8, workspace=None, stream=None):
        import torch
        self._keep = []
        arr = (BatchItem * len(items))()
        self.outs = []
        for i, (plan, x1, sb, se) in enumerate(items):
            _need(x1, f"items[{i}] x1", size=8, device=items[0][1].device)
            out = torch.empty((plan.batch_of(x1), 1 << len(plan.open_sites)), dtype=torch.complex128,
                              device=x1.device)
            self.outs.append(out)
            self._keep += [plan, x1, out]
            arr[i] = BatchItem(plan._h.value, x1.data_ptr(), plan.batch_of(x1), sb,
                               plan.n_slices if se is None else se, out.data_ptr())
        self._arr = arr
        if workspace is None:
            nbytes = int(lib.qfx_batch_workspace_bytes(arr, len(items), slots))
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=items[0][1].device)
        _need(workspace, "workspace", dtype=torch.uint8, device=items[0][1].device)
        self.workspace = workspace
        h = C.c_void_p()
        _check(lib.qfx_batch_prepare(arr, len(items), workspace.data_ptr(), workspace.numel(),
                                     C.byref(h), _stream_ptr(stream)))
        self._h = h
        nw, nt, sl = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.qfx_batch_info(h, C.byref(nw), C.byref(nt), C.byref(sl)))
        self.n_work, self.n_tasks, self.slots = nw.value, nt.value, sl.value

    def run(self, stream=None):
        _check(lib.qfx_batch_run(self._h, _stream_ptr(stream)))
        return self.outs

    def debug_stall(self, wait_ns: int):
        """Test hook: makes one dependency unreachable and limits every wait to wait_ns,
        so the next run() gives up and sync() raises QFX_ETIMEOUT (the batch stays broken)."""
        _check(lib.qfx_debug_batch_stall(self._h, int(wait_ns)))

    def __del__(self):
        if getattr(self, "_h", None):
            lib.qfx_batch_destroy(self._h)
            self._h = None


def autotune(plan: Plan, cache_path: str, *, workspace=None, stream=None):
    """Times the FP32 tile variants of the plan's step shapes; writes/extends the cache."""
    import torch
    if workspace is None:
        workspace = torch.empty(min(plan.workspace_bytes(1), 4 << 30), dtype=torch.uint8,
                                device="cuda")
    _need(workspace, "workspace", dtype=torch.uint8)
    _check(lib.qfx_autotune(plan._h, cache_path.encode(), workspace.data_ptr(), workspace.numel(),
                            _stream_ptr(stream)))


STATIC_SCRATCH_BYTES = 64 << 20   # QFX_STATIC_SCRATCH_BYTES in include/qfx.h


def amplitudes_static(plan: Plan, x1, *, slice_begin: int = 0, slice_end: Optional[int] = None,
                      out=None, stream=None):
    """As amplitudes(), but the library's built-in 64 MiB scratch array replaces the
    caller's workspace (for callers that cannot allocate device memory; the output
    buffer is still the caller's).  Calls that overlap on the GPU race on that array."""
    import torch
    _need(x1, "x1", size=8)
    n_batch = plan.batch_of(x1)
    if slice_end is None:
        slice_end = plan.n_slices
    if out is None:
        out = torch.empty((n_batch, 1 << len(plan.open_sites)), dtype=torch.complex128,
                          device=x1.device)
    _need(out, "out", dtype=torch.complex128, numel=n_batch << len(plan.open_sites),
          device=x1.device)
    _check(lib.qfx_amplitudes_static(plan._h, x1.data_ptr(), n_batch, slice_begin, slice_end,
                                     out.data_ptr(), _stream_ptr(stream)))
    return out


def debug_permute_withhold(wait_ns: int):
    """Test hook: the calling thread's next tensor-map permute issues no copies and gives up
    after wait_ns; sync() then raises QFX_ETIMEOUT."""
    _check(lib.qfx_debug_permute_withhold(int(wait_ns)))


def sync(stream=None):
    _check(lib.qfx_sync(_stream_ptr(stream)))


def tensor_peak(precision: str, mmas_per_sm: int = 1 << 16, stream=None) -> float:
    """Measured dense tensor-core TFLOP/s of a split mode's operand kind (see qfx.h)."""
    out = C.c_double()
    _check(lib.qfx_tensor_peak(PRECISIONS[precision], mmas_per_sm, C.byref(out), _stream_ptr(stream)))
    return out.value


def step_scratch_bytes(K: int, N: int, precision: str = "fp32") -> int:
    return int(lib.qfx_step_scratch_bytes(K, N, PRECISIONS[precision]))


def contract_step(S, B, P, K, N, NL, Sd, *, out=None, variant: int = -1, precision="fp32",
                  scratch=None, stream=None):
    """C[nh][p][nl][s] = sum_k S[k][nh*NL+nl] B[p][k][s] on complex64 CUDA tensors."""
    import torch
    _need(S, "S", dtype=torch.complex64, numel=K * N)
    _need(B, "B", dtype=torch.complex64, numel=P * K * Sd, device=S.device)
    if out is None:
        out = torch.empty(P * N * Sd, dtype=torch.complex64, device=S.device)
    _need(out, "out", dtype=torch.complex64, numel=P * N * Sd, device=S.device)
    need = step_scratch_bytes(K, N, precision)
    if scratch is None and need:
        scratch = torch.empty(need, dtype=torch.uint8, device=S.device)
    if scratch is not None:
        _need(scratch, "scratch", dtype=torch.uint8, numel=need, device=S.device)
    sp, sb = (scratch.data_ptr(), scratch.numel()) if scratch is not None else (None, 0)
    _check(lib.qfx_contract_step(S.data_ptr(), B.data_ptr(), out.data_ptr(), P, K, N, NL, Sd,
                                 PRECISIONS[precision], variant, sp, sb, _stream_ptr(stream)))
    return out


def permute(x, shape: Sequence[int], perm: Sequence[int], *, out=None, stream=None):
    """out = x viewed with `shape`, axes reordered by `perm` (complex64 CUDA tensors)."""
    import torch
    n = 1
    for d in shape:
        n *= int(d)
    _need(x, "x", dtype=torch.complex64, numel=n)
    if out is None:
        out = torch.empty(x.numel(), dtype=torch.complex64, device=x.device)
    _need(out, "out", dtype=torch.complex64, numel=n, device=x.device)
    r = len(shape)
    sh = (C.c_int64 * r)(*shape)
    pm = (C.c_int32 * r)(*perm)
    _check(lib.qfx_permute(x.data_ptr(), out.data_ptr(), r, sh, pm, _stream_ptr(stream)))
    return out


def profile_enable(on: bool = True):
    _check(lib.qfx_profile_enable(1 if on else 0))


def profile_collect(max_records: int = 1 << 16):
    arr = (KernelTime * max_records)()
    n = C.c_int32()
    _check(lib.qfx_profile_collect(arr, max_records, C.byref(n)))
    return [{f: getattr(arr[i], f) for f, _ in KernelTime._fields_}
            for i in range(min(n.value, max_records))]
