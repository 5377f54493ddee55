"""torch.autograd.Function over libqfx: amplitudes as a differentiable function of the
gate tensors.  The forward pass is qfx_amplitudes, the backward pass the library's
adjoint contraction (qfx_amplitudes_backward); both run in the library's kernels."""
from __future__ import annotations

import copy
from typing import Optional, Sequence

from . import qfx


def _circuit_with(template, gates_host):
    """The template with its gate matrices replaced by the rows of gates_host ([n, 4] or
    [n, 16]): 2x2 for a single-qubit gate, 4 diagonal entries for a diagonal two-qubit
    gate (its first 4 values), 4x4 for a general one (16 values, rows of width 16 only)."""
    c = copy.copy(template)
    c.gates = []
    for g, m in zip(template.gates, gates_host):
        g2 = copy.copy(g)
        if g.q1 < 0:
            g2.mat = m[:4].reshape(2, 2).copy()
        elif g.mat.size == 16:
            if m.size != 16:
                raise ValueError("a general (U4) gate needs gates rows of 16 entries")
            g2.mat = m.reshape(4, 4).copy()
        else:
            g2.mat = m[:4].reshape(4).copy()
        c.gates.append(g2)
    return c


def _make():
    import torch

    class CircuitAmplitudes(torch.autograd.Function):
        """amp = CircuitAmplitudes.apply(gates, template, x1, n_open, open_sites, cuts)

        gates: complex128 [n_gates, 4] (each gate's 2x2 matrix row-major, or the 4 diagonal
        entries of a diagonal two-qubit gate) or [n_gates, 16] (also a general gate's 4x4
        matrix row-major; other gates in their first 4 entries), in the template circuit's
        gate order.  The backward pass returns dL/dRe + i dL/dIm for every entry (PyTorch's
        convention), in the same shape."""

        @staticmethod
        def forward(ctx, gates, template, x1, n_open: int = 0, open_sites=None, cuts=()):
            circ = _circuit_with(template, gates.detach().cpu().numpy())
            plan = qfx.Plan(qfx.Circuit(circ), n_open=n_open, open_sites=open_sites, cuts=cuts)
            ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device=x1.device)
            amp = qfx.amplitudes(plan, x1, workspace=ws)
            ctx.plan = plan
            ctx.entries = int(gates.shape[1])
            ctx.gates_device = gates.device
            ctx.save_for_backward(x1)
            return amp

        @staticmethod
        def backward(ctx, grad_amp):
            (x1,) = ctx.saved_tensors
            g = qfx.amplitudes_backward(ctx.plan, x1, grad_amp, entries=ctx.entries)
            return g.to(ctx.gates_device), None, None, None, None, None

    return CircuitAmplitudes


CircuitAmplitudes = _make()


def circuit_amplitudes(gates, template, x1, *, n_open: int = 0,
                       open_sites: Optional[Sequence[int]] = None, cuts=()):
    return CircuitAmplitudes.apply(gates, template, x1, n_open,
                                   list(open_sites) if open_sites is not None else None, tuple(cuts))
