"""torch.autograd.Function over libqfx: amplitudes as a differentiable function of the
gate tensors.  The forward pass is qfx_amplitudes, the backward pass the library's
adjoint contraction (qfx_amplitudes_backward); both run in the library's kernels."""
from __future__ import annotations

import copy
from typing import Optional, Sequence

from . import qfx


def _circuit_with(template, gates_host):
    c = copy.copy(template)
    c.gates = []
    for g, m in zip(template.gates, gates_host):
        g2 = copy.copy(g)
        g2.mat = m.reshape(2, 2).copy() if g.q1 < 0 else m.reshape(4).copy()
        c.gates.append(g2)
    return c


def _make():
    import torch

    class CircuitAmplitudes(torch.autograd.Function):
        """amp = CircuitAmplitudes.apply(gates, template, x1, n_open, open_sites, cuts)

        gates: complex128 [n_gates, 4] (each gate's 2x2 matrix row-major, or the 4 diagonal
        entries of a two-qubit gate), in the template circuit's gate order.  The backward
        pass returns dL/dRe + i dL/dIm for every entry (PyTorch's convention)."""

        @staticmethod
        def forward(ctx, gates, template, x1, n_open: int = 0, open_sites=None, cuts=()):
            circ = _circuit_with(template, gates.detach().cpu().numpy())
            plan = qfx.Plan(qfx.Circuit(circ), n_open=n_open, open_sites=open_sites, cuts=cuts)
            ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device=x1.device)
            amp = qfx.amplitudes(plan, x1, workspace=ws)
            ctx.plan = plan
            ctx.gates_device = gates.device
            ctx.save_for_backward(x1)
            return amp

        @staticmethod
        def backward(ctx, grad_amp):
            (x1,) = ctx.saved_tensors
            g = qfx.amplitudes_backward(ctx.plan, x1, grad_amp)
            return g.to(ctx.gates_device), None, None, None, None, None

    return CircuitAmplitudes


CircuitAmplitudes = _make()


def circuit_amplitudes(gates, template, x1, *, n_open: int = 0,
                       open_sites: Optional[Sequence[int]] = None, cuts=()):
    return CircuitAmplitudes.apply(gates, template, x1, n_open,
                                   list(open_sites) if open_sites is not None else None, tuple(cuts))
