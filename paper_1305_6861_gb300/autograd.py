"""torch.autograd.Function over the adjoint kernels: the signal as a differentiable function of
every spin's M0, T1, T2 and of learnable RF flip angles.

The forward and backward passes both run in libmrsim (float64); torch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import mrsim as M


class _Signal(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, t1, t2, rf, adj, geom):
        x, y, z, dw = geom
        stream = torch.cuda.current_stream()
        ph = M.Phantom(adj.ctx, [x, y, z, rho.detach().contiguous(), t1.detach().contiguous(),
                                 t2.detach().contiguous(), dw], stream=stream)
        rf_d = rf.detach().contiguous()
        sig = torch.zeros(2 * adj.n_adc, dtype=torch.float64, device=rho.device)
        adj.forward(ph, rf_d if adj.n_params else None, sig, stream)
        adj._last = ph
        ctx.adj, ctx.ph, ctx.rf = adj, ph, rf_d
        return sig.view(adj.n_adc, 2)

    @staticmethod
    def backward(ctx, grad):
        adj, ph, rf = ctx.adj, ctx.ph, ctx.rf
        stream = torch.cuda.current_stream()
        dev = grad.device
        if getattr(adj, "_last", None) is not ph:  # checkpoints belong to another forward call: redo
            scratch = torch.zeros(2 * adj.n_adc, dtype=torch.float64, device=dev)
            adj.forward(ph, rf if adj.n_params else None, scratch, stream)
            adj._last = ph
        g = grad.contiguous().to(torch.float64).view(-1)
        n = ph.n
        d_rho = torch.zeros(n, dtype=torch.float64, device=dev)
        d_t1 = torch.zeros(n, dtype=torch.float64, device=dev)
        d_t2 = torch.zeros(n, dtype=torch.float64, device=dev)
        d_rf = torch.zeros(max(adj.n_params, 1), dtype=torch.float64, device=dev)
        adj.backward(ph, g, rf if adj.n_params else None, d_rho, d_t1, d_t2, d_rf if adj.n_params else None, stream)
        return d_rho, d_t1, d_t2, d_rf[: adj.n_params], None, None


def signal(adj: M.Adjoint, x, y, z, dw, rho, t1, t2, rf):
    """Complex signal as a (n_adc, 2) float64 tensor [Re, Im], differentiable in rho, t1, t2 (per
    spin) and rf (the adjoint's learnable flip angles).  All tensors float64 on the same GPU."""
    return _Signal.apply(rho, t1, t2, rf, adj, (x, y, z, dw))
