"""torch.autograd.Function around tn_grad: log|Z| as a differentiable function of the input tensors.

Argument marshalling only: the forward call runs the taped contraction and its
reverse pass in the CUDA library (tn_grad) and keeps d log|Z| / d T_v; the
backward call scales those by the incoming gradient.  Chain rules through how
the tensors were built (d/d beta, d/d J_ij of an Ising model, ...) are then
torch's ordinary autograd on the host side of the tensors.
"""
from __future__ import annotations

from typing import Sequence

import torch


class LogZ(torch.autograd.Function):
    """log|Z|(T_0, ..., T_{N-1}) of one loaded instance at bond dimension chi."""

    @staticmethod
    def forward(fctx, context, inst_id: int, chi: int, prec: str, *tensors):
        net_id = context._inst_net[inst_id]
        on_dev = tensors[0].is_cuda
        data = [t.detach().to(torch.float64).contiguous() for t in tensors]
        context.set_network_data(net_id, data, on_device=on_dev)
        total = sum(t.numel() for t in data)
        buf = torch.empty(total, dtype=torch.float64, device=data[0].device)
        logz, sign, _ = context.grad([inst_id], chi, prec, out=[buf])
        grads, off = [], 0
        for t in data:
            grads.append(buf[off:off + t.numel()].view(t.shape).to(tensors[0].dtype))
            off += t.numel()
        fctx.save_for_backward(*grads)
        fctx.sign = int(sign[0])
        return torch.tensor(float(logz[0]), dtype=torch.float64, device=data[0].device)

    @staticmethod
    def backward(fctx, gout):
        grads = fctx.saved_tensors
        return (None, None, None, None) + tuple(gout * g for g in grads)


def log_z(context, inst_id: int, tensors: Sequence[torch.Tensor], chi: int, prec: str = "f64") -> torch.Tensor:
    """Differentiable log|Z| of instance ``inst_id`` with its entries replaced by ``tensors``."""
    return LogZ.apply(context, inst_id, chi, prec, *tensors)
