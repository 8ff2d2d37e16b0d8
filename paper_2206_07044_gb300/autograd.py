"""torch.autograd.Function around tn_grad: log|Z| as a differentiable function of the input tensors.

Argument marshalling only: the forward call runs the taped contraction and its
reverse pass in the CUDA library (tn_grad) and keeps d log|Z| / d T_v; the
backward call scales those by the incoming gradient.  Chain rules through how
the tensors were built (d/d beta, d/d J_ij of an Ising model, ...) are then
torch's ordinary autograd on the host side of the tensors.

``log_z`` differentiates one instance; ``log_z_batch`` differentiates many
instances (e.g. every beta of a sweep) with one tn_grad call, so instances
that share a network structure and tree run as one batch on the GPU.
"""
from __future__ import annotations

from typing import Sequence

import torch


def _run_grad(context, inst_ids, chi, prec, tensor_lists):
    """Load every instance's entries, run one tn_grad call; returns (log|Z| [n], signs, per-instance grads)."""
    bufs, datas = [], []
    for inst_id, tensors in zip(inst_ids, tensor_lists):
        net_id = context._inst_net[inst_id]
        on_dev = tensors[0].is_cuda
        data = [t.detach().to(torch.float64).contiguous() for t in tensors]
        context.set_network_data(net_id, data, on_device=on_dev)
        datas.append(data)
        bufs.append(torch.empty(sum(t.numel() for t in data), dtype=torch.float64, device=data[0].device))
    logz, sign, _ = context.grad(list(inst_ids), chi, prec, out=bufs)
    grads = []
    for data, buf, tensors in zip(datas, bufs, tensor_lists):
        gl, off = [], 0
        for t in data:
            gl.append(buf[off:off + t.numel()].view(t.shape).to(tensors[0].dtype))
            off += t.numel()
        grads.append(gl)
    return logz, sign, grads


class LogZ(torch.autograd.Function):
    """log|Z|(T_0, ..., T_{N-1}) of one loaded instance at bond dimension chi."""

    @staticmethod
    def forward(fctx, context, inst_id: int, chi: int, prec: str, *tensors):
        logz, sign, grads = _run_grad(context, [inst_id], chi, prec, [tensors])
        fctx.save_for_backward(*grads[0])
        fctx.sign = int(sign[0])
        return torch.tensor(float(logz[0]), dtype=torch.float64, device=tensors[0].device)

    @staticmethod
    def backward(fctx, gout):
        grads = fctx.saved_tensors
        return (None, None, None, None) + tuple(gout * g for g in grads)


class LogZBatch(torch.autograd.Function):
    """log|Z| of n loaded instances (a vector of n values) from one tn_grad call.

    The flat argument list holds the tensors of instance 0, then those of
    instance 1, ...; ``counts[i]`` is the number of tensors of instance i.
    """

    @staticmethod
    def forward(fctx, context, inst_ids, counts, chi: int, prec: str, *flat):
        lists, off = [], 0
        for c in counts:
            lists.append(flat[off:off + c])
            off += c
        logz, sign, grads = _run_grad(context, inst_ids, chi, prec, lists)
        fctx.save_for_backward(*[g for gl in grads for g in gl])
        fctx.counts = list(counts)
        fctx.signs = [int(s) for s in sign]
        return torch.tensor(logz, dtype=torch.float64, device=flat[0].device)

    @staticmethod
    def backward(fctx, gout):
        saved = fctx.saved_tensors
        out, off = [], 0
        for i, c in enumerate(fctx.counts):
            out.extend(gout[i] * g for g in saved[off:off + c])
            off += c
        return (None, None, None, None, None) + tuple(out)


def log_z(context, inst_id: int, tensors: Sequence[torch.Tensor], chi: int, prec: str = "f64") -> torch.Tensor:
    """Differentiable log|Z| of instance ``inst_id`` with its entries replaced by ``tensors``."""
    return LogZ.apply(context, inst_id, chi, prec, *tensors)


def log_z_batch(context, inst_ids: Sequence[int], tensor_lists: Sequence[Sequence[torch.Tensor]], chi: int,
                prec: str = "f64") -> torch.Tensor:
    """Differentiable log|Z| of every instance in ``inst_ids`` (a length-n vector), one tn_grad call.

    ``tensor_lists[i]`` replaces the entries of instance ``inst_ids[i]``; the
    instances must belong to different loaded networks.
    """
    ids = [int(i) for i in inst_ids]
    nets = [context._inst_net[i] for i in ids]
    if len(set(nets)) != len(nets):
        raise ValueError("log_z_batch: every instance needs its own loaded network")
    counts = [len(t) for t in tensor_lists]
    flat = [t for tl in tensor_lists for t in tl]
    return LogZBatch.apply(context, ids, counts, chi, prec, *flat)
