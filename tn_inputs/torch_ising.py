"""Ising site tensors as torch functions of beta and the couplings (for autograd chain rules).

Same construction as tn_inputs.networks.ising_network (bond factors W with
W_L W_R^T = [[e^{bJ}, e^{-bJ}], [e^{-bJ}, e^{bJ}]] and a copy tensor per site
with one factor per leg), written in torch ops so that d/d beta and d/d J_ij
follow from the tensors' gradients.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import torch

from .formats import edges_to_bonds


def bond_factors(beta: torch.Tensor, J: torch.Tensor, symmetric: bool) -> Tuple[torch.Tensor, torch.Tensor]:
    c = torch.cosh(beta * J)
    s = torch.sinh(beta * J)
    if symmetric:
        a, b = torch.sqrt(c), torch.sqrt(s)
        w = torch.stack([torch.stack([a + b, a - b]), torch.stack([a - b, a + b])]) / math.sqrt(2.0)
        return w, w
    h = torch.tensor([[1.0, 1.0], [1.0, -1.0]], dtype=beta.dtype) / math.sqrt(2.0)
    sc = torch.sqrt(2 * c)
    ss = torch.sqrt(2 * torch.abs(s))
    wl = h @ torch.diag(torch.stack([sc, ss]))
    wr = h @ torch.diag(torch.stack([sc, torch.sign(s) * ss]))
    return wl, wr


def ising_tensors(n: int, edges: Sequence[Tuple[int, int]], beta: torch.Tensor, J: torch.Tensor,
                  symmetric: bool) -> List[torch.Tensor]:
    """Site tensors T_v[a_1..a_d] = sum_s prod_e F_e[s, a_e], in edges_to_bonds order."""
    bonds = edges_to_bonds(n, edges)
    per_edge = [bond_factors(beta, J[e], symmetric) for e in range(len(edges))]
    out = []
    for v in range(n):
        total = None
        for s in range(2):
            term = torch.ones((), dtype=beta.dtype)
            for e in bonds[v]:
                u, w = edges[e]
                f = per_edge[e][0] if v == min(u, w) else per_edge[e][1]
                term = torch.tensordot(term, f[s], dims=0)
            total = term if total is None else total + term
        out.append(total)
    return out
