"""Independent exact references used to pin the oracle (test infrastructure).

None of these go through the tree executor in ``approx``:

* ``ising_bruteforce``: Z = sum over all 2^n spin states of
  prod_<ij> exp(beta J_ij s_i s_j) (SI Eq. "ising-partition-fn"), with
  <E> and <s_i s_j> for derivative pins.
* ``ising_transfer_2d``: the same Z on an open lx x ly square lattice by
  row-to-row transfer matrices (2^lx states per row).
* closed forms: open chains / trees Z = 2 prod_e 2 cosh(beta J_e); ring
  Z = (2 cosh b)^n + (2 sinh b)^n.
* ``perfect_matchings``: dimer-cover count W (SI "Dimer covers") by
  recursion on the lowest uncovered vertex.
* ``einsum_contract``: Eq. 1 evaluated by numpy.einsum over the whole
  network (tiny networks only).
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

from tn_inputs.formats import Network


def _logsumexp(x: np.ndarray) -> float:
    m = float(np.max(x))
    return m + math.log(float(np.sum(np.exp(x - m))))


def _spin_states(n: int, lo: int, hi: int) -> np.ndarray:
    """Rows = states lo..hi-1; spin +1 <-> bit 0 (index 0), -1 <-> bit 1."""
    idx = np.arange(lo, hi, dtype=np.int64)[:, None]
    bits = (idx >> np.arange(n, dtype=np.int64)[None, :]) & 1
    return 1.0 - 2.0 * bits


def ising_bruteforce(n: int, edges: Sequence[Tuple[int, int]], beta: float,
                     J: "float | Sequence[float]" = 1.0) -> Dict[str, object]:
    """ln Z, dlnZ/dbeta = <sum J s s>, and dlnZ/dJ_e = beta <s_u s_v> by enumeration."""
    if n > 26:
        raise ValueError("too many spins for enumeration")
    Js = np.full(len(edges), float(J)) if np.isscalar(J) else np.asarray(J, dtype=np.float64)
    eu = np.array([u for u, _ in edges])
    ev = np.array([v for _, v in edges])
    chunk = 1 << min(n, 18)
    logw_all = []
    ss_all = []
    for lo in range(0, 1 << n, chunk):
        s = _spin_states(n, lo, min(1 << n, lo + chunk))
        ss = s[:, eu] * s[:, ev]              # (states, edges)
        logw_all.append(beta * ss @ Js)
        ss_all.append(ss)
    logw = np.concatenate(logw_all)
    ss = np.concatenate(ss_all)
    lnz = _logsumexp(logw)
    p = np.exp(logw - lnz)
    corr = p @ ss                              # <s_u s_v> per edge
    return {"lnZ": lnz, "dlnZ_dbeta": float(corr @ Js), "dlnZ_dJ": beta * corr}


def ising_transfer_2d(lx: int, ly: int, beta: float, J: float = 1.0) -> Dict[str, float]:
    """ln Z of the open lx x ly square-lattice Ising model by row transfer matrices.

    Also d lnZ / d beta by forward differentiation of the same recursion
    (each factor exp(beta h) contributes h to the derivative).
    """
    s = _spin_states(lx, 0, 1 << lx)                   # (2^lx, lx)
    h_row = (s[:, :-1] * s[:, 1:]).sum(1) * J          # horizontal energy-like term in a row
    h_vert = (s @ s.T) * J                             # vertical term between consecutive rows
    w_row = np.exp(beta * h_row)
    tm = np.exp(beta * h_vert)
    v = w_row.copy()
    dv = h_row * w_row                                 # d v / d beta
    lognorm = 0.0
    for _ in range(1, ly):
        nv = (v @ tm) * w_row
        ndv = ((dv @ tm) + (v @ (tm * h_vert))) * w_row + (v @ tm) * w_row * h_row
        c = float(np.max(np.abs(nv)))
        v, dv = nv / c, ndv / c
        lognorm += math.log(c)
    z = float(v.sum())
    return {"lnZ": math.log(z) + lognorm, "dlnZ_dbeta": float(dv.sum()) / z}


def ising_tree_closed_form(edges: Sequence[Tuple[int, int]], beta: float,
                           J: "float | Sequence[float]" = 1.0) -> float:
    """ln Z on a tree graph: 2 prod_e 2 cosh(beta J_e)."""
    Js = np.full(len(edges), float(J)) if np.isscalar(J) else np.asarray(J, dtype=np.float64)
    return math.log(2.0) + float(np.sum(np.log(2.0 * np.cosh(beta * Js))))


def ising_ring_closed_form(n: int, beta: float) -> float:
    """ln Z of the uniform ring of n spins: (2 cosh b)^n + (2 sinh b)^n."""
    a = n * math.log(2 * math.cosh(beta))
    if beta == 0:
        return a
    r = (math.tanh(beta)) ** n
    return a + math.log1p(r)


def perfect_matchings(n: int, edges: Sequence[Tuple[int, int]]) -> int:
    """Number of perfect matchings (dimer covers), by recursion on the lowest free vertex."""
    adj: List[List[int]] = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    memo: Dict[int, int] = {}

    def rec(mask: int) -> int:
        if mask == (1 << n) - 1:
            return 1
        if mask in memo:
            return memo[mask]
        v = 0
        while mask >> v & 1:
            v += 1
        tot = 0
        for u in adj[v]:
            if not mask >> u & 1:
                tot += rec(mask | (1 << v) | (1 << u))
        memo[mask] = tot
        return tot

    return rec(0)


def einsum_contract(net: Network) -> float:
    """Eq. 1 for a closed network, evaluated by numpy.einsum over all tensors."""
    args = []
    for bl, d in zip(net.bonds, net.data):
        args.append(d)
        args.append(list(bl))
    args.append([])
    return float(np.einsum(*args, optimize="greedy"))
