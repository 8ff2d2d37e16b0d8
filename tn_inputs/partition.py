"""Balanced graph partitioning for the Agglom tree builder (host side, numpy).

The SI's Agglom builder cuts the tensor graph into about N / K communities
with a hypergraph partitioner, under an imbalance bound, in a "direct"
(k-way) or "recursive" (repeated bisection) mode, minimising the cut or the
connectivity-minus-one objective.  In these networks every bond joins exactly
two tensors, so the hypergraph is a plain weighted graph and the two
objectives are the same number; this module is a plain partitioner for such
graphs:

* recursive mode: spectral bisection (the Fiedler vector of the weighted
  Laplacian, split at the size the part counts ask for; a disconnected graph
  is split along whole components first), refined by single moves and swaps
  of positive gain, applied recursively;
* direct mode: k regions grown at once from far-apart seeds, each taking the
  free node most strongly connected to it, then refined by moving nodes to
  the neighbouring part of largest gain.

Part sizes stay within (1 +- imbalance) of their targets (at least one node
of slack either way).  Edge weights are given by the caller (the Agglom
builder weights each bond by 1 or by log2 of its size).
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np


def _weights(nodes: Sequence[int], w: Dict[Tuple[int, int], float]) -> np.ndarray:
    pos = {v: i for i, v in enumerate(nodes)}
    W = np.zeros((len(nodes), len(nodes)))
    for (a, b), x in w.items():
        if a in pos and b in pos and a != b:
            W[pos[a], pos[b]] += x
            W[pos[b], pos[a]] += x
    return W


def _components(W: np.ndarray) -> List[List[int]]:
    n = W.shape[0]
    seen = np.zeros(n, bool)
    comps = []
    for s in range(n):
        if seen[s]:
            continue
        seen[s] = True
        comp, q = [s], [s]
        while q:
            u = q.pop()
            for v in np.nonzero(W[u] > 0)[0]:
                if not seen[v]:
                    seen[v] = True
                    comp.append(int(v))
                    q.append(int(v))
        comps.append(sorted(comp))
    return comps


def _spectral_order(W: np.ndarray) -> List[int]:
    """Nodes by component (largest first), each component by its Fiedler vector."""
    order: List[int] = []
    for comp in sorted(_components(W), key=lambda c: (-len(c), c[0])):
        if len(comp) <= 2:
            order.extend(comp)
            continue
        sub = W[np.ix_(comp, comp)]
        lap = np.diag(sub.sum(axis=1)) - sub
        _, vecs = np.linalg.eigh(lap)
        f = vecs[:, 1]
        if f[np.argmax(np.abs(f))] < 0:  # fix the eigenvector's sign for reproducibility
            f = -f
        order.extend(comp[i] for i in sorted(range(len(comp)), key=lambda i: (f[i], comp[i])))
    return order


def _bounds(target: float, imbalance: float) -> Tuple[int, int]:
    slack = max(1.0, imbalance * target)
    return int(math.ceil(target - slack)), int(math.floor(target + slack))


def _refine_two(W: np.ndarray, side: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Hill-climb the cut of a bisection: side[v] = +1 (part A) or -1 (B),
    |A| kept in [lo, hi].  The gain of moving v is the weight of its cut
    edges minus that of its uncut ones, -side[v] (W side)[v]; the best
    allowed move of positive gain is made, else the best positive swap among
    the 16 best nodes of each side; each step lowers the cut, so it ends."""
    s = side.astype(float).copy()
    ws = W @ s
    n = len(s)
    for _ in range(8 * n + 16):
        g = -s * ws
        na = int((s > 0).sum())
        allow = np.where(s > 0, na - 1 >= lo, na + 1 <= hi)
        cand = np.where(allow, g, -np.inf)
        v = int(np.argmax(cand))
        if cand[v] > 1e-12:
            ws -= 2.0 * s[v] * W[:, v]
            s[v] = -s[v]
            continue
        ia = np.nonzero(s > 0)[0]
        ib = np.nonzero(s < 0)[0]
        if len(ia) == 0 or len(ib) == 0:
            break
        ta = ia[np.argsort(-g[ia], kind="stable")[:16]]
        tb = ib[np.argsort(-g[ib], kind="stable")[:16]]
        sw = g[ta][:, None] + g[tb][None, :] - 2.0 * W[np.ix_(ta, tb)]
        a, b = np.unravel_index(int(np.argmax(sw)), sw.shape)
        if sw[a, b] <= 1e-12:
            break
        for u in (int(ta[a]), int(tb[b])):
            ws -= 2.0 * s[u] * W[:, u]
            s[u] = -s[u]
    return s


def _bisect(W: np.ndarray, frac: float, imbalance: float) -> np.ndarray:
    """Boolean mask of part A, |A| ~ frac * n, from the spectral order and refinement."""
    n = W.shape[0]
    ta = frac * n
    lo, hi = _bounds(ta, imbalance)
    lb, hb = _bounds(n - ta, imbalance)
    lo, hi = max(lo, n - hb, 1), min(hi, n - lb, n - 1)
    k = min(max(int(round(ta)), lo), hi)
    order = _spectral_order(W)
    side = -np.ones(n)
    side[order[:k]] = 1.0
    return _refine_two(W, side, lo, hi) > 0


def _recursive(W: np.ndarray, idx: List[int], p: int, imbalance: float, out: List[List[int]]) -> None:
    if p <= 1 or len(idx) <= 1:
        out.append(idx)
        return
    pa = p // 2
    mask = _bisect(W[np.ix_(idx, idx)], pa / p, imbalance)
    _recursive(W, [v for v, m in zip(idx, mask) if m], pa, imbalance, out)
    _recursive(W, [v for v, m in zip(idx, mask) if not m], p - pa, imbalance, out)


def _bfs(W: np.ndarray, src: List[int]) -> np.ndarray:
    n = W.shape[0]
    dist = np.full(n, np.inf)
    q = list(src)
    for s in src:
        dist[s] = 0
    h = 0
    while h < len(q):
        u = q[h]
        h += 1
        for v in np.nonzero(W[u] > 0)[0]:
            if dist[v] == np.inf:
                dist[v] = dist[u] + 1
                q.append(int(v))
    return dist


def _direct(W: np.ndarray, p: int, imbalance: float, rng: np.random.Generator) -> List[List[int]]:
    n = W.shape[0]
    lo, cap = _bounds(n / p, imbalance)
    lo = max(lo, 1)
    # seeds: a random node, then repeatedly the node farthest from the chosen ones
    seeds = [int(rng.integers(n))]
    while len(seeds) < p:
        d = _bfs(W, seeds)
        d[seeds] = -1.0
        seeds.append(int(np.argmax(np.where(np.isinf(d), 1e18, d))))
    part = np.full(n, -1)
    size = np.zeros(p, int)
    conn = np.zeros((n, p))  # weight from each node into each part
    for q, s in enumerate(seeds):
        part[s] = q
        size[q] = 1
        conn[:, q] += W[:, s]
    while (part < 0).any():
        free = part < 0
        grew = False
        for q in np.argsort(size, kind="stable"):
            if size[q] >= cap or not free.any():
                continue
            c = np.where(free, conn[:, q], -1.0)
            v = int(np.argmax(c))
            if c[v] <= 0:
                continue
            part[v] = q
            size[q] += 1
            conn[:, q] += W[:, v]
            free[v] = False
            grew = True
        if not grew:  # no free node touches a part with room: start it in the smallest part
            v = int(np.nonzero(part < 0)[0][0])
            q = int(np.argmin(size))
            part[v] = q
            size[q] += 1
            conn[:, q] += W[:, v]
    # k-way refinement: move a node to the part it is most strongly tied to
    for _ in range(8 * n + 16):
        own = conn[np.arange(n), part]
        gain = conn - own[:, None]
        gain[np.arange(n), part] = -np.inf
        gain[size[part] - 1 < lo, :] = -np.inf
        gain[:, size + 1 > cap] = -np.inf
        v, q = np.unravel_index(int(np.argmax(gain)), gain.shape)
        if gain[v, q] <= 1e-12:
            break
        a = part[v]
        conn[:, a] -= W[:, v]
        conn[:, q] += W[:, v]
        size[a] -= 1
        size[q] += 1
        part[v] = q
    return [sorted(int(v) for v in np.nonzero(part == q)[0]) for q in range(p) if size[q] > 0]


def partition(nodes: Sequence[int], w: Dict[Tuple[int, int], float], n_parts: int, imbalance: float = 0.1,
              mode: str = "recursive", seed: int = 0) -> List[List[int]]:
    """Split ``nodes`` into ``n_parts`` parts of near-equal size, few cut edges.

    w[(a, b)]: weight of the edge between nodes a and b (summed if given both
    ways).  Returns lists of node ids; every node is in exactly one part.  A
    recursive split can end with fewer parts than asked when a refinement
    move leaves one side with fewer nodes than parts; no part is empty.
    """
    nodes = list(nodes)
    n_parts = max(1, min(int(n_parts), len(nodes)))
    if n_parts == 1:
        return [sorted(nodes)]
    W = _weights(nodes, w)
    if mode == "recursive":
        out: List[List[int]] = []
        _recursive(W, list(range(len(nodes))), n_parts, imbalance, out)
    elif mode == "direct":
        out = _direct(W, n_parts, imbalance, np.random.default_rng(seed))
    else:
        raise ValueError(f"unknown partition mode {mode!r}")
    return [sorted(nodes[i] for i in part) for part in out if part]


def cut_weight(parts: Sequence[Sequence[int]], w: Dict[Tuple[int, int], float]) -> float:
    """Total weight of the edges whose ends lie in different parts."""
    where = {v: q for q, part in enumerate(parts) for v in part}
    return sum(x for (a, b), x in w.items() if where[a] != where[b])
