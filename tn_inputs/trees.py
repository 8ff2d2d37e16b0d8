"""Ordered approximate contraction tree generators (host side, plain Python).

A tree is independent of the tensor entries, so one tree serves a whole beta
sweep or every seed of a random ensemble.  Generators:

* ``boundary_rows``: the hand-coded boundary contraction of a 2D lattice
  (rows absorbed from the bottom, then the bonds between neighbouring
  boundary tensors compressed left to right after each row).
* ``from_pairs``: any sequence of pairwise contractions, with explicit
  compressions inserted either after each contraction ("early") or before it
  ("late"), following the two policies of Algorithm 1.
* ``greedy``: the Greedy builder of the SI (local score from the sizes before
  and after compression, input sizes, sub-graph sizes, centrality and a
  Gumbel noise term), simulated with chi_greedy.
* ``span``: the Span builder (a spanning tree grown by Algorithm 2,
  contracted leaves inwards).
* ``hyper_search``: random search over any builder's parameters scored by
  the cost tracer (Algorithm 3).

The shape simulation here only decides an order; it never touches tensor
entries.  A compression of the bonds shared by A and B yields one bond of
size min(chi, D_A, D_B) when the shared size D_AB exceeds chi.
"""
from __future__ import annotations

import heapq
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .formats import Network, Tree

# ---------------------------------------------------------------------------
# fixed orders


def boundary_rows(lx: int, ly: int) -> Tree:
    """Row-by-row boundary order for ``networks.square_lattice(lx, ly)`` ids.

    Row 0 is the initial boundary.  For each next row, site (x, y) is
    contracted into boundary tensor x for x = 0..lx-1, then S ops compress
    the bonds between boundary tensors (0,1), (1,2), ... left to right.
    Finally the boundary is contracted left to right into one scalar.
    """
    n = lx * ly
    nxt = n
    ops: List[tuple] = []
    b = list(range(lx))
    for y in range(1, ly):
        for x in range(lx):
            ops.append(("C", b[x], y * lx + x, nxt))
            b[x] = nxt
            nxt += 1
        if lx > 1:
            for x in range(lx - 1):
                ops.append(("S", b[x], b[x + 1]))
    acc = b[0]
    for x in range(1, lx):
        ops.append(("C", acc, b[x], nxt))
        acc = nxt
        nxt += 1
    return Tree(n, ops)


def boundary_layers(lx: int, ly: int, lz: int) -> Tree:
    """Layer-by-layer boundary order for ``networks.cubic_lattice(lx, ly, lz)`` ids
    (the 3D counterpart of boundary_rows: a boundary PEPS swept along z).

    Layer 0 is the initial boundary.  For each next layer, site (x, y, z) is
    contracted into boundary tensor (x, y) in row-major order, and right after
    each absorption the bonds to the already-updated neighbours (x-1, y) and
    (x, y-1) are compressed.  Finally the boundary PEPS itself is contracted
    by boundary_rows' order (row y absorbed into the row MPS, then its bonds
    compressed left to right) and the last MPS left to right.
    """
    n = lx * ly * lz
    nxt = n
    ops: List[tuple] = []
    b = list(range(lx * ly))
    for z in range(1, lz):
        for y in range(ly):
            for x in range(lx):
                q = y * lx + x
                ops.append(("C", b[q], (z * ly + y) * lx + x, nxt))
                b[q] = nxt
                nxt += 1
                if x > 0:
                    ops.append(("S", b[q - 1], b[q]))
                if y > 0:
                    ops.append(("S", b[q - lx], b[q]))
    m = [b[x] for x in range(lx)]
    for y in range(1, ly):
        for x in range(lx):
            ops.append(("C", m[x], b[y * lx + x], nxt))
            m[x] = nxt
            nxt += 1
        for x in range(lx - 1):
            ops.append(("S", m[x], m[x + 1]))
    acc = m[0]
    for x in range(1, lx):
        ops.append(("C", acc, m[x], nxt))
        acc = nxt
        nxt += 1
    return Tree(n, ops)


def _neighbours(bonds: Dict[int, List[int]], bond_owner: Dict[int, List[int]], t: int) -> List[int]:
    out = set()
    for b in bonds[t]:
        for o in bond_owner[b]:
            if o != t:
                out.add(o)
    return sorted(out)


def from_pairs(net_bonds: Sequence[Sequence[int]], pairs: Sequence[Tuple[int, int]],
               policy: str = "early") -> Tree:
    """Emit C ops for ``pairs`` (ids refer to live tensors; new ids are
    allocated in order) and S ops around them.

    early: after C i j -> k, S k l for every neighbour l of k, ascending l.
    late:  before C i j, S i l for every neighbour l != j of i (ascending),
           then S j l for every neighbour l != i of j.
    S ops whose shared size is <= chi are skipped at run time, so the same
    tree serves every chi.
    """
    n = len(net_bonds)
    bonds: Dict[int, List[int]] = {t: list(b) for t, b in enumerate(net_bonds)}
    owner: Dict[int, List[int]] = {}
    for t, bl in bonds.items():
        for b in bl:
            owner.setdefault(b, []).append(t)
    nxt = n
    ops: List[tuple] = []
    for i, j in pairs:
        if i not in bonds or j not in bonds or i == j:
            raise ValueError(f"pair ({i}, {j}) is not two live tensors")
        if policy == "late":
            for l in _neighbours(bonds, owner, i):
                if l != j:
                    ops.append(("S", i, l))
            for l in _neighbours(bonds, owner, j):
                if l != i:
                    ops.append(("S", j, l))
        k = nxt
        nxt += 1
        ops.append(("C", i, j, k))
        sj = set(bonds[j])
        si = set(bonds[i])
        newb = [b for b in bonds[i] if b not in sj] + [b for b in bonds[j] if b not in si]
        for b in si & sj:
            del owner[b]
        for b in newb:
            owner[b] = [k if o in (i, j) else o for o in owner[b]]
        del bonds[i], bonds[j]
        bonds[k] = newb
        if policy == "early":
            for l in _neighbours(bonds, owner, k):
                ops.append(("S", k, l))
    return Tree(n, ops)


def sequential_pairs(n: int) -> List[Tuple[int, int]]:
    """Contract tensors 0, 1, 2, ... into one growing tensor."""
    pairs = []
    acc = 0
    nxt = n
    for t in range(1, n):
        pairs.append((acc, t))
        acc = nxt
        nxt += 1
    return pairs


# ---------------------------------------------------------------------------
# greedy builder


def centrality(n: int, adj: Sequence[Sequence[int]]) -> np.ndarray:
    """c[v] ~ sum_{u != v} 1/sqrt(d(u, v) + 1), rescaled to [0, 1] (SI, tree builders)."""
    c = np.zeros(n)
    for s in range(n):
        dist = [-1] * n
        dist[s] = 0
        q = [s]
        h = 0
        while h < len(q):
            u = q[h]
            h += 1
            for w in adj[u]:
                if dist[w] < 0:
                    dist[w] = dist[u] + 1
                    q.append(w)
        c[s] = sum(1.0 / math.sqrt(d + 1) for u, d in enumerate(dist) if u != s and d >= 0)
    lo, hi = c.min(), c.max()
    return (c - lo) / (hi - lo) if hi > lo else np.zeros(n)


class _Sim:
    """Live tensors with bond sizes, for scoring candidate contractions."""

    def __init__(self, net_bonds: Sequence[Sequence[int]], bond_dims: Sequence[int]):
        self.bonds: Dict[int, List[int]] = {t: list(b) for t, b in enumerate(net_bonds)}
        self.dim: Dict[int, int] = {b: int(d) for b, d in enumerate(bond_dims)}
        self.owner: Dict[int, List[int]] = {}
        for t, bl in self.bonds.items():
            for b in bl:
                self.owner.setdefault(b, []).append(t)
        self.next_bond = len(bond_dims)

    def log2size(self, t: int) -> float:
        return sum(math.log2(self.dim[b]) for b in self.bonds[t])

    def groups(self, t: int) -> Dict[int, List[int]]:
        """neighbour -> shared bonds (in t's order)."""
        g: Dict[int, List[int]] = {}
        for b in self.bonds[t]:
            for o in self.owner[b]:
                if o != t:
                    g.setdefault(o, []).append(b)
        return g

    def contract_sizes(self, i: int, j: int, chi: int) -> Tuple[float, float]:
        """(log2 size before, log2 size after early compression) of the new tensor."""
        gi, gj = self.groups(i), self.groups(j)
        before = 0.0
        after = 0.0
        li, lj = self.log2size(i), self.log2size(j)
        nb = set(gi) | set(gj)
        nb.discard(i)
        nb.discard(j)
        tot: Dict[int, float] = {}
        for src in (gi, gj):
            for l, bl in src.items():
                if l in (i, j):
                    continue
                tot[l] = tot.get(l, 0.0) + sum(math.log2(self.dim[b]) for b in bl)
        shared = sum(math.log2(self.dim[b]) for b in gi.get(j, []))
        lk = li + lj - 2 * shared
        for l, s in tot.items():
            before += s
            if s > math.log2(chi) + 1e-9:
                other = self.log2size(l) - s
                after += min(math.log2(chi), lk - s, other)
            else:
                after += s
        return before, after

    def contract(self, i: int, j: int, k: int) -> None:
        si, sj = set(self.bonds[i]), set(self.bonds[j])
        newb = [b for b in self.bonds[i] if b not in sj] + [b for b in self.bonds[j] if b not in si]
        for b in si & sj:
            del self.owner[b]
        for b in newb:
            self.owner[b] = [k if o in (i, j) else o for o in self.owner[b]]
        del self.bonds[i], self.bonds[j]
        self.bonds[k] = newb

    def compress(self, i: int, j: int, chi: int) -> bool:
        sh = [b for b in self.bonds[i] if b in set(self.bonds[j])]
        dab = 1
        for b in sh:
            dab *= self.dim[b]
        if dab <= chi:
            return False
        da = 1
        for b in self.bonds[i]:
            if b not in sh:
                da *= self.dim[b]
        db = 1
        for b in self.bonds[j]:
            if b not in sh:
                db *= self.dim[b]
        knew = min(chi, da, db)
        nb = self.next_bond
        self.next_bond += 1
        self.dim[nb] = knew
        for t in (i, j):
            out = []
            placed = False
            for b in self.bonds[t]:
                if b in sh:
                    if not placed:
                        out.append(nb)
                        placed = True
                else:
                    out.append(b)
            self.bonds[t] = out
        for b in sh:
            del self.owner[b]
        self.owner[nb] = [i, j]
        return True


def local_spanning_tree(net_bonds: Sequence[Sequence[int]], bond_dims: Sequence[int], start: Sequence[int],
                        r: Optional[int] = None, score=None) -> Tuple[List[Tuple[int, int]], List[int]]:
    """The r-local spanning tree of Algorithm 2 (r = None: unbounded).

    Grows a region from the nodes `start` one node at a time: candidates are
    (u, v, r_uv) with u in the region, v a neighbour outside it and r_uv its
    distance from the start region; the best candidate (largest `score(u, v,
    r_uv, region)`, default: the closest, then the largest connectivity -- the
    product of the sizes of the bonds v shares with the region) is popped,
    and v, if still outside and within distance r, joins the region with the
    pair (u, v) appended to the tree.  Returns (ordered pairs, region).
    """
    n = len(net_bonds)
    owner: Dict[int, List[int]] = {}
    for t, bl in enumerate(net_bonds):
        for b in bl:
            owner.setdefault(b, []).append(t)
    nbr: List[Dict[int, float]] = [dict() for _ in range(n)]   # neighbour -> log2 shared size
    for t, bl in enumerate(net_bonds):
        for b in bl:
            for o in owner[b]:
                if o != t:
                    nbr[t][o] = nbr[t].get(o, 0.0) + math.log2(bond_dims[b])
    region = set(start)
    order = list(start)

    def connectivity(v):
        return sum(w for o, w in nbr[v].items() if o in region)

    if score is None:
        def score(u, v, ruv, reg):
            return (-ruv, connectivity(v), -v)

    cands: Dict[Tuple[int, int], int] = {}
    for u in start:
        for v in nbr[u]:
            if v not in region:
                cands[(u, v)] = 1
    tau: List[Tuple[int, int]] = []
    while cands:
        (u, v), ruv = max(cands.items(), key=lambda kv: score(kv[0][0], kv[0][1], kv[1], region))
        del cands[(u, v)]
        if v in region or (r is not None and ruv > r):
            continue
        region.add(v)
        order.append(v)
        tau.append((u, v))
        for w in nbr[v]:
            if w not in region and (v, w) not in cands:
                cands[(v, w)] = ruv + 1
    return tau, order


def span(net_bonds: Sequence[Sequence[int]], bond_dims: Sequence[int], policy: str = "early",
         start: str = "central", priority: Sequence[str] = ("distance", "connectivity", "ndim", "centrality"),
         signs: Optional[Dict[str, float]] = None, temperature: float = 0.0, seed: int = 0) -> Tree:
    """Span tree builder (SI "Span"): a spanning tree grown from one node by
    Algorithm 2 with r unbounded, contracted leaves inwards.

    The start node has the highest (start="central") or lowest ("peripheral")
    centrality.  Candidates (u, v) are ranked by the features in `priority`
    order (lexicographically), each multiplied by its sign (default: prefer
    close, well connected, low-dimensional, central nodes):
      distance     -- v's distance from the start node,
      connectivity -- log2 of the product of the bond sizes v shares with the region,
      ndim         -- number of bonds of v,
      centrality   -- v's centrality in [0, 1],
    with `temperature` times Gumbel noise added to the first feature.  The
    spanning tree's ordered pairs, reversed, are the contractions (each leaf
    into its parent), with S ops placed by `policy` as in from_pairs.
    """
    n = len(net_bonds)
    sg = {"distance": -1.0, "connectivity": 1.0, "ndim": -1.0, "centrality": 1.0}
    sg.update(signs or {})
    owner: Dict[int, List[int]] = {}
    for t, bl in enumerate(net_bonds):
        for b in bl:
            owner.setdefault(b, []).append(t)
    adj = [sorted(set(o for b in net_bonds[v] for o in owner[b] if o != v)) for v in range(n)]
    cent = centrality(n, adj)
    s0 = int(np.argmax(cent)) if start == "central" else int(np.argmin(cent))
    rng = np.random.default_rng(seed)
    noise: Dict[Tuple[int, int], float] = {}
    shared: List[Dict[int, float]] = [dict() for _ in range(n)]
    for t, bl in enumerate(net_bonds):
        for b in bl:
            for o in owner[b]:
                if o != t:
                    shared[t][o] = shared[t].get(o, 0.0) + math.log2(bond_dims[b])

    def score(u, v, ruv, region):
        feats = {"distance": float(ruv),
                 "connectivity": sum(w for o, w in shared[v].items() if o in region),
                 "ndim": float(len(net_bonds[v])),
                 "centrality": float(cent[v])}
        key = [sg[f] * feats[f] for f in priority]
        if temperature > 0.0:
            if (u, v) not in noise:
                noise[(u, v)] = float(rng.gumbel())
            key[0] += temperature * noise[(u, v)]
        return tuple(key) + (-v,)

    tau, order = local_spanning_tree(net_bonds, bond_dims, [s0], None, score)
    if len(order) != n:
        raise ValueError("span: the network is not connected")
    cur = {v: v for v in range(n)}
    nxt = n
    pairs: List[Tuple[int, int]] = []
    for u, v in reversed(tau):
        pairs.append((cur[u], cur[v]))
        cur[u] = nxt
        nxt += 1
    return from_pairs(net_bonds, pairs, policy)


def _combine(mode: str, a: float, b: float) -> float:
    """The SI's reductions of a pair of input features: min, max, sum, mean or difference."""
    if mode == "sum":
        return a + b
    if mode == "min":
        return min(a, b)
    if mode == "max":
        return max(a, b)
    if mode == "mean":
        return 0.5 * (a + b)
    if mode == "diff":
        return abs(a - b)
    raise ValueError(f"unknown reduction {mode!r}")


# Greedy weights that grow boundary-like fronts on regular 2D lattices (found by
# hyper_search over the SI's 11 dimensions on a 32 x 32, D = 4, chi = 64
# lattice): the size after compression against the larger input's size, and a
# simulated chi_greedy of chi / 2.
def greedy_front_params(chi: int) -> Dict[str, object]:
    return dict(w_new=1.0, w_old=0.2, w_inputs=-0.85, inputs_mode="max", chi_greedy=max(1, chi // 2))


# Span parameters that hyper_search(builder="span", n_trials=24, seed=0) found on
# the 32 x 32, D = 4, chi = 64 lattice: late compression from a peripheral
# start, candidates by centrality, then connectivity, then distance (traced
# cost 1.59e11 against 1.82e11 for boundary rows; 2.62e10 against 3.38e10 on
# 16 x 16).
def span_square_params() -> Dict[str, object]:
    return dict(policy="late", start="peripheral", priority=("centrality", "connectivity", "distance", "ndim"),
                signs={"distance": -1.0, "connectivity": 1.0, "ndim": 1.0, "centrality": 1.0},
                temperature=0.0, seed=18)


def _greedy_loop(sim: "_Sim", members: set, chig: int, score, ops: List[tuple], nxt: int, on_contract=None) -> int:
    """Contract adjacent pairs of the live tensors in ``members`` (updated in
    place), lowest ``score(i, j)`` first, until no two members share a bond.
    After each contraction C i j -> k, an S op with every neighbour of k
    (ascending, members or not), simulated at chig: Algorithm 1's early
    compression.  Stale heap entries are recognised by per-tensor versions,
    bumped when a compression changes a tensor.  Returns the next free id."""
    version: Dict[int, int] = {v: 0 for v in members}
    heap: List[Tuple[float, int, int, int, int]] = []

    def push_around(t: int) -> None:
        for l in sim.groups(t):
            if l in members:
                a, b = (t, l) if t < l else (l, t)
                heapq.heappush(heap, (score(a, b), a, b, version[a], version[b]))

    for v in sorted(members):
        for l in sim.groups(v):
            if v < l and l in members:
                heapq.heappush(heap, (score(v, l), v, l, 0, 0))
    while heap:
        _, i, j, vi, vj = heapq.heappop(heap)
        if i not in members or j not in members or version[i] != vi or version[j] != vj:
            continue
        k = nxt
        nxt += 1
        ops.append(("C", i, j, k))
        sim.contract(i, j, k)
        members.discard(i)
        members.discard(j)
        members.add(k)
        if on_contract is not None:
            on_contract(i, j, k)
        version[k] = 0
        for l in sorted(sim.groups(k)):
            ops.append(("S", k, l))
            if sim.compress(k, l, chig) and l in version:
                version[l] += 1
        push_around(k)
        for l in sim.groups(k):
            if l in members:
                push_around(l)
    return nxt


def greedy(net_bonds: Sequence[Sequence[int]], bond_dims: Sequence[int], chi: int,
           seed: int = 0, temperature: float = 0.0, w_new: float = 1.0, w_old: float = 0.0,
           w_inputs: float = -1.0, w_subgraph: float = 0.0, w_centrality: float = 0.0,
           chi_greedy: Optional[int] = None, policy: str = "early", inputs_mode: str = "sum",
           subgraph_mode: str = "sum", centrality_mode: str = "mean", centrality_prop: str = "mean") -> Tree:
    """Greedy ordered tree (SI "Greedy"): repeatedly contract the adjacent pair of lowest score

        score = w_new * log2|k after compression| + w_old * log2|k before|
              + w_inputs * R_in(log2|i|, log2|j|) + w_subgraph * R_sub(|S(i)|, |S(j)|)
              + w_centrality * R_cen(c_i, c_j) + temperature * Gumbel,

    each R one of the SI's reductions (min, max, sum, mean or difference; the
    centrality takes min, max, mean or difference) chosen by ``*_mode``, and a
    contracted tensor's centrality propagated from its inputs by
    ``centrality_prop`` (min, max or mean).  Early compression is simulated at
    chi_greedy (default chi) after each step.  Disconnected components are
    joined by outer products at the end.

    On lattices the reduction matters: with inputs_mode="max" and
    w_inputs = -w_new, absorbing a small tensor into a large one scores the
    growth of the large one, so boundary-like fronts grow instead of 2D blobs
    whose perimeters blow up the tensor sizes.
    """
    chig = chi_greedy or chi
    rng = np.random.default_rng(seed)
    n = len(net_bonds)
    sim = _Sim(net_bonds, bond_dims)
    adj0 = [sorted(set(o for b in net_bonds[v] for o in sim.owner[b] if o != v)) for v in range(n)]
    cent = {v: float(c) for v, c in enumerate(centrality(n, adj0))} if w_centrality else {v: 0.0 for v in range(n)}
    sub = {v: 1 for v in range(n)}
    ops: List[tuple] = []
    nxt = n

    def score(i: int, j: int) -> float:
        before, after = sim.contract_sizes(i, j, chig)
        s = w_new * after + w_old * before + w_inputs * _combine(inputs_mode, sim.log2size(i), sim.log2size(j))
        s += w_subgraph * _combine(subgraph_mode, sub[i], sub[j])
        if w_centrality:
            s += w_centrality * _combine(centrality_mode, cent[i], cent[j])
        if temperature:
            s += temperature * float(-math.log(-math.log(rng.uniform(1e-12, 1.0))))
        return s

    def on_contract(i: int, j: int, k: int) -> None:
        sub[k] = sub[i] + sub[j]
        cent[k] = {"min": min, "max": max}.get(centrality_prop, lambda a, b: 0.5 * (a + b))(cent[i], cent[j])

    nxt = _greedy_loop(sim, set(range(n)), chig, score, ops, nxt, on_contract)
    live = sorted(sim.bonds)
    acc = live[0] if live else None
    for t in live[1:]:
        ops.append(("C", acc, t, nxt))
        sim.contract(acc, t, nxt)
        acc = nxt
        nxt += 1
    if policy != "early":
        raise ValueError("greedy emits early compression")
    return Tree(n, ops)


# ---------------------------------------------------------------------------
# tracing (Sec. "Tree cost functions" of the SI)


class _Tracer:
    """Running cost of an ordered tree, one op at a time (the SI's cost units)

    contraction (m, n) x (n, k): m n k;  QR of (m, n), m >= n: 2 m n^2 - 2/3 n^3;
    SVD of (m, n), m >= n: 4 m n^2 - 4/3 n^3;  plus peak live memory M (elements)
    and the largest tensor W.  QR here is of each side of a compression
    (D_A x D_AB and D_AB x D_B), the SVD of the r_A x r_B core.
    """

    def __init__(self, net_bonds: Sequence[Sequence[int]], bond_dims: Sequence[int], chi: int):
        self.sim = _Sim(net_bonds, bond_dims)
        self.chi = chi
        self.cost_c = self.cost_qr = self.cost_svd = 0.0
        self.sizes = {t: 2.0 ** self.sim.log2size(t) for t in self.sim.bonds}
        self.live = sum(self.sizes.values())
        self.peak = self.live
        self.wmax = max(self.sizes.values()) if self.sizes else 0.0
        self.n_comp = 0

    @staticmethod
    def _qr(m: float, nn: float) -> float:
        if m < nn:
            m, nn = nn, m
        return 2 * m * nn * nn - 2.0 / 3.0 * nn ** 3

    @staticmethod
    def _svd(m: float, nn: float) -> float:
        if m < nn:
            m, nn = nn, m
        return 4 * m * nn * nn - 4.0 / 3.0 * nn ** 3

    def contract(self, i: int, j: int, k: int) -> None:
        sim, sizes = self.sim, self.sizes
        sh = [b for b in sim.bonds[i] if b in set(sim.bonds[j])]
        dab = 2.0 ** sum(math.log2(sim.dim[b]) for b in sh)
        m = sizes[i] / dab
        nn = sizes[j] / dab
        self.cost_c += m * dab * nn
        sim.contract(i, j, k)
        sizes[k] = m * nn
        self.live += sizes[k]
        self.peak = max(self.peak, self.live)
        self.live -= sizes.pop(i) + sizes.pop(j)
        self.wmax = max(self.wmax, sizes[k])

    def compress(self, i: int, j: int) -> None:
        sim, sizes, chi = self.sim, self.sizes, self.chi
        sh = [b for b in sim.bonds[i] if b in set(sim.bonds[j])]
        dab = 2.0 ** sum(math.log2(sim.dim[b]) for b in sh)
        if dab <= chi:
            return
        da = sizes[i] / dab
        db = sizes[j] / dab
        ra, rb = min(da, dab), min(db, dab)
        self.cost_qr += self._qr(da, dab) + self._qr(dab, db)
        self.cost_c += ra * dab * rb
        self.cost_svd += self._svd(ra, rb)
        kk = min(chi, da, db)
        self.cost_c += da * ra * kk + kk * rb * db
        sim.compress(i, j, chi)
        self.live -= sizes[i] + sizes[j]
        sizes[i] = da * kk
        sizes[j] = kk * db
        self.live += sizes[i] + sizes[j]
        self.n_comp += 1

    def step(self, op: tuple) -> None:
        if op[0] == "C":
            self.contract(op[1], op[2], op[3])
        else:
            self.compress(op[1], op[2])

    def result(self) -> Dict[str, float]:
        return {"contract": self.cost_c, "qr": self.cost_qr, "svd": self.cost_svd,
                "total": self.cost_c + self.cost_qr + self.cost_svd, "peak": self.peak, "wmax": self.wmax,
                "compressions": self.n_comp}


def trace_cost(net_bonds: Sequence[Sequence[int]], bond_dims: Sequence[int], tree: Tree, chi: int) -> Dict[str, float]:
    """Walk the tree for one chi and count the paper's cost units (see _Tracer):
    contraction, QR and SVD costs, their total C, the peak live memory M and
    the largest tensor W, and the number of compressions that fire."""
    tr_ = _Tracer(net_bonds, bond_dims, chi)
    for op in tree.ops:
        tr_.step(op)
    return tr_.result()


# ---------------------------------------------------------------------------
# hyper-optimization loop (Algorithm 3) by random search

SPAN_FEATURES = ("distance", "connectivity", "ndim", "centrality")


def hyper_search(net_bonds: Sequence[Sequence[int]], bond_dims: Sequence[int], chi: int, n_trials: int = 64,
                 seed: int = 0, builder: str = "span", objective: str = "total"):
    """Sample builder hyper-parameters, build a tree, score it with the cost
    tracer, keep the best (Algorithm 3 with random sampling in place of a
    Bayesian optimizer).

    builder "span": the feature priority order, the signs, the start node
    (central / peripheral), a temperature in {0, 0.5, 2} and the compression
    policy (early / late).  builder "greedy": the score weights, the
    temperature and chi_greedy.  objective: a key of trace_cost's result
    ("total" = the SI's cost C, "peak" = largest intermediate, ...).
    Returns (best tree, its parameters, its objective value, [objective of each trial]).
    """
    rng = np.random.default_rng(seed)
    best = (None, None, math.inf)
    hist: List[float] = []
    for trial in range(n_trials):
        if builder == "span":
            params = dict(policy=str(rng.choice(["early", "late"])),
                          start=str(rng.choice(["central", "peripheral"])),
                          priority=tuple(str(x) for x in rng.permutation(SPAN_FEATURES)),
                          signs={f: float(rng.choice([-1.0, 1.0])) for f in SPAN_FEATURES},
                          temperature=float(rng.choice([0.0, 0.0, 0.5, 2.0])), seed=trial)
            tree = span(net_bonds, bond_dims, **params)
        elif builder == "greedy":
            # the SI's 11 dimensions: three size weights, the input-size reduction,
            # subgraph weight and reduction, centrality weight, reduction and
            # propagation, temperature and chi_greedy; sizes after compression
            # keep weight 1 (only ratios matter), the input weight is drawn
            # around -1 where a front grows by absorbing small tensors
            params = dict(seed=trial, temperature=float(rng.choice([0.0, 0.0, 0.05, 0.2])),
                          w_new=1.0, w_old=float(rng.uniform(-0.3, 0.3)),
                          w_inputs=float(rng.uniform(-1.1, -0.7)),
                          inputs_mode=str(rng.choice(["max", "max", "sum", "mean", "diff", "min"])),
                          w_subgraph=float(rng.choice([0.0, 1.0]) * rng.uniform(-0.02, 0.05)),
                          subgraph_mode=str(rng.choice(["sum", "max", "min", "mean", "diff"])),
                          w_centrality=float(rng.choice([0.0, 1.0]) * rng.uniform(-1.0, 1.0)),
                          centrality_mode=str(rng.choice(["mean", "min", "max", "diff"])),
                          centrality_prop=str(rng.choice(["mean", "min", "max"])),
                          chi_greedy=int(rng.choice([chi, chi, 2 * chi, max(1, chi // 2)])))
            tree = greedy(net_bonds, bond_dims, chi, **params)
        else:
            raise ValueError(builder)
        cost = float(trace_cost(net_bonds, bond_dims, tree, chi)[objective])
        hist.append(cost)
        if cost < best[2]:
            best = (tree, params, cost)
    return best[0], best[1], best[2], hist
