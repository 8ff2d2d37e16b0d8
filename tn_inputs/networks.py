"""Seeded tensor-network builders for the paper's benchmark models.

Graphs: square / cubic lattices with open boundaries, random 3-regular graphs
(pairing model with rejection), rings and trees.  Tensors:

* Ising (SI "Ising Model"): one tensor per spin, T_v = sum_s prod_e W_e[s, a_e]
  with W_L W_R^T = exp(beta J s s') on every bond.  For J > 0 the paper's
  real symmetric W is used on both ends; for any sign of J the split
  W_L = h diag(sqrt(2 cosh bJ), sqrt(2|sinh bJ|)),
  W_R = h diag(sqrt(2 cosh bJ), sgn(sinh bJ) sqrt(2|sinh bJ|)), h the 2x2
  Hadamard, is used, the lower vertex id taking W_L.  Spin +1 is index 0.
* Random entries: i.i.d. Normal(mean, std) (config of the 32x32 D=4 study)
  or Uniform[lambda, 1] (the paper's URand model).
* Dimer covers / positive #1-in-3SAT (SI "Dimer covers"): T = 1 iff the
  indices around the vertex sum to 1.
* Corner double line (SI "CDL"): each plaquette carries a loop of four d x d
  identities; bonds on the open boundary keep only their inner half.

Random numbers come from numpy's PCG64 ``default_rng(seed)``; both sides of
every comparison read the same written network, so the generator choice
never affects parity.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .formats import Network, edges_to_bonds

# ---------------------------------------------------------------------------
# graphs


def square_lattice(lx: int, ly: int) -> Tuple[int, List[Tuple[int, int]]]:
    """Open-boundary lx x ly square lattice; site (x, y) has id y*lx + x.

    Edge order: for each site in id order, its +x edge then its +y edge.
    """
    edges = []
    for y in range(ly):
        for x in range(lx):
            s = y * lx + x
            if x + 1 < lx:
                edges.append((s, s + 1))
            if y + 1 < ly:
                edges.append((s, s + lx))
    return lx * ly, edges


def cubic_lattice(lx: int, ly: int, lz: int) -> Tuple[int, List[Tuple[int, int]]]:
    """Open-boundary cubic lattice; site (x, y, z) has id (z*ly + y)*lx + x."""
    edges = []
    for z in range(lz):
        for y in range(ly):
            for x in range(lx):
                s = (z * ly + y) * lx + x
                if x + 1 < lx:
                    edges.append((s, s + 1))
                if y + 1 < ly:
                    edges.append((s, s + lx))
                if z + 1 < lz:
                    edges.append((s, s + lx * ly))
    return lx * ly * lz, edges


def ring(n: int) -> Tuple[int, List[Tuple[int, int]]]:
    return n, [(i, (i + 1) % n) if i + 1 < n else (0, n - 1) for i in range(n)]


def random_tree_graph(n: int, seed: int) -> Tuple[int, List[Tuple[int, int]]]:
    """Random labelled tree: vertex v > 0 attaches to a uniformly chosen earlier vertex."""
    rng = np.random.default_rng(seed)
    return n, [(int(rng.integers(0, v)), v) for v in range(1, n)]


def _connected(n: int, edges: Sequence[Tuple[int, int]]) -> bool:
    adj: List[List[int]] = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    seen = [False] * n
    stack = [0]
    seen[0] = True
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if not seen[w]:
                seen[w] = True
                stack.append(w)
    return all(seen)


def random_regular_graph(n: int, d: int, seed: int, max_tries: int = 10000) -> Tuple[int, List[Tuple[int, int]]]:
    """Uniform random simple connected d-regular graph by the pairing model.

    Each vertex gets d stubs, the stubs are shuffled and paired; a pairing
    with a self-loop or a repeated edge, or a disconnected result, is
    rejected and redrawn.  Edges are returned sorted (u < v, lexicographic).
    """
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    rng = np.random.default_rng(seed)
    stubs = np.repeat(np.arange(n), d)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        pairs = perm.reshape(-1, 2)
        if np.any(pairs[:, 0] == pairs[:, 1]):
            continue
        es = {(int(min(a, b)), int(max(a, b))) for a, b in pairs}
        if len(es) != len(pairs):
            continue
        edges = sorted(es)
        if _connected(n, edges):
            return n, edges
    raise RuntimeError("random_regular_graph: too many rejections")


# fixed small cubic graphs with known perfect-matching counts
def k4() -> Tuple[int, List[Tuple[int, int]]]:
    return 4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def k33() -> Tuple[int, List[Tuple[int, int]]]:
    return 6, [(a, b) for a in range(3) for b in range(3, 6)]


def petersen() -> Tuple[int, List[Tuple[int, int]]]:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return 10, [(min(u, v), max(u, v)) for u, v in outer + spokes + inner]


def cube_q3() -> Tuple[int, List[Tuple[int, int]]]:
    edges = []
    for v in range(8):
        for bit in range(3):
            w = v ^ (1 << bit)
            if v < w:
                edges.append((v, w))
    return 8, edges


# ---------------------------------------------------------------------------
# tensors


def ising_bond_factors(beta: float, J: float, symmetric: bool) -> Tuple[np.ndarray, np.ndarray]:
    """(W_L, W_R) with W_L @ W_R.T == [[e^{bJ}, e^{-bJ}], [e^{-bJ}, e^{bJ}]]."""
    c = math.cosh(beta * J)
    s = math.sinh(beta * J)
    if symmetric:
        if J < 0:
            raise ValueError("the symmetric split needs J >= 0")
        a, b = math.sqrt(c), math.sqrt(s)
        w = np.array([[a + b, a - b], [a - b, a + b]]) / math.sqrt(2.0)
        return w, w
    h = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
    wl = h @ np.diag([math.sqrt(2 * c), math.sqrt(2 * abs(s))])
    wr = h @ np.diag([math.sqrt(2 * c), math.copysign(math.sqrt(2 * abs(s)), s) if s != 0 else 0.0])
    return wl, wr


def _site_from_factors(factors: Sequence[np.ndarray]) -> np.ndarray:
    """T[a_1..a_d] = sum_s prod_e F_e[s, a_e] (COPY tensor with a factor on every leg)."""
    out = None
    for s in range(2):
        term = np.ones(())
        for f in factors:
            term = np.multiply.outer(term, f[s])
        out = term if out is None else out + term
    return np.asarray(out, dtype=np.float64)


def ising_network(n: int, edges: Sequence[Tuple[int, int]], beta: float,
                  J: "float | Sequence[float]" = 1.0, symmetric: Optional[bool] = None) -> Network:
    """Partition function Z = sum_s prod_<ij> exp(beta J_ij s_i s_j) as a network.

    ``symmetric`` defaults to True when every J_ij > 0 (the paper's W),
    else the W_L / W_R split.  Every bond has dimension 2.
    """
    Js = np.full(len(edges), float(J)) if np.isscalar(J) else np.asarray(J, dtype=np.float64)
    if symmetric is None:
        symmetric = bool(np.all(Js > 0))
    bonds = edges_to_bonds(n, edges)
    per_edge = [ising_bond_factors(beta, float(j), symmetric) for j in Js]
    data = []
    for v in range(n):
        facs = []
        for e in bonds[v]:
            u, w = edges[e]
            wl, wr = per_edge[e]
            facs.append(wl if v == min(u, w) else wr)
        data.append(_site_from_factors(facs))
    return Network([2] * len(edges), bonds, data)


def random_network(n: int, edges: Sequence[Tuple[int, int]], D: int, seed: int,
                   dist: str = "normal", mean: float = 0.2, std: float = 1.0, lam: float = 0.0) -> Network:
    """Every bond of size D, entries i.i.d. Normal(mean, std) or Uniform[lam, 1]."""
    rng = np.random.default_rng(seed)
    bonds = edges_to_bonds(n, edges)
    data = []
    for v in range(n):
        shp = (D,) * len(bonds[v])
        if dist == "normal":
            data.append(rng.normal(mean, std, size=shp))
        elif dist == "uniform":
            data.append(rng.uniform(lam, 1.0, size=shp))
        else:
            raise ValueError(dist)
    return Network([D] * len(edges), bonds, data)


def dimer_network(n: int, edges: Sequence[Tuple[int, int]]) -> Network:
    """Perfect-matching count W as a network: T = 1 iff the vertex's indices sum to 1."""
    bonds = edges_to_bonds(n, edges)
    data = []
    for v in range(n):
        d = len(bonds[v])
        t = np.zeros((2,) * d)
        for leg in range(d):
            idx = [0] * d
            idx[leg] = 1
            t[tuple(idx)] = 1.0
        data.append(t)
    return Network([2] * len(edges), bonds, data)


def cdl_network(lx: int, ly: int, d: int) -> Network:
    """Open-boundary corner-double-line network on an lx x ly square lattice.

    Plaquette (x, y) (lower-left corner site (x, y)) exists for x < lx-1,
    y < ly-1 and carries a loop of four d x d identities, one at each corner
    site.  A bond is the pair (halves for the two plaquettes beside it); a
    half with no plaquette has size 1.  Z = d ** ((lx-1)*(ly-1)).
    Bond order per site follows ``square_lattice``'s edge order.
    """
    n, edges = square_lattice(lx, ly)
    bonds = edges_to_bonds(n, edges)

    def plaq(x: int, y: int) -> bool:
        return 0 <= x < lx - 1 and 0 <= y < ly - 1

    # each edge: two halves; record (plaquette, size) for half 0 and half 1
    halves: Dict[int, Tuple[Tuple[int, int], Tuple[int, int]]] = {}
    for e, (u, v) in enumerate(edges):
        x, y = u % lx, u // lx
        if v == u + 1:   # horizontal: plaquette above (x, y), below (x, y-1)
            halves[e] = ((x, y), (x, y - 1))
        else:            # vertical: plaquette right (x, y), left (x-1, y)
            halves[e] = ((x, y), (x - 1, y))
    dims = []
    for e in range(len(edges)):
        p0, p1 = halves[e]
        dims.append((d if plaq(*p0) else 1) * (d if plaq(*p1) else 1))
    data = []
    for s in range(n):
        legs = bonds[s]
        # each leg e has halves (h0, h1) of sizes (a0, a1); leg index = i0 * a1 + i1
        # site tensor = product over plaquettes touching s of delta between the two halves
        shape = []
        half_axes = []  # per leg: list of (plaquette, axis position)
        for e in legs:
            p0, p1 = halves[e]
            a0 = d if plaq(*p0) else 1
            a1 = d if plaq(*p1) else 1
            shape += [a0, a1]
            half_axes.append(((p0, a0), (p1, a1)))
        t = np.ones(shape)
        # group axes by plaquette
        by_p: Dict[Tuple[int, int], List[int]] = {}
        ax = 0
        for (p0, a0), (p1, a1) in half_axes:
            if a0 > 1:
                by_p.setdefault(p0, []).append(ax)
            if a1 > 1:
                by_p.setdefault(p1, []).append(ax + 1)
            ax += 2
        for p, axes in by_p.items():
            if len(axes) != 2:
                raise AssertionError("a plaquette corner must join two halves")
            shp = [1] * len(shape)
            shp[axes[0]] = d
            shp[axes[1]] = d
            t = t * np.eye(d).reshape(shp)
        data.append(t.reshape([dims[e] for e in legs]))
    return Network(dims, bonds, data)


def dimer_entropy_k_regular(k: int) -> float:
    """Large-n limit of log(mean perfect-matching count)/n on random k-regular graphs."""
    return 0.5 * (k - 1) * math.log(k - 1) + 0.5 * (2 - k) * math.log(k)


def beta_sweep(n: int, lo: float = 0.2, hi: float = 0.7) -> np.ndarray:
    """n inverse temperatures spaced uniformly over [lo, hi], both ends included."""
    return lo + (hi - lo) * np.arange(n) / (n - 1)


def spin_glass_couplings(n_edges: int, seed: int, p: float = 0.5) -> np.ndarray:
    """+1 / -1 couplings, -1 with probability p."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random(n_edges) < p, -1.0, 1.0)
