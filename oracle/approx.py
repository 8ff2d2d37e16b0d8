"""Oracle: approximate contraction along an ordered tree (Algorithm 1), FP64.

Test infrastructure only (see the package docstring).

The tree is a list of explicit ops, so the early / late policies of
Algorithm 1 are already expanded into ``S`` ops by the tree generator:

  C i j k : k <- sum over the bonds shared by i and j of T_i T_j (Eq. 1 for one
            pair; Fig. 3A/B).  k lists i's remaining bonds in i's order, then
            j's remaining bonds in j's order.
  S i j   : if the product D_AB of the shared bond sizes exceeds chi, compress
            them (Sec. "Bond compression strategies"):
              A = T_i as (D_A x D_AB), B = T_j as (D_AB x D_B), shared bonds in
              i's order on both;
              A = Q_A R_A (QR), B = L_B Q_B (LQ), R_AB = R_A L_B;
              R_AB = U sigma V^T (SVD), keep the k = min(chi, D_A, D_B) largest;
              A_bar = Q_A U_k sigma_k^(1/2), B_bar = sigma_k^(1/2) V_k^T Q_B.
            In each tensor the new bond takes the place of that tensor's first
            shared bond; the other shared bonds disappear.

Readings where the paper is silent:
  * running log-norm: after every op, each output X is divided by 2^e with
    e the binary exponent of max|X| (exact), and e is added to a counter E;
    log|Z| = ln|x| + E ln 2 for the final scalar x.
  * no singular-value cutoff: exactly k values are kept, zeros included.
  * a wide side (D_A < D_AB) is factored with a square Q_A (numpy's reduced
    QR of a wide matrix), i.e. R_A = Q_A^T A.
  * Z = 0 gives log|Z| = -inf and sign 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from tn_inputs.formats import Network, Tree


@dataclass
class Result:
    logabs: float
    sign: int
    compressions: int = 0
    # per executed compression: (k, discarded weight sum_{i>k} s_i^2 / sum s_i^2,
    #                            gap (s_k - s_{k+1}) / s_1, or 1 when s_k <= 1e-13 s_1)
    diag: List[Tuple[int, float, float]] = field(default_factory=list)


def _prod(dims) -> int:
    p = 1
    for d in dims:
        p *= int(d)
    return p


def _matricize(t: np.ndarray, bonds: List[int], rows: List[int], cols: List[int]) -> np.ndarray:
    """Group the axes of t: rows bonds (in the given order) x cols bonds (Fig. 3A)."""
    perm = [bonds.index(b) for b in rows + cols]
    shp = t.shape
    return np.transpose(t, perm).reshape(_prod(shp[p] for p in perm[: len(rows)]),
                                         _prod(shp[p] for p in perm[len(rows):]))


def _rescale(x: np.ndarray) -> Tuple[np.ndarray, int]:
    """X -> X * 2^-e with e = exponent of max|X| (frexp convention, mantissa in [0.5, 1))."""
    m = float(np.max(np.abs(x))) if x.size else 0.0
    if m == 0.0 or not math.isfinite(m):
        return x, 0
    e = math.frexp(m)[1]
    return np.ldexp(x, -e), e


def contract_pair(ti: np.ndarray, bi: List[int], tj: np.ndarray, bj: List[int]):
    """Pairwise contraction over the shared bonds (Eq. 1 restricted to two tensors)."""
    sj = set(bj)
    si = set(bi)
    shared = [b for b in bi if b in sj]
    ri = [b for b in bi if b not in sj]
    rj = [b for b in bj if b not in si]
    a = _matricize(ti, bi, ri, shared)
    b = _matricize(tj, bj, shared, rj)
    c = a @ b
    dims = [ti.shape[bi.index(x)] for x in ri] + [tj.shape[bj.index(x)] for x in rj]
    return c.reshape(dims), ri + rj


def compress_pair(ti: np.ndarray, bi: List[int], tj: np.ndarray, bj: List[int], chi: int, new_bond: int):
    """Truncated QR/LQ/SVD compression of the bonds shared by i and j.

    Returns None when D_AB <= chi (Algorithm 1 only compresses bonds larger
    than chi), else (A_bar, bonds_i, B_bar, bonds_j, k, discarded, gap).
    """
    sj = set(bj)
    shared = [b for b in bi if b in sj]
    dab = _prod(ti.shape[bi.index(b)] for b in shared)
    if dab <= chi:
        return None
    ri = [b for b in bi if b not in sj]
    si = set(bi)
    rj = [b for b in bj if b not in si]
    a = _matricize(ti, bi, ri, shared)            # D_A x D_AB
    b = _matricize(tj, bj, shared, rj)            # D_AB x D_B
    qa, ra = np.linalg.qr(a)                      # A = Q_A R_A
    qbt, lbt = np.linalg.qr(b.T)                  # B^T = Q' R'  ->  B = R'^T Q'^T = L_B Q_B
    lb, qb = lbt.T, qbt.T
    rab = ra @ lb                                 # R_AB = R_A L_B
    u, s, vt = np.linalg.svd(rab, full_matrices=False)
    k = min(chi, len(s))
    sq = np.sqrt(s[:k])
    abar = qa @ (u[:, :k] * sq[None, :])          # A_bar = Q_A U sigma^(1/2)
    bbar = (sq[:, None] * vt[:k, :]) @ qb         # B_bar = sigma^(1/2) V^T Q_B
    tot = float(np.sum(s * s))
    disc = float(np.sum(s[k:] ** 2)) / tot if tot > 0 else 0.0
    # gap at the cut; a cut that only drops rounding-level values is unambiguous
    if k < len(s) and s[0] > 0 and s[k - 1] > 1e-13 * s[0]:
        gap = float((s[k - 1] - s[k]) / s[0])
    else:
        gap = 1.0

    def place(bonds: List[int], rem: List[int], mat: np.ndarray, rem_first: bool, shape_src, bonds_src):
        # new bond goes where the first shared bond was; other shared bonds vanish
        out, placed = [], False
        for x in bonds:
            if x in sj and x in si:
                if not placed:
                    out.append(new_bond)
                    placed = True
            else:
                out.append(x)
        rem_dims = [shape_src[bonds_src.index(x)] for x in rem]
        cur = (rem + [new_bond]) if rem_first else ([new_bond] + rem)
        t = mat.reshape((rem_dims + [k]) if rem_first else ([k] + rem_dims))
        t = np.transpose(t, [cur.index(x) for x in out])
        return np.ascontiguousarray(t), out

    ai, nbi = place(bi, ri, abar, True, ti.shape, bi)
    bj2, nbj = place(bj, rj, bbar, False, tj.shape, bj)
    return ai, nbi, bj2, nbj, k, disc, gap


def contract(net: Network, tree: Tree, chi: Optional[int], rescale: bool = True) -> Result:
    """Run the ordered tree on ``net`` (Algorithm 1 with explicit ops).

    chi=None means no compression (exact contraction along the tree).
    """
    if tree.n_inputs != net.n_tensors:
        raise ValueError("tree and network disagree on the number of tensors")
    T: Dict[int, np.ndarray] = {i: np.asarray(d, dtype=np.float64) for i, d in enumerate(net.data)}
    B: Dict[int, List[int]] = {i: list(b) for i, b in enumerate(net.bonds)}
    E = 0
    nxt_id = net.n_tensors
    nxt_bond = len(net.bond_dims)
    res = Result(0.0, 0)
    for op in tree.ops:
        if op[0] == "C":
            _, i, j, k = op
            if k != nxt_id:
                raise ValueError(f"C op creates id {k}, expected {nxt_id}")
            c, bc = contract_pair(T.pop(i), B.pop(i), T.pop(j), B.pop(j))
            if rescale:
                c, e = _rescale(c)
                E += e
            T[k], B[k] = c, bc
            nxt_id += 1
        elif op[0] == "S":
            _, i, j = op
            if chi is None:
                continue
            r = compress_pair(T[i], B[i], T[j], B[j], chi, nxt_bond)
            if r is None:
                continue
            ai, nbi, bj2, nbj, k, disc, gap = r
            nxt_bond += 1
            if rescale:
                ai, e1 = _rescale(ai)
                bj2, e2 = _rescale(bj2)
                E += e1 + e2
            T[i], B[i], T[j], B[j] = ai, nbi, bj2, nbj
            res.compressions += 1
            res.diag.append((k, disc, gap))
        else:
            raise ValueError(f"unknown op {op!r}")
    # final: product of the remaining scalars (disconnected parts are joined by C ops)
    x = 1.0
    for t in T.values():
        if t.size != 1:
            raise ValueError("tree leaves a tensor with open bonds")
        x *= float(t.reshape(()))
    if x == 0.0:
        res.logabs, res.sign = -math.inf, 0
    else:
        res.logabs = math.log(abs(x)) + E * math.log(2.0)
        res.sign = 1 if x > 0 else -1
    return res


def contract_exact(net: Network, tree: Tree) -> Result:
    """Exact contraction along the tree's C ops (all S ops skipped)."""
    return contract(net, tree, None)
