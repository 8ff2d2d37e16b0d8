"""Oracle: bond compression in the tree gauge of distance r, projector form (FP64).

Test infrastructure only (see the package docstring).

Sec. "Bond compression strategies" (tree gauge) with the SI's r-local
spanning tree (Algorithm 2) and explicit projector form:

  * The environment of the bond between A = T_i and B = T_j is cut to a tree:
    Algorithm 2 grows a region from {i, j}, adding one neighbour at a time
    within graph distance r; each added node hangs off the node that reached
    it, and bonds to other region nodes stay open (the cut loops).
  * QR inwards on virtual copies: for the spanning-tree pairs (u, v) from the
    last added to the first, v's virtual copy is matricized as (its other
    bonds) x (its bonds to u) and replaced by its R factor, which is absorbed
    into u's virtual copy over those bonds.  A and B end up carrying the R
    factors of their sides of the tree.
  * R_A from a QR of A's virtual copy as (other bonds) x (bonds shared with
    B), L_B from an LQ of B's as (shared) x (other); the SVD of R_A L_B =
    U s V^T, kept to k = min(chi, its size); the projectors
    P_L = L_B V_k s_k^-1/2 and P_R = s_k^-1/2 U_k^T R_A are inserted on the
    bond of the original tensors: A <- A P_L, B <- P_R B.  No other tensor
    changes.  With r = 0 this is the plain compression (A P_L = Q_A U_k s_k^1/2).

Readings where the paper is silent:
  * Only tensors made by a contraction (ids >= the number of inputs) join the
    spanning tree besides A and B (the SI excludes input tensors);
    `include_inputs=True` lifts that restriction (used by a pin).
  * Algorithm 2's score: the closest candidate first, then the largest
    connectivity (the product of the sizes of the bonds u and v share),
    then the smallest id of v, then of u.
  * A factor whose matrix has no more rows than columns is not reduced
    (R = the matrix itself): a QR would only rotate the new bond, which the
    projectors do not see.
  * s_k^-1/2 of a kept singular value at or below 1e-13 s_1 is taken as 0
    (the projector form cannot invert a zero singular value).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from tn_inputs.formats import Network, Tree

from .approx import Result, _matricize, _prod, _rescale, contract_pair


def spanning_tree(bonds: Dict[int, List[int]], dims: Dict[int, int], start: Sequence[int], r: int,
                  allowed) -> List[Tuple[int, int]]:
    """Algorithm 2: ordered pairs (u, v) of the r-local spanning tree grown from `start`."""
    owner: Dict[int, List[int]] = {}
    for t, bl in bonds.items():
        for b in bl:
            owner.setdefault(b, []).append(t)

    def nbrs(u):
        out = set()
        for b in bonds[u]:
            for o in owner[b]:
                if o != u:
                    out.add(o)
        return sorted(out)

    def conn(u, v):
        sv = set(bonds[v])
        p = 1
        for b in bonds[u]:
            if b in sv:
                p *= dims[b]
        return p

    region = set(start)
    cands: Dict[Tuple[int, int], int] = {}
    for u in start:
        for v in nbrs(u):
            if v not in region and allowed(v):
                cands[(u, v)] = 1
    tau: List[Tuple[int, int]] = []
    while cands:
        (u, v), d = min(cands.items(), key=lambda kv: (kv[1], -conn(*kv[0]), kv[0][1], kv[0][0]))
        del cands[(u, v)]
        if v in region or d > r:
            continue
        region.add(v)
        tau.append((u, v))
        for w in nbrs(v):
            if w not in region and allowed(w) and (v, w) not in cands:
                cands[(v, w)] = d + 1
    return tau


def _reduce_rows(mat: np.ndarray) -> np.ndarray:
    """R factor of mat (rows x cols); mat itself when rows <= cols."""
    if mat.shape[0] <= mat.shape[1]:
        return mat
    return np.linalg.qr(mat, mode="r")


def compress_gauged(T: Dict[int, np.ndarray], B: Dict[int, List[int]], dims: Dict[int, int], i: int, j: int,
                    chi: int, r: int, new_bond: int, allowed):
    """Compress the bonds shared by i and j in the tree gauge of distance r.

    Returns None when D_AB <= chi, else (A_new, bonds_i, B_new, bonds_j, k, gap, s_k / s_1).
    """
    ti, bi, tj, bj = T[i], B[i], T[j], B[j]
    sj, si = set(bj), set(bi)
    shared = [b for b in bi if b in sj]
    if _prod(dims[b] for b in shared) <= chi:
        return None
    ri = [b for b in bi if b not in sj]
    rj = [b for b in bj if b not in si]
    # virtual copies of the spanning tree, R factors pushed inwards
    tau = spanning_tree(B, dims, [i, j], r, allowed) if r > 0 else []
    vdims = dict(dims)
    vb = -1
    V: Dict[int, Tuple[np.ndarray, List[int]]] = {t: (T[t], list(B[t])) for t in {i, j} | {v for _, v in tau}}
    for u, v in reversed(tau):
        tv, bv = V[v]
        tu, bu = V[u]
        sh = [b for b in bv if b in set(bu)]
        rest = [b for b in bv if b not in sh]
        R = _reduce_rows(_matricize_d(tv, bv, rest, sh, vdims))
        vdims[vb] = R.shape[0]
        rest_u = [b for b in bu if b not in sh]
        umat = _matricize_d(tu, bu, sh, rest_u, vdims)
        newu = (R @ umat).reshape([R.shape[0]] + [vdims[b] for b in rest_u])
        V[u] = (newu, [vb] + rest_u)
        vb -= 1
    (ta, ba), (tb, bb) = V[i], V[j]
    R_A = _reduce_rows(_matricize_d(ta, ba, [b for b in ba if b not in set(shared)], shared, vdims))
    L_B = _reduce_rows(_matricize_d(tb, bb, [b for b in bb if b not in set(shared)], shared, vdims)).T
    u, s, vt = np.linalg.svd(R_A @ L_B, full_matrices=False)
    k = min(chi, len(s))
    keep = s[:k] > 1e-13 * s[0] if len(s) and s[0] > 0 else np.zeros(k, dtype=bool)
    isq = np.where(keep, 1.0 / np.sqrt(np.where(keep, s[:k], 1.0)), 0.0)
    P_L = L_B @ (vt[:k].T * isq[None, :])           # D_AB x k
    P_R = (u[:, :k] * isq[None, :]).T @ R_A          # k x D_AB
    a_new = _matricize(ti, bi, ri, shared) @ P_L      # the original A
    b_new = P_R @ _matricize(tj, bj, shared, rj)      # the original B
    if k < len(s) and s[0] > 0 and s[k - 1] > 1e-13 * s[0]:
        gap = float((s[k - 1] - s[k]) / s[0])
    else:
        gap = 1.0
    kept = float(s[k - 1] / s[0]) if len(s) and s[0] > 0 else 0.0

    def place(bonds, rem, mat, rem_first, shape_src, bonds_src):
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
        return np.ascontiguousarray(np.transpose(t, [cur.index(x) for x in out])), out

    ai, nbi = place(bi, ri, a_new, True, ti.shape, bi)
    bj2, nbj = place(bj, rj, b_new, False, tj.shape, bj)
    return ai, nbi, bj2, nbj, k, gap, kept


def _matricize_d(t: np.ndarray, bonds: List[int], rows: List[int], cols: List[int], dims) -> np.ndarray:
    perm = [bonds.index(b) for b in rows + cols]
    return np.transpose(t, perm).reshape(_prod(dims[b] for b in rows), _prod(dims[b] for b in cols))


def contract_gauged(net: Network, tree: Tree, chi: int, r: int, include_inputs: bool = False) -> Result:
    """Algorithm 1 over the explicit ops, every compression in the tree gauge of distance r.

    The result also carries min_kept: the smallest kept s_k / s_1 (the projector
    form divides by s_k^1/2, so rounding grows as it approaches zero).
    """
    if tree.n_inputs != net.n_tensors:
        raise ValueError("tree and network disagree on the number of tensors")
    T: Dict[int, np.ndarray] = {i: np.asarray(d, dtype=np.float64) for i, d in enumerate(net.data)}
    Bn: Dict[int, List[int]] = {i: list(b) for i, b in enumerate(net.bonds)}
    dims: Dict[int, int] = {b: int(d) for b, d in enumerate(net.bond_dims)}
    n_in = net.n_tensors
    allowed = (lambda t: True) if include_inputs else (lambda t: t >= n_in)
    E = 0
    nxt_bond = len(net.bond_dims)
    res = Result(0.0, 0)
    for op in tree.ops:
        if op[0] == "C":
            _, i, j, k = op
            c, bc = contract_pair(T.pop(i), Bn.pop(i), T.pop(j), Bn.pop(j))
            c, e = _rescale(c)
            E += e
            T[k], Bn[k] = c, bc
        else:
            _, i, j = op
            out = compress_gauged(T, Bn, dims, i, j, chi, r, nxt_bond, allowed)
            if out is None:
                continue
            ai, nbi, bj2, nbj, k, gap, kept = out
            res.min_kept = min(getattr(res, "min_kept", 1.0), kept)
            dims[nxt_bond] = k
            nxt_bond += 1
            ai, e1 = _rescale(ai)
            bj2, e2 = _rescale(bj2)
            E += e1 + e2
            T[i], Bn[i], T[j], Bn[j] = ai, nbi, bj2, nbj
            res.compressions += 1
            res.diag.append((k, 0.0, gap))
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
