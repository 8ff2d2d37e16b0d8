"""Oracle: reverse pass of the approximate contraction, d log|Z| / d T_v (FP64).

Test infrastructure only (see the package docstring).

The forward pass is oracle.approx's schedule (Algorithm 1 with explicit ops),
re-run here with every operand kept; the reverse pass walks the ops backwards.
The paper gives no adjoint; the steps below are the chain rule of each
forward step, written out.

  * C i j k  (C = A B on the matricized operands):  A_bar = C_bar B^T,
    B_bar = A^T C_bar, then un-matricized to each operand's bond order.
  * rescale X -> X 2^-e: e is piecewise constant in the inputs, so the
    adjoint of the unscaled X is 2^-e times that of the scaled one.
  * final log|Z| = ln|x| + E ln 2 with x the product of the remaining
    scalars: each scalar t gets 1 / t.
  * S i j with D_AB > chi: the Q-form factors equal, up to an orthogonal gauge
    on the new bond that the rest of the contraction does not see,
    A_bar = U_k s_k^1/2 and B_bar = s_k^1/2 V_k^T with U s V^T the SVD of
    X = A B (Eq. "svd": R_A L_B has the singular values of X, and Q_A U, Q_B V
    are X's singular vectors).  So the reverse step is the adjoint of a
    truncated SVD of X, taken with X's own SVD (not through the QR factors):
        U' = [A_bar' s_k^1/2, 0],  V' = [B_bar'^T s_k^1/2, 0],
        s'_i = (u_i . A_bar'_i + v_i . B_bar'^T_i) / (2 s_i^1/2)   (i < k),
        X' = U [ (F o (U^T U' - U'^T U)) S + diag(s') + S (F o (V^T V' - V'^T V)) ] V^T
             + (1 - U U^T) U' S^-1 V^T + U S^-1 V'^T (1 - V V^T),
    with F_ij = 1 / (s_j^2 - s_i^2) for i != j (the standard real-SVD adjoint),
    then A' = X' B^T and B' = A^T X'.

Readings where the paper is silent (it has no gradient):
  * F is Lorentzian-broadened: F_ij = d / (d^2 + eps), d = s_j^2 - s_i^2,
    eps = 1e-12 s_1^2, so exactly degenerate pairs contribute nothing.
  * s^-1/2 and s^-1 of a kept singular value at or below 1e-13 s_1 are taken
    as 0 (such columns of A_bar and B_bar are numerically zero and their
    derivative is singular).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Optional, Tuple

import numpy as np

from tn_inputs.formats import Network, Tree

EPS_REL = 1e-12     # Lorentzian broadening, relative to s_1^2
ZERO_REL = 1e-13    # kept singular values at or below this times s_1 get no inverse


@dataclass
class GradResult:
    logabs: float
    sign: int
    grads: List[np.ndarray]    # d log|Z| / d T_v, in each input's own bond order
    compressions: int = 0
    min_gap: float = 1.0       # smallest relative gap (s_k - s_{k+1}) / s_1 at a cut
    min_kept: float = 1.0      # smallest kept s_k / s_1 (near 0: a kept value is zero and
                               # the result is not differentiable there)


def _prod(dims) -> int:
    p = 1
    for d in dims:
        p *= int(d)
    return p


def _matricize(t, bonds, rows, cols):
    perm = [bonds.index(b) for b in rows + cols]
    shp = t.shape
    m = _prod(shp[p] for p in perm[: len(rows)])
    return np.transpose(t, perm).reshape(m, -1), perm


def _unmatricize(mat, shape, perm):
    """Inverse of _matricize: a (rows x cols) matrix back to the tensor's own axis order."""
    t = mat.reshape([shape[p] for p in perm])
    return np.transpose(t, np.argsort(perm))


def _rescale(x):
    m = float(np.max(np.abs(x))) if x.size else 0.0
    if m == 0.0 or not math.isfinite(m):
        return x, 0
    e = math.frexp(m)[1]
    return np.ldexp(x, -e), e


def svd_truncated_adjoint(u, s, vt, k, abar_bar, bbar_bar):
    """X' for (A_bar, B_bar) = (U_k s^1/2, s^1/2 V_k^T), X = u diag(s) vt (thin SVD).

    u: m x q, s: q (descending), vt: q x p; abar_bar: m x k, bbar_bar: k x p.
    """
    m, q = u.shape
    p = vt.shape[1]
    v = vt.T
    s1 = float(s[0]) if q else 0.0
    eps = EPS_REL * s1 * s1
    keep = s[:k] > ZERO_REL * s1
    isq = np.where(keep, 1.0 / np.sqrt(np.where(keep, s[:k], 1.0)), 0.0)    # s^-1/2 (0 if tiny)
    sq = np.sqrt(s[:k])
    ub = np.zeros((m, q))
    vb = np.zeros((p, q))
    ub[:, :k] = abar_bar * sq[None, :]
    vb[:, :k] = bbar_bar.T * sq[None, :]
    sb = np.zeros(q)
    sb[:k] = 0.5 * isq * (np.einsum("ij,ij->j", u[:, :k], abar_bar) + np.einsum("ij,ij->j", v[:, :k], bbar_bar.T))
    d = s[None, :] ** 2 - s[:, None] ** 2          # d_ij = s_j^2 - s_i^2
    F = d / (d * d + eps)
    np.fill_diagonal(F, 0.0)
    S = np.diag(s)
    J = F * (u.T @ ub - ub.T @ u)
    K = F * (v.T @ vb - vb.T @ v)
    core = J @ S + np.diag(sb) + S @ K
    xb = u @ core @ vt
    # complement terms; U' and V' vanish beyond column k, and S^-1 U'_i = U-bar-bar_i s_i^-1/2
    sinv_ub = abar_bar * isq[None, :]              # U'_k S_k^-1
    sinv_vb = bbar_bar.T * isq[None, :]            # V'_k S_k^-1
    xb += (sinv_ub - u @ (u.T @ sinv_ub)) @ vt[:k, :]
    xb += u[:, :k] @ (sinv_vb - v @ (v.T @ sinv_vb)).T
    return xb


def contract_with_grad(net: Network, tree: Tree, chi: Optional[int]) -> GradResult:
    """log|Z|, sign and d log|Z| / d T_v of the approximate contraction (Algorithm 1)."""
    if tree.n_inputs != net.n_tensors:
        raise ValueError("tree and network disagree on the number of tensors")
    T: Dict[int, np.ndarray] = {i: np.asarray(d, dtype=np.float64) for i, d in enumerate(net.data)}
    B: Dict[int, List[int]] = {i: list(b) for i, b in enumerate(net.bonds)}
    # each live tensor id -> the node of the computation that holds its current value
    node_of: Dict[int, int] = {i: i for i in T}
    tape = []            # forward records, in order
    n_nodes = net.n_tensors
    E = 0
    nxt_id = net.n_tensors
    nxt_bond = len(net.bond_dims)
    compressions = 0
    min_gap = 1.0
    min_kept = 1.0

    for op in tree.ops:
        if op[0] == "C":
            _, i, j, k = op
            ti, bi, tj, bj = T.pop(i), B.pop(i), T.pop(j), B.pop(j)
            sj, si = set(bj), set(bi)
            shared = [b for b in bi if b in sj]
            ri = [b for b in bi if b not in sj]
            rj = [b for b in bj if b not in si]
            a, pa = _matricize(ti, bi, ri, shared)
            b, pb = _matricize(tj, bj, shared, rj)
            c = a @ b
            dims = [ti.shape[bi.index(x)] for x in ri] + [tj.shape[bj.index(x)] for x in rj]
            c, e = _rescale(c.reshape(dims))
            E += e
            out = n_nodes
            n_nodes += 1
            tape.append(("C", node_of.pop(i), node_of.pop(j), out, a, b, pa, pb, ti.shape, tj.shape, e))
            T[k], B[k] = c, ri + rj
            node_of[k] = out
            nxt_id += 1
        elif op[0] == "S":
            _, i, j = op
            if chi is None:
                continue
            ti, bi, tj, bj = T[i], B[i], T[j], B[j]
            sj, si = set(bj), set(bi)
            shared = [b for b in bi if b in sj]
            if _prod(ti.shape[bi.index(b)] for b in shared) <= chi:
                continue
            ri = [b for b in bi if b not in sj]
            rj = [b for b in bj if b not in si]
            a, pa = _matricize(ti, bi, ri, shared)
            b, pb = _matricize(tj, bj, shared, rj)
            x = a @ b
            u, s, vt = np.linalg.svd(x, full_matrices=False)
            kk = min(chi, len(s), a.shape[0], b.shape[1], a.shape[1])
            if kk < len(s) and s[0] > 0 and s[kk - 1] > ZERO_REL * s[0]:
                min_gap = min(min_gap, float((s[kk - 1] - s[kk]) / s[0]))
            if s[0] > 0:
                min_kept = min(min_kept, float(s[kk - 1] / s[0]))
            sq = np.sqrt(s[:kk])
            abar = u[:, :kk] * sq[None, :]
            bbar = sq[:, None] * vt[:kk, :]
            new = nxt_bond
            nxt_bond += 1
            # new bond where each tensor's first shared bond was
            nbi, nbj = [], []
            for xb_, lst, src in ((bi, nbi, si), (bj, nbj, sj)):
                placed = False
                for y in xb_:
                    if y in sj and y in si:
                        if not placed:
                            lst.append(new)
                            placed = True
                    else:
                        lst.append(y)
            dims_i = [ti.shape[bi.index(y)] for y in ri]
            dims_j = [tj.shape[bj.index(y)] for y in rj]
            cur_i = ri + [new]
            cur_j = [new] + rj
            perm_i = [cur_i.index(y) for y in nbi]
            perm_j = [cur_j.index(y) for y in nbj]
            ai = np.transpose(abar.reshape(dims_i + [kk]), perm_i)
            bj2 = np.transpose(bbar.reshape([kk] + dims_j), perm_j)
            ai, e1 = _rescale(np.ascontiguousarray(ai))
            bj2, e2 = _rescale(np.ascontiguousarray(bj2))
            E += e1 + e2
            out_i, out_j = n_nodes, n_nodes + 1
            n_nodes += 2
            tape.append(("S", node_of[i], node_of[j], out_i, out_j, a, b, pa, pb, ti.shape, tj.shape,
                         u, s, vt, kk, dims_i, dims_j, perm_i, perm_j, e1, e2))
            T[i], B[i], T[j], B[j] = ai, nbi, bj2, nbj
            node_of[i], node_of[j] = out_i, out_j
            compressions += 1
        else:
            raise ValueError(f"unknown op {op!r}")

    xs = []
    for t in T.values():
        if t.size != 1:
            raise ValueError("tree leaves a tensor with open bonds")
        xs.append(float(t.reshape(())))
    x = float(np.prod(xs))
    if x == 0.0:
        raise ValueError("Z = 0: log|Z| has no gradient")
    logabs = math.log(abs(x)) + E * math.log(2.0)
    sign = 1 if x > 0 else -1

    # reverse pass: adjoint of every node's (scaled) value
    adj: Dict[int, np.ndarray] = {}
    for tid, t in T.items():
        adj[node_of[tid]] = np.full(t.shape, 1.0 / float(t.reshape(())))
    for rec in reversed(tape):
        if rec[0] == "C":
            _, ni, nj, out, a, b, pa, pb, shi, shj, e = rec
            cb = np.ldexp(adj.pop(out), -e).reshape(a.shape[0], b.shape[1])
            adj[ni] = _unmatricize(cb @ b.T, shi, pa)
            adj[nj] = _unmatricize(a.T @ cb, shj, pb)
        else:
            (_, ni, nj, out_i, out_j, a, b, pa, pb, shi, shj, u, s, vt, kk,
             dims_i, dims_j, perm_i, perm_j, e1, e2) = rec
            gi = np.ldexp(adj.pop(out_i), -e1)
            gj = np.ldexp(adj.pop(out_j), -e2)
            abar_bar = np.transpose(gi, np.argsort(perm_i)).reshape(a.shape[0], kk)
            bbar_bar = np.transpose(gj, np.argsort(perm_j)).reshape(kk, b.shape[1])
            xb = svd_truncated_adjoint(u, s, vt, kk, abar_bar, bbar_bar)
            adj[ni] = _unmatricize(xb @ b.T, shi, pa)
            adj[nj] = _unmatricize(a.T @ xb, shj, pb)
    grads = [adj[v] for v in range(net.n_tensors)]
    return GradResult(logabs, sign, grads, compressions, min_gap, min_kept)
