"""Op-by-op parity at full size: the GPU's inputs to each op go through the oracle's step.

For a batch already loaded in a context, walk whole rows of a boundary-row tree
(Algorithm 1 with explicit ops): for every op, fetch the GPU's input tensors
(state after the previous op) and its outputs (state after the op) with
tn_debug_tensor, run the oracle's own step (contract_pair, compress_pair) on
those inputs, and compare -- elementwise for a contraction, through the
gauge-free product A_bar B_bar for a compression (the new bond's gauge is not
unique).  Both sides carry power-of-two scales, so results are compared after
normalisation.  Consecutive debug calls continue from the previous stop, so a
walk costs about one pass of the schedule.
"""
from __future__ import annotations

import numpy as np

from oracle import approx


def bond_order_array(t, bonds, order):
    return np.transpose(t, [bonds.index(b) for b in order])


def pair_product(ta, ba, tb, bb, new_bond):
    """Contract two tensors over `new_bond`; remaining axes sorted by bond id (gauge-free)."""
    ia, ib = ba.index(new_bond), bb.index(new_bond)
    p = np.tensordot(ta, tb, axes=([ia], [ib]))
    rest = [b for b in ba if b != new_bond] + [b for b in bb if b != new_bond]
    return bond_order_array(p, rest, sorted(rest))


def unit(x):
    return x / np.linalg.norm(x)


def row_ops(lx, y):
    """Op indices of boundary row y (1-based) in trees.boundary_rows(lx, ly)."""
    base = (y - 1) * (2 * lx - 1)
    return list(range(base, base + 2 * lx - 1))


def walk(ctx, ids, tree, chi, ops, whiches, tol_c=1e-12, tol_s=1e-10, min_gap=1e-8):
    """Compare every op in `ops` (increasing) for instances ids[w], w in whiches.

    Returns a summary dict: ops checked, S ops that did not fire (shared bond
    size <= chi, as Algorithm 1 skips them), compressions skipped as ambiguous
    (relative cut gap below min_gap, where several truncations are correct),
    and the largest deviations seen.  A compression whose cut gap g is small
    but above min_gap is allowed a deviation of 1e-15 / g when that exceeds
    tol_s: the kept subspace itself is only determined to about that.
    """
    out = {"c_ops": 0, "s_ops": 0, "ambiguous": 0, "noop": 0, "max_c": 0.0, "max_s": 0.0}
    for r in ops:
        op = tree.ops[r]
        # every instance's inputs first (state after op r - 1), then the outputs:
        # the stops never go backwards, so each debug call continues the last one
        inputs = {w: (ctx.debug_tensor(ids, w, chi, r - 1, op[1]), ctx.debug_tensor(ids, w, chi, r - 1, op[2]))
                  for w in whiches}
        for w in whiches:
            (ti, bi), (tj, bj) = inputs[w]
            if op[0] == "C":
                tk, bk = ctx.debug_tensor(ids, w, chi, r, op[3])
                want, bw = approx.contract_pair(ti, bi, tj, bj)
                got = bond_order_array(tk, bk, bw)
                d = float(np.linalg.norm(unit(got) - unit(want)))
                out["max_c"] = max(out["max_c"], d)
                out["c_ops"] += 1
                assert d < tol_c, (r, w, d)
            else:
                ai, bai = ctx.debug_tensor(ids, w, chi, r, op[1])
                aj, baj = ctx.debug_tensor(ids, w, chi, r, op[2])
                new = [b for b in bai if b not in bi]
                if not new:          # D_AB <= chi: the op did not compress
                    out["noop"] += 1
                    continue
                res = approx.compress_pair(ti, bi, tj, bj, chi, new[0])
                assert res is not None
                if res[6] <= min_gap:
                    out["ambiguous"] += 1
                    continue
                want = pair_product(res[0], res[1], res[2], res[3], new[0])
                got = pair_product(ai, bai, aj, baj, new[0])
                assert got.shape == want.shape
                d = float(np.linalg.norm(unit(got) - unit(want)))
                out["max_s"] = max(out["max_s"], d)
                out["s_ops"] += 1
                # the kept subspace is determined to about (rounding) / (relative gap at the cut)
                assert d < max(tol_s, 1e-15 / res[6]), (r, w, d, res[6])
    return out
