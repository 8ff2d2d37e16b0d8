"""CPU emulation of the library's static schedule (host-logic test, not an oracle).

`tn_plan_describe` exports the schedule the GPU executor runs: every step with
its kind, sizes and buffer views.  This module replays those steps in numpy on
a flat arena laid out exactly as the executor lays it out (arena buffers at
offset * batch + instance * stride, inputs and input adjoints in the input
block), with plain numpy stand-ins for each kernel: matrix products, a
Householder QR with the executor's reflector convention, an SVD from LAPACK in
place of Jacobi (any exact SVD is a fixed point of the Jacobi kernels), and the
selection, absorb, log-norm and reverse-pass steps.  Comparing its results
with the oracle checks the planner -- views, strides, orientations, arena
reuse, the reverse-pass emission -- without a GPU.  The mixed-precision GEMM
steps are emulated in FP64, so every form's schedule is checked at FP64
accuracy.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

BUF_ARENA, BUF_INPUT, BUF_GIN = 0, 1, 2
(ST_PERMUTE, ST_GEMM, ST_QR, ST_JACOBI, ST_SELECT, ST_RESCALE, ST_FINAL, ST_TO_F32, ST_JACOBI32, ST_TO_F64,
 ST_COPY, ST_APPLYQ, ST_GEMM_TC, ST_SCALE_POW2, ST_FINAL_GRAD, ST_SVD_FACTORS, ST_SVD_ADJ_CORE,
 ST_COPY2D, ST_MARK_ACTIVE) = range(19)


class Emulator:
    def __init__(self, plan: dict, nets: Sequence):
        self.p = plan
        self.B = len(nets)
        self.arena_bytes = np.zeros(max(plan["arena_units"], 1) * self.B * 8, dtype=np.uint8)
        self.arena = self.arena_bytes.view(np.float64)
        self.arena32 = self.arena_bytes.view(np.float32)
        nt = plan["in_total"]
        self.inbuf = np.zeros(max(nt, 1) * self.B)
        self.ginbuf = np.zeros(max(nt, 1) * self.B)
        self.etape = np.zeros(max(plan["n_slots"], 1) * self.B, dtype=np.int64)
        self.expo = np.zeros(self.B, dtype=np.int64)
        self.status = np.zeros(self.B, dtype=np.int64)
        self.logabs = np.zeros(self.B)
        self.sign = np.zeros(self.B, dtype=np.int64)
        for b, net in enumerate(nets):
            for t, d in enumerate(net.data):
                a = np.ascontiguousarray(d, dtype=np.float64).ravel()
                o = b * nt + plan["in_off"][t]
                self.inbuf[o:o + a.size] = a

    # a view -> (array, element index of instance 0)
    def base(self, v):
        buf, off, rs, cs, bs, eo = v
        if buf == BUF_INPUT:
            return self.inbuf, off + eo
        if buf == BUF_GIN:
            return self.ginbuf, off + eo
        return self.arena, off * self.B + eo

    def idx(self, v, b, rows, cols):
        arr, base = self.base(v)
        _, _, rs, cs, bs, _ = v
        r = np.arange(rows)[:, None]
        c = np.arange(cols)[None, :]
        return arr, base + b * bs + r * rs + c * cs

    def get(self, v, b, rows, cols):
        arr, ix = self.idx(v, b, rows, cols)
        return arr[ix].copy()

    def put(self, v, b, rows, cols, val):
        arr, ix = self.idx(v, b, rows, cols)
        arr[ix] = val

    def colmajor(self, v, b, ld, cols, rows=None):
        """A column-major block (ld rows per column) at a raw view pointer, as (array, index)."""
        arr, base = self.base(v)
        rows = ld if rows is None else rows
        r = np.arange(rows)[:, None]
        c = np.arange(cols)[None, :]
        return arr, base + b * v[4] + r + c * ld

    def f32(self, v, b, fbs, count):
        arr, base = self.base(v)
        assert arr is self.arena
        start = 2 * base + b * fbs
        return start, start + count

    def run(self):
        for st in self.p["steps"]:
            getattr(self, "k%d" % st["kind"])(st)
        return self

    # ---- forward steps
    def k0(self, st):  # permute: output axis a is input axis perm[a]
        dims = st["in_dims"]
        size = int(np.prod(dims, dtype=np.int64)) if dims else 1
        sa, sb = self.base(st["src"])
        da, db = self.base(st["dst"])
        for b in range(self.B):
            x = sa[sb + b * st["src"][4]: sb + b * st["src"][4] + size].reshape(dims)
            da[db + b * st["dst"][4]: db + b * st["dst"][4] + size] = np.transpose(x, st["perm"]).ravel()

    def k1(self, st):  # C = alpha A B + beta C
        m, n, k = st["m"], st["n"], st["k"]
        for b in range(self.B):
            c = st["alpha"] * (self.get(st["A"], b, m, k) @ self.get(st["B"], b, k, n))
            if st["beta"] != 0.0:
                c = c + st["beta"] * self.get(st["C"], b, m, n)
            self.put(st["C"], b, m, n, c)

    def k12(self, st):  # tensor-core GEMM, emulated in FP64
        m, n, k = st["m"], st["n"], st["k"]
        for b in range(self.B):
            self.put(st["C"], b, m, n, self.get(st["A"], b, m, k) @ self.get(st["B"], b, k, n))

    def k2(self, st):  # Householder QR: reflectors (v_j = 1 implicit) in work, taus after the batch
        m, n = st["m"], st["n"]
        r = min(m, n)
        warr, wbase = self.base(st["work"])
        wbs = st["work"][4]
        for b in range(self.B):
            a = self.get(st["A"], b, m, n)
            taus = np.zeros(n)
            for j in range(r):
                x = a[j:, j].copy()
                alpha = x[0]
                xn = np.linalg.norm(x[1:])
                if xn == 0.0:
                    tau, beta, v = 0.0, alpha, np.zeros_like(x)
                else:
                    beta = -math.copysign(math.hypot(alpha, xn), alpha)
                    tau = (beta - alpha) / beta
                    v = x / (alpha - beta)
                v[0] = 1.0
                if tau != 0.0:
                    a[j:, j:] -= tau * np.outer(v, v @ a[j:, j:])
                a[j, j] = beta
                a[j + 1:, j] = v[1:]
                taus[j] = tau
            # work column-major m x n, then the reflectors' rows below the diagonal are what apply_q reads
            w = np.asfortranarray(a).ravel(order="F")
            warr[wbase + b * wbs: wbase + b * wbs + m * n] = w
            warr[wbase + self.B * wbs + b * n: wbase + self.B * wbs + b * n + n] = taus
            R = np.triu(a[:r, :])
            self.put(st["C"], b, r, n, R)

    def _reflectors(self, st, b, m, n):
        warr, wbase = self.base(st["work"])
        wbs = st["work"][4]
        W = warr[wbase + b * wbs: wbase + b * wbs + m * n].reshape((m, n), order="F")
        taus = warr[wbase + self.B * wbs + b * n: wbase + self.B * wbs + b * n + n]
        return W, taus

    def k11(self, st):  # X <- Q X (flag: Q^T X), X m x k column-major at C
        m, n, k = st["m"], st["n"], st["k"]
        r = min(m, n)
        for b in range(self.B):
            W, taus = self._reflectors(st, b, m, n)
            arr, ix = self.colmajor(st["C"], b, m, k)
            X = arr[ix].copy()
            order = range(r) if st["flag"] else range(r - 1, -1, -1)
            for j in order:
                if taus[j] == 0.0:
                    continue
                v = np.zeros(m)
                v[j] = 1.0
                v[j + 1:] = W[j + 1:, j]
                X -= taus[j] * np.outer(v, v @ X)
            arr[ix] = X

    def k3(self, st):  # FP64 Jacobi: G <- G W, V <- V W (W orthogonal, G W orthogonal columns); sig = norms
        m, n = st["m"], st["n"]
        for b in range(self.B):
            arr, ix = self.colmajor(st["C"], b, m, n)
            G = arr[ix].copy()
            _, _, wt = np.linalg.svd(G, full_matrices=True)
            W = wt.T
            G2 = G @ W
            arr[ix] = G2
            if not st["no_v"]:
                varr, vix = self.colmajor(st["aux1"], b, n, n)
                V = np.eye(n) if st["init_v"] else varr[vix].copy()
                varr[vix] = V @ W
            sarr, six = self.colmajor(st["aux2"], b, n, 1)
            sarr[six] = np.linalg.norm(G2, axis=0)[:, None]

    def k18(self, st):  # active columns of the FP64 polish
        # Nothing to replay: they only decide when the polish's sweep loop may
        # stop, and the emulated polish (k3) is an exact SVD of the core.
        pass

    def k7(self, st):  # FP64 -> FP32
        n = st["count"]
        sarr, sbase = self.base(st["src"])
        for b in range(self.B):
            x = sarr[sbase + b * st["src"][4]: sbase + b * st["src"][4] + n]
            s0, s1 = self.f32(st["dst"], b, st["fbs_dst"], n)
            self.arena32[s0:s1] = x.astype(np.float32)

    def k8(self, st):  # FP32 Jacobi preconditioner, V = I first
        m, n = st["m"], st["n"]
        for b in range(self.B):
            g0, g1 = self.f32(st["C"], b, st["fbs_src"], m * n)
            G = self.arena32[g0:g1].astype(np.float64).reshape((m, n), order="F")
            _, _, wt = np.linalg.svd(G, full_matrices=True)
            W = wt.T
            self.arena32[g0:g1] = (G @ W).ravel(order="F").astype(np.float32)
            v0, v1 = self.f32(st["aux1"], b, st["fbs_dst"], n * n)
            self.arena32[v0:v1] = W.ravel(order="F").astype(np.float32)

    def k9(self, st):  # FP32 -> FP64 into dst and out1
        n = st["count"]
        for b in range(self.B):
            s0, s1 = self.f32(st["src"], b, st["fbs_src"], n)
            x = self.arena32[s0:s1].astype(np.float64)
            for v in (st["dst"], st["out1"]):
                arr, base = self.base(v)
                arr[base + b * st["dst"][4]: base + b * st["dst"][4] + n] = x

    def k10(self, st):  # block copy of the whole batch
        sa, sb = self.base(st["src"])
        da, db = self.base(st["dst"])
        size = st["dst"][4] * self.B
        da[db:db + size] = sa[sb:sb + size]

    def k4(self, st):  # select the k largest sigma; factors with sigma^1/2 absorbed
        m, n, k = st["m"], st["n"], st["k"]
        ldl, ldr = st["count"], st["init_v"]
        for b in range(self.B):
            garr, gix = self.colmajor(st["C"], b, m, n)
            G = garr[gix]
            sarr, six = self.colmajor(st["aux2"], b, n, 1)
            sig = sarr[six][:, 0]
            order = sorted(range(n), key=lambda i: (-sig[i], i))
            smax = max(sig.max(), 0.0)
            larr, lix = self.colmajor(st["out1"], b, ldl, k)
            rarr, rix = self.colmajor(st["out2"], b, ldr, k)
            L = np.zeros((ldl, k))
            R = rarr[rix].copy()
            if st["no_v"]:
                karr, kix = self.colmajor(st["work"], b, m, k)
                K3 = np.zeros((m, k))
            else:
                varr, vix = self.colmajor(st["aux1"], b, n, n)
                V = varr[vix]
            for p in range(k):
                i = order[p]
                si = sig[i]
                rs = math.sqrt(si)
                if not st["no_v"]:
                    L[:m, p] = G[:, i] * (1.0 / rs if si > 0.0 else 0.0)
                    R[:, p] = 0.0
                    R[:n, p] = V[:, i] * rs
                else:
                    keep = si > 1e-13 * smax and si > 0.0
                    L[:m, p] = G[:, i] * (1.0 / rs if keep else 0.0)
                    K3[:, p] = G[:, i] * (1.0 / (si * rs) if keep else 0.0)
                    R[n:, p] = 0.0
            larr[lix] = L
            rarr[rix] = R
            if st["no_v"]:
                karr[kix] = K3

    def k5(self, st):  # rescale by 2^-e, e the exponent of max |X|
        n = st["count"]
        arr, base = self.base(st["C"])
        for b in range(self.B):
            x = arr[base + b * st["C"][4]: base + b * st["C"][4] + n]
            mx = float(np.max(np.abs(x))) if n else 0.0
            e = 0
            if not math.isfinite(mx):
                self.status[b] = -7
            elif mx != 0.0:
                e = math.frexp(mx)[1]
                x *= 2.0 ** (-e)
                self.expo[b] += e
            if st["slot"] >= 0:
                self.etape[st["slot"] * self.B + b] = e

    def k6(self, st):
        arr, base = self.base(st["C"])
        for b in range(self.B):
            v = arr[base + b * st["C"][4]]
            if v == 0.0:
                self.logabs[b], self.sign[b] = -math.inf, 0
            else:
                self.logabs[b] = math.log(abs(v)) + self.expo[b] * math.log(2.0)
                self.sign[b] = 1 if v > 0 else -1

    # ---- reverse-pass steps
    def k13(self, st):
        n = st["count"]
        arr, base = self.base(st["C"])
        for b in range(self.B):
            e = int(self.etape[st["slot"] * self.B + b])
            arr[base + b * st["C"][4]: base + b * st["C"][4] + n] *= 2.0 ** (-e)

    def k14(self, st):
        xa, xb = self.base(st["C"])
        ga, gb = self.base(st["out1"])
        for b in range(self.B):
            ga[gb + b * st["out1"][4]] = 1.0 / xa[xb + b * st["C"][4]]

    def k15(self, st):  # sorted factors of a Jacobi SVD
        m, n, k, tall = st["m"], st["n"], st["k"], st["flag"]
        ru, rw = (m, n) if tall else (n, m)
        for b in range(self.B):
            garr, gix = self.colmajor(st["C"], b, m, n)
            G = garr[gix]
            varr, vix = self.colmajor(st["aux1"], b, n, n)
            V = varr[vix]
            sarr, six = self.colmajor(st["aux2"], b, n, 1)
            sig = sarr[six][:, 0]
            smax = sig.max()
            order = sorted(range(n), key=lambda i: (-sig[i], i))
            U = np.zeros((ru, n))
            Wm = np.zeros((rw, n))
            s = np.zeros(n)
            Us = np.zeros((ru, k))
            Ws = np.zeros((rw, k))
            for p, i in enumerate(order):
                nz = sig[i] > 1e-13 * smax and sig[i] > 0.0
                g = G[:, i] * (1.0 / sig[i] if nz else 0.0)
                v = V[:, i]
                u_col, w_col = (g, v) if tall else (v, g)
                U[:, p] = u_col
                Wm[:, p] = w_col
                s[p] = sig[i]
                if p < k:
                    isq = 1.0 / math.sqrt(sig[i]) if nz else 0.0
                    Us[:, p] = u_col * isq
                    Ws[:, p] = w_col * isq
            for v_, mat, ld in ((st["out1"], U, ru), (st["out2"], Wm, rw), (st["A"], Us, ru), (st["B"], Ws, rw)):
                arr, ix = self.colmajor(v_, b, ld, mat.shape[1])
                arr[ix] = mat
            arr, ix = self.colmajor(st["work"], b, n, 1)
            arr[ix] = s[:, None]

    def k16(self, st):  # core matrix of the truncated-SVD adjoint
        q, k = st["n"], st["k"]
        for b in range(self.B):
            parr, pix = self.colmajor(st["A"], b, q, k)
            P = parr[pix]
            qarr, qix = self.colmajor(st["B"], b, q, k)
            Q = qarr[qix]
            sarr, six = self.colmajor(st["work"], b, q, 1)
            s = sarr[six][:, 0]
            s0 = s[0]
            C = np.zeros((q, q))
            sq = np.sqrt(s)
            a = np.zeros((q, q))
            bb = np.zeros((q, q))
            a[:, :k] = P * sq[None, :k]
            bb[:, :k] = Q * sq[None, :k]
            d = s[None, :] ** 2 - s[:, None] ** 2
            F = d / (d * d + 1e-12 * s0 * s0)
            np.fill_diagonal(F, 0.0)
            C = F * (a - a.T) * s[None, :] + s[:, None] * F * (bb - bb.T)
            for i in range(k):
                isq = 1.0 / math.sqrt(s[i]) if (s[i] > 1e-13 * s0 and s[i] > 0.0) else 0.0
                C[i, i] = 0.5 * isq * (P[i, i] + Q[i, i])
            arr, ix = self.colmajor(st["C"], b, q, q)
            arr[ix] = C

    def k17(self, st):
        m, n = st["m"], st["n"]
        for b in range(self.B):
            self.put(st["C"], b, m, n, self.get(st["A"], b, m, n))

    # ---- results
    def grads(self, b: int, shapes: List[tuple]) -> List[np.ndarray]:
        nt = self.p["in_total"]
        out = []
        for t, shp in enumerate(shapes):
            size = int(np.prod(shp, dtype=np.int64)) if shp else 1
            o = b * nt + self.p["in_off"][t]
            out.append(self.ginbuf[o:o + size].reshape(shp).copy())
        return out
