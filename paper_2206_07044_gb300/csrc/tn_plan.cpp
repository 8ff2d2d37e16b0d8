// Schedule expansion: tree file + network structure + chi -> static steps.
//
// Semantics (Algorithm 1 with explicit ops; Sec. "Bond compression strategies"):
//   C i j k  contracts all bonds shared by i and j; k's bonds are i's remaining
//            bonds then j's remaining bonds.
//   S i j    runs iff D_AB = prod(shared sizes) > chi; the shared bonds become one
//            bond of size k = min(chi, D_A, D_B).
// Physical layouts of intermediates are free (log Z does not depend on them),
// so the planner tracks each tensor's storage order and hands row- or
// column-major views to the GEMM / QR kernels instead of permuting; a permute
// is issued only when the shared bonds are not contiguous at one end.
//
// A compression follows Eq. "svd" in its Q-form: R_A from a Householder QR
// of A and L_B from one of B^T, the SVD R_A L_B = U s V^T, then
// A_bar = Q_A U_k s^1/2 and B_bar = s^1/2 V_k^T Q_B with the Householder
// products applied to the zero-padded factors (Q is never formed).  The
// projector form of the SI (A P_L with P_L = L_B V_k s^-1/2) is the same
// matrix in exact arithmetic but multiplies rounding by |A||B|/|AB|, which is
// large when the entries cancel.  When D_A <= D_AB the QR of A is skipped
// (R_A = A, i.e. Q_A = 1); likewise for B.
#include "tn_plan.h"

#include "tn_kernels.h"

#include <algorithm>
#include <functional>
#include <map>
#include <set>
#include <unordered_map>
#include <unordered_set>

namespace tnp {
namespace {

constexpr int64_t kAlign = 32;  // doubles: keeps every per-instance block 256-byte aligned

int64_t round_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

class Arena {
 public:
  int64_t alloc(int64_t size) {
    size = round_up(std::max<int64_t>(size, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= size) {
        int64_t off = it->first, rest = it->second - size;
        free_.erase(it);
        if (rest) free_[off + size] = rest;
        return off;
      }
    }
    int64_t off = top_;
    top_ += size;
    peak_ = std::max(peak_, top_);
    return off;
  }
  void release(int64_t off, int64_t size) {
    size = round_up(std::max<int64_t>(size, 1));
    auto it = free_.emplace(off, size).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
        it = pv;
      }
    }
    if (it->first + it->second == top_) {
      top_ = it->first;
      free_.erase(it);
    }
  }
  int64_t peak() const { return peak_; }

 private:
  std::map<int64_t, int64_t> free_;
  int64_t top_ = 0, peak_ = 0;
};

struct Value {
  std::vector<int> bonds;   // storage order
  int64_t size = 1;
  int buf = BUF_ARENA;
  int64_t off = 0;
  int64_t bs = 0;
};

int64_t prod_dims(const std::vector<int>& bl, const std::vector<int64_t>& dim) {
  int64_t p = 1;
  for (int b : bl) p *= dim[b];
  return p;
}

// 0: bonds == X + Y; 1: bonds == Y + X; -1: neither.
int layout_of(const std::vector<int>& bonds, const std::vector<int>& X, const std::vector<int>& Y) {
  if (bonds.size() != X.size() + Y.size()) return -1;
  bool xy = std::equal(X.begin(), X.end(), bonds.begin()) &&
            std::equal(Y.begin(), Y.end(), bonds.begin() + X.size());
  if (xy) return 0;
  bool yx = std::equal(Y.begin(), Y.end(), bonds.begin()) &&
            std::equal(X.begin(), X.end(), bonds.begin() + Y.size());
  return yx ? 1 : -1;
}

double qr_flops(double m, double n) {
  double M = std::max(m, n), r = std::min(m, n);
  return 2.0 * M * r * r - 2.0 / 3.0 * r * r * r;
}
double svd_flops(double m, double n) {
  double M = std::max(m, n), r = std::min(m, n);
  return 4.0 * M * r * r - 4.0 / 3.0 * r * r * r;
}

struct Builder {
  const Structure& s;
  int chi;
  Plan* plan;
  Arena arena;
  std::vector<Value> vals;
  std::unordered_map<int, int> cur;  // tensor id -> value index
  std::vector<int64_t> dim;          // bond sizes (grows with new bonds)
  int op_index = -1;
  // reverse pass: the forward keeps every value (keep), each forward op pushes
  // a closure that emits its reverse steps, run in reverse order at the end
  bool grad = false;
  bool keep = false;
  bool in_bwd = false;
  bool keep_v = false;   // gradient plans: the FP64 Jacobi keeps V (in every pass, so all passes agree)
  std::vector<std::pair<int64_t, int64_t>>* rec_alloc = nullptr;  // records allocations (segment tapes)
  std::vector<std::function<void()>> bwd;
  std::unordered_map<int, PView> gv;  // value index -> buffer of its adjoint

  void rel(int64_t off, int64_t size) {
    if (!keep) arena.release(off, size);
  }

  PView base_view(const Value& v) const {
    PView p;
    p.buf = v.buf;
    p.off = v.off;
    p.bs = v.bs;
    return p;
  }
  int new_arena_value(std::vector<int> bonds) {
    Value v;
    v.bonds = std::move(bonds);
    v.size = prod_dims(v.bonds, dim);
    v.buf = BUF_ARENA;
    v.off = arena.alloc(v.size);
    if (rec_alloc) rec_alloc->push_back({v.off, v.size});
    v.bs = round_up(std::max<int64_t>(v.size, 1));
    vals.push_back(v);
    return (int)vals.size() - 1;
  }
  PView temp(int64_t size, int64_t* off_out) {
    PView p;
    p.buf = BUF_ARENA;
    p.off = arena.alloc(size);
    if (rec_alloc) rec_alloc->push_back({p.off, size});
    p.bs = round_up(std::max<int64_t>(size, 1));
    *off_out = p.off;
    return p;
  }
  void record(int tensor_id, int vi) {
    TensorRec r;
    r.op_index = op_index;
    r.tensor_id = tensor_id;
    r.view = base_view(vals[vi]);
    r.bonds = vals[vi].bonds;
    for (int b : r.bonds) r.dims.push_back(dim[b]);
    plan->records.push_back(std::move(r));
  }
  void release_value(int vi) {
    Value& v = vals[vi];
    if (v.buf == BUF_ARENA) rel(v.off, v.size);
  }
  void add(Step st) {
    st.op_index = op_index;
    plan->steps.push_back(std::move(st));
  }
  // permute value v into a new arena value whose storage order is `order`
  int permute_to(int vi, const std::vector<int>& order) {
    const Value src = vals[vi];
    int out = new_arena_value(order);
    Step st;
    st.kind = ST_PERMUTE;
    st.src = base_view(src);
    st.dst = base_view(vals[out]);
    for (int b : src.bonds) st.in_dims.push_back(dim[b]);
    for (int b : order)
      st.perm.push_back((int)(std::find(src.bonds.begin(), src.bonds.end(), b) - src.bonds.begin()));
    st.count = src.size;
    st.bytes = 16.0 * (double)src.size;
    plan->permute_bytes += st.bytes;
    add(st);
    return out;
  }
  // overhead: a GEMM of the SVD's preconditioning (not counted as algorithmic work)
  void gemm(int m, int n, int k, PView A, PView B, PView C, double alpha = 1.0, double beta = 0.0,
            bool overhead = false) {
    Step st;
    st.kind = ST_GEMM;
    st.m = m;
    st.n = n;
    st.k = k;
    st.A = A;
    st.B = B;
    st.C = C;
    st.alpha = alpha;
    st.beta = beta;
    st.flops = overhead ? 0.0 : 2.0 * m * n * (double)k;
    st.bytes = 8.0 * ((double)m * k + (double)k * n + (double)m * n);
    if (in_bwd) {
      plan->bwd_flops += 2.0 * m * n * (double)k;
      st.flops = 0.0;
    }
    plan->gemm_flops += st.flops;
    add(st);
  }
  bool mixed() const { return plan->prec != 0; }
  int tc_mode() const { return plan->prec == 1 ? 0 : (plan->prec == 2 ? 1 : 2); }
  // C = A B on the tensor cores; the staged-operand scratch is a temporary
  void gemm_tc_step(int m, int n, int k, PView A, PView B, PView C, bool count_flops) {
    Step st;
    st.kind = ST_GEMM_TC;
    st.tc_mode = tc_mode();
    st.m = m;
    st.n = n;
    st.k = k;
    st.A = A;
    st.B = B;
    st.C = C;
    // per-instance share of the batch's staged operands (+ slack for the 256-byte roundings)
    const int64_t per = (int64_t)tnk::gemm_tc_workspace_bytes(m, n, k, st.tc_mode, 1) + 1024;
    int64_t off;
    st.work = temp((per + 7) / 8, &off);
    st.flops = count_flops ? 2.0 * m * n * (double)k : 0.0;
    st.bytes = 8.0 * ((double)m * k + (double)k * n + (double)m * n);
    if (in_bwd) {
      plan->bwd_flops += 2.0 * m * n * (double)k;
      st.flops = 0.0;
    }
    plan->gemm_flops += st.flops;
    add(st);
    rel(off, (per + 7) / 8);
  }
  // returns the exponent-tape slot (reverse-pass plans) or -1
  int rescale(int vi) {
    Step st;
    st.kind = ST_RESCALE;
    st.C = base_view(vals[vi]);
    st.count = vals[vi].size;
    st.bytes = 24.0 * (double)vals[vi].size;
    if (grad) st.slot = plan->n_slots++;
    add(st);
    return st.slot;
  }

  // ---- reverse-pass helpers
  // Adjoint buffer of value vi (same layout as the value); inputs map to BUF_GIN.
  PView gview(int vi) {
    auto it = gv.find(vi);
    if (it != gv.end()) return it->second;
    const Value& v = vals[vi];
    PView p;
    if (v.buf == BUF_INPUT) {
      p.buf = BUF_GIN;
      p.off = v.off;
      p.bs = v.bs;
    } else {
      int64_t off;
      p = temp(v.size, &off);
    }
    gv[vi] = p;
    return p;
  }
  void gfree(int vi) {
    auto it = gv.find(vi);
    if (it == gv.end()) return;
    if (it->second.buf == BUF_ARENA) arena.release(it->second.off, vals[vi].size);
    gv.erase(it);
  }
  void scale_pow2(const PView& g, int64_t count, int slot) {
    Step st;
    st.kind = ST_SCALE_POW2;
    st.C = g;
    st.count = count;
    st.slot = slot;
    st.bytes = 16.0 * (double)count;
    add(st);
  }
  // adjoint of `tmp = permute(orig)`: orig' = inverse permutation of tmp'
  void permute_back(int tmp, int orig) {
    Step st;
    st.kind = ST_PERMUTE;
    st.src = gview(tmp);
    st.dst = gview(orig);
    const std::vector<int>& tb = vals[tmp].bonds;
    for (int b : tb) st.in_dims.push_back(dim[b]);
    for (int b : vals[orig].bonds) st.perm.push_back((int)(std::find(tb.begin(), tb.end(), b) - tb.begin()));
    st.count = vals[tmp].size;
    st.bytes = 16.0 * (double)st.count;
    add(st);
  }
  // C = A B in the plan's form (tensor cores in the mixed forms)
  void gemm_form(int m, int n, int k, PView A, PView B, PView C) {
    if (mixed())
      gemm_tc_step(m, n, k, A, B, C, false);
    else
      gemm(m, n, k, A, B, C);
  }

  // Shared bonds in the order of `order_src`, plus the remaining bonds of each side.
  struct Split {
    std::vector<int> sh_i, sh_j, rem_i, rem_j;
  };
  Split split(const Value& a, const Value& b) const {
    Split sp;
    std::unordered_set<int> sb(b.bonds.begin(), b.bonds.end()), sa(a.bonds.begin(), a.bonds.end());
    for (int x : a.bonds) (sb.count(x) ? sp.sh_i : sp.rem_i).push_back(x);
    for (int x : b.bonds) (sa.count(x) ? sp.sh_j : sp.rem_j).push_back(x);
    return sp;
  }
  // Choose the shared-bond order and permute operands only when needed.
  // Returns (la, lb) layouts after any permutes; updates ia/ib to the values used.
  void orient(int& ia, int& ib, const Split& sp, std::vector<int>& s_out, int& la, int& lb,
              std::vector<int>& tmps) {
    const std::vector<int>* cand[2] = {&sp.sh_i, &sp.sh_j};
    int best = -1;
    double best_cost = 1e300;
    for (int c = 0; c < 2; ++c) {
      const std::vector<int>& sv = *cand[c];
      int a = layout_of(vals[ia].bonds, sp.rem_i, sv);
      int b = layout_of(vals[ib].bonds, sv, sp.rem_j);
      double cost = (a < 0 ? (double)vals[ia].size : 0.0) + (b < 0 ? (double)vals[ib].size : 0.0);
      if (cost < best_cost) {
        best_cost = cost;
        best = c;
      }
    }
    s_out = *cand[best];
    la = layout_of(vals[ia].bonds, sp.rem_i, s_out);
    lb = layout_of(vals[ib].bonds, s_out, sp.rem_j);
    if (la < 0) {
      std::vector<int> order = sp.rem_i;
      order.insert(order.end(), s_out.begin(), s_out.end());
      ia = permute_to(ia, order);
      tmps.push_back(ia);
      la = 0;
    }
    if (lb < 0) {
      std::vector<int> order = s_out;
      order.insert(order.end(), sp.rem_j.begin(), sp.rem_j.end());
      ib = permute_to(ib, order);
      tmps.push_back(ib);
      lb = 0;
    }
  }

  std::string contract(int i, int j, int k) {
    int ia = cur.at(i), ib = cur.at(j);
    const int ia0 = ia, ib0 = ib;
    Split sp = split(vals[ia], vals[ib]);
    std::vector<int> sh;
    int la, lb;
    std::vector<int> tmps;
    orient(ia, ib, sp, sh, la, lb, tmps);
    const int64_t m = prod_dims(sp.rem_i, dim), n = prod_dims(sp.rem_j, dim), kk = prod_dims(sh, dim);
    if (m > INT32_MAX || n > INT32_MAX || kk > INT32_MAX) return "contraction too large";
    PView A = base_view(vals[ia]);
    if (la == 0) { A.rs = kk; A.cs = 1; } else { A.rs = 1; A.cs = m; }
    PView B = base_view(vals[ib]);
    if (lb == 0) { B.rs = n; B.cs = 1; } else { B.rs = 1; B.cs = kk; }
    std::vector<int> nb = sp.rem_i;
    nb.insert(nb.end(), sp.rem_j.begin(), sp.rem_j.end());
    int ic = new_arena_value(nb);
    PView C = base_view(vals[ic]);
    C.rs = n;
    C.cs = 1;
    if (mixed())
      gemm_tc_step((int)m, (int)n, (int)kk, A, B, C, true);
    else
      gemm((int)m, (int)n, (int)kk, A, B, C);
    const int slot = rescale(ic);
    if (grad) {
      const int my_op = op_index;
      bwd.push_back([=, this]() {
        // C = A B: A' = C' B^T, B' = A^T C' (C' unscaled first)
        op_index = my_op;
        PView gC = gview(ic);
        scale_pow2(gC, m * n, slot);
        gC.rs = n;
        gC.cs = 1;
        PView gA = gview(ia), Bt = B;
        gA.rs = A.rs;
        gA.cs = A.cs;
        std::swap(Bt.rs, Bt.cs);
        gemm_form((int)m, (int)kk, (int)n, gC, Bt, gA);
        PView gB = gview(ib), At = A;
        gB.rs = B.rs;
        gB.cs = B.cs;
        std::swap(At.rs, At.cs);
        gemm_form((int)kk, (int)n, (int)m, At, gC, gB);
        gfree(ic);
        if (ia != ia0) {
          permute_back(ia, ia0);
          gfree(ia);
        }
        if (ib != ib0) {
          permute_back(ib, ib0);
          gfree(ib);
        }
      });
    }
    for (int t : tmps) release_value(t);
    release_value(ia0);
    release_value(ib0);
    cur.erase(i);
    cur.erase(j);
    cur[k] = ic;
    record(k, ic);
    plan->consumed.push_back({op_index, i});
    plan->consumed.push_back({op_index, j});
    plan->n_contractions++;
    return "";
  }

  // Reverse steps of one compression (see k_adjoint.cu for the algebra).
  // A (DA x dab) and B (dab x DB) are the forward operand views, RA (rA x dab)
  // and LB (dab x rB) the triangular factors (A / B themselves when no QR ran),
  // G, V, sig the Jacobi outputs of the core (Jm x Jn, tall: core = M, else M^T).
  void compress_adjoint(int ia, int ib, int ia0, int ib0, PView A, PView B, int64_t DA, int64_t DB, int64_t dab,
                        int64_t rA, int64_t rB, int64_t kk, bool tall, int64_t Jm, int64_t Jn, PView workA,
                        PView workB, PView RA, PView LB, PView G, PView V, PView sig, int na, int nbv, int slot_a,
                        int slot_b) {
    const int64_t q = Jn;
    std::vector<std::pair<int64_t, int64_t>> tr;
    auto tmp = [&](int64_t size) {
      int64_t off;
      PView p = temp(size, &off);
      tr.push_back({off, size});
      return p;
    };
    auto cm = [](PView p, int64_t ld) {  // column-major with leading dimension ld
      p.rs = 1;
      p.cs = ld;
      return p;
    };
    auto tp = [](PView p) {
      std::swap(p.rs, p.cs);
      return p;
    };
    // incoming adjoints of A_bar (DA x kk) and B_bar^T (DB x kk), unscaled, then in the QR bases
    PView gAb = gview(na), gBb = gview(nbv);
    scale_pow2(gAb, DA * kk, slot_a);
    scale_pow2(gBb, DB * kk, slot_b);
    auto applyq = [&](int64_t mm, const PView& work, const PView& X, int64_t ncols, int trans) {
      Step st;
      st.kind = ST_APPLYQ;
      st.m = (int)mm;
      st.n = (int)dab;
      st.k = (int)ncols;
      st.work = work;
      st.C = X;
      st.flag = trans;
      st.bytes = 8.0 * (mm * dab + 2.0 * mm * ncols);
      add(st);
    };
    if (DA > dab) applyq(DA, workA, gAb, kk, 1);
    if (DB > dab) applyq(DB, workB, gBb, kk, 1);
    // sorted singular factors of the core M = U diag(s) W^T (rA x rB)
    PView U = cm(tmp(rA * q), rA), W = cm(tmp(rB * q), rB), sv = tmp(q);
    PView Us = cm(tmp(rA * kk), rA), Ws = cm(tmp(rB * kk), rB);
    {
      Step st;
      st.kind = ST_SVD_FACTORS;
      st.m = (int)Jm;
      st.n = (int)Jn;
      st.k = (int)kk;
      st.flag = tall ? 1 : 0;
      st.C = G;
      st.aux1 = V;
      st.aux2 = sig;
      st.out1 = U;
      st.out2 = W;
      st.work = sv;
      st.A = Us;
      st.B = Ws;
      add(st);
    }
    PView dU = cm(gAb, DA), dV = cm(gBb, DB);   // top rA / rB rows
    PView P = cm(tmp(q * kk), q), Qm = cm(tmp(q * kk), q);
    gemm((int)q, (int)kk, (int)rA, tp(U), dU, P);
    gemm((int)q, (int)kk, (int)rB, tp(W), dV, Qm);
    PView Cc = cm(tmp(q * q), q);
    {
      Step st;
      st.kind = ST_SVD_ADJ_CORE;
      st.n = (int)q;
      st.k = (int)kk;
      st.A = P;
      st.B = Qm;
      st.work = sv;
      st.C = Cc;
      add(st);
    }
    // dU <- dU - U P, dV <- dV - W Q (in place: the complements inside the core)
    gemm((int)rA, (int)kk, (int)q, U, P, dU, -1.0, 1.0);
    gemm((int)rB, (int)kk, (int)q, W, Qm, dV, -1.0, 1.0);
    // D11 = U (C W^T) + dU Ws^T + Us dV^T
    PView T1 = cm(tmp(q * rB), q), D11 = cm(tmp(rA * rB), rA);
    gemm((int)q, (int)rB, (int)q, Cc, tp(W), T1);
    gemm((int)rA, (int)rB, (int)q, U, T1, D11);
    gemm((int)rA, (int)rB, (int)kk, dU, tp(Ws), D11, 1.0, 1.0);
    gemm((int)rA, (int)rB, (int)kk, Us, tp(dV), D11, 1.0, 1.0);
    // A' (DA x dab) into the adjoint of A's value, with A's strides
    const PView RBp = tp(LB);   // R_B' = L_B^T (rB x dab)
    PView gA = gview(ia);
    gA.rs = A.rs;
    gA.cs = A.cs;
    if (DA > dab) {
      PView ZA = cm(tmp(DA * dab), DA);
      gemm((int)rA, (int)dab, (int)rB, D11, RBp, ZA);
      if (DA > rA) {
        PView HB = cm(tmp(kk * dab), kk);
        gemm((int)kk, (int)dab, (int)rB, tp(Ws), RBp, HB);
        PView WA = dU, ZAb = ZA;
        WA.eo = rA;
        ZAb.eo = rA;
        gemm((int)(DA - rA), (int)dab, (int)kk, WA, HB, ZAb);
      }
      applyq(DA, workA, ZA, dab, 0);
      Step cp;
      cp.kind = ST_COPY2D;
      cp.m = (int)DA;
      cp.n = (int)dab;
      cp.A = ZA;
      cp.C = gA;
      cp.bytes = 16.0 * DA * dab;
      add(cp);
    } else {
      gemm((int)DA, (int)dab, (int)rB, D11, RBp, gA);
    }
    // B'^T (DB x dab) into the adjoint of B's value, through B's transposed strides
    PView gBt = gview(ib);
    gBt.rs = B.cs;
    gBt.cs = B.rs;
    if (DB > dab) {
      PView ZB = cm(tmp(DB * dab), DB);
      gemm((int)rB, (int)dab, (int)rA, tp(D11), RA, ZB);
      if (DB > rB) {
        PView HA = cm(tmp(kk * dab), kk);
        gemm((int)kk, (int)dab, (int)rA, tp(Us), RA, HA);
        PView WB = dV, ZBb = ZB;
        WB.eo = rB;
        ZBb.eo = rB;
        gemm((int)(DB - rB), (int)dab, (int)kk, WB, HA, ZBb);
      }
      applyq(DB, workB, ZB, dab, 0);
      Step cp;
      cp.kind = ST_COPY2D;
      cp.m = (int)DB;
      cp.n = (int)dab;
      cp.A = ZB;
      cp.C = gBt;
      cp.bytes = 16.0 * DB * dab;
      add(cp);
    } else {
      gemm((int)DB, (int)dab, (int)rA, tp(D11), RA, gBt);
    }
    for (auto& t : tr) arena.release(t.first, t.second);
    gfree(na);
    gfree(nbv);
    if (ia != ia0) {
      permute_back(ia, ia0);
      gfree(ia);
    }
    if (ib != ib0) {
      permute_back(ib, ib0);
      gfree(ib);
    }
  }

  // ---- tree gauge of distance r, projector form (gauge_r >= 0)
  int gauge_r = -1;

  // Algorithm 2 over the live tensors: ordered pairs (u, v) of the r-local
  // spanning tree grown from {i, j}; only tensors made by a contraction join;
  // candidates are taken closest first, then by the largest product of the
  // bond sizes u and v share, then by the smallest v, then u.
  std::vector<std::pair<int, int>> spanning_tree(int i, int j, int r) {
    const int n_inputs = (int)s.bonds.size();
    std::map<int, std::vector<int>> owner;
    for (const auto& tv : cur)
      for (int b : vals[tv.second].bonds) owner[b].push_back(tv.first);
    auto nbrs = [&](int u) {
      std::set<int> out;
      for (int b : vals[cur.at(u)].bonds)
        for (int o : owner[b])
          if (o != u) out.insert(o);
      return out;
    };
    auto conn = [&](int u, int v) {
      const std::vector<int>& bv = vals[cur.at(v)].bonds;
      double p = 1.0;
      for (int b : vals[cur.at(u)].bonds)
        if (std::find(bv.begin(), bv.end(), b) != bv.end()) p *= (double)dim[b];
      return p;
    };
    std::set<int> region = {i, j};
    std::map<std::pair<int, int>, int> cands;
    for (int u : {i, j})
      for (int v : nbrs(u))
        if (!region.count(v) && v >= n_inputs) cands[{u, v}] = 1;
    std::vector<std::pair<int, int>> tau;
    while (!cands.empty()) {
      auto best = cands.begin();
      for (auto it = cands.begin(); it != cands.end(); ++it) {
        const auto key = std::make_tuple(it->second, -conn(it->first.first, it->first.second), it->first.second,
                                         it->first.first);
        const auto bk = std::make_tuple(best->second, -conn(best->first.first, best->first.second),
                                        best->first.second, best->first.first);
        if (key < bk) best = it;
      }
      const int u = best->first.first, v = best->first.second, d = best->second;
      cands.erase(best);
      if (region.count(v) || d > r) continue;
      region.insert(v);
      tau.push_back({u, v});
      for (int w : nbrs(v))
        if (!region.count(w) && w >= n_inputs && !cands.count({v, w})) cands[{v, w}] = d + 1;
    }
    return tau;
  }

  // A matrix view of value vi with rows `rows` and columns `cols` (bond lists
  // covering the value); permutes into a temporary when neither row-major nor
  // column-major order fits.  Temporaries are appended to `tv`.
  PView mat_view(int vi, const std::vector<int>& rows, const std::vector<int>& cols, std::vector<int>& tv) {
    int lay = layout_of(vals[vi].bonds, rows, cols);
    if (lay < 0) {
      std::vector<int> order = rows;
      order.insert(order.end(), cols.begin(), cols.end());
      vi = permute_to(vi, order);
      tv.push_back(vi);
      lay = 0;
    }
    const int64_t R = prod_dims(rows, dim), Cn = prod_dims(cols, dim);
    PView p = base_view(vals[vi]);
    if (lay == 0) {
      p.rs = Cn;
      p.cs = 1;
    } else {
      p.rs = 1;
      p.cs = R;
    }
    return p;
  }

  // Compression in the tree gauge of distance r (projector form): R factors
  // pushed inwards along the spanning tree on virtual copies, R_A and L_B from
  // the gauged A and B, the SVD of R_A L_B, and P_L = L_B V_k s^-1/2,
  // P_R = s^-1/2 U_k^T R_A applied to the original A and B.
  std::string compress_gauged(int i, int j) {
    int ia = cur.at(i), ib = cur.at(j);
    const int ia0 = ia, ib0 = ib;
    Split sp = split(vals[ia], vals[ib]);
    const int64_t dab = prod_dims(sp.sh_i, dim);
    if (dab <= chi) return "";
    std::vector<int> sh;
    int la, lb;
    std::vector<int> tmps;
    orient(ia, ib, sp, sh, la, lb, tmps);
    const int64_t DA = prod_dims(sp.rem_i, dim), DB = prod_dims(sp.rem_j, dim);
    if (DA > INT32_MAX || DB > INT32_MAX || dab > INT32_MAX) return "compression too large";
    std::vector<std::pair<int64_t, int64_t>> trel;
    auto tmp = [&](int64_t size) {
      int64_t off;
      PView p = temp(size, &off);
      trel.push_back({off, size});
      return p;
    };
    std::vector<int> tvals;  // temporary values (virtual copies, permutes)
    auto qr_r = [&](int64_t m, int64_t n, const PView& A) {
      // R factor (n x n, row-major) of an m x n matrix view, m > n
      PView work = tmp(m * n + n);
      work.bs = m * n;
      PView R = tmp(n * n);
      R.rs = n;
      R.cs = 1;
      Step st;
      st.kind = ST_QR;
      st.m = (int)m;
      st.n = (int)n;
      st.A = A;
      st.work = work;
      st.C = R;
      st.flops = qr_flops((double)m, (double)n);
      st.bytes = 8.0 * (2.0 * m * n + (double)n * n);
      plan->qr_flops += st.flops;
      add(st);
      return R;
    };
    // 1. QR inwards along the spanning tree, on virtual copies
    std::map<int, int> virt;
    const auto tau = gauge_r > 0 ? spanning_tree(i, j, gauge_r) : std::vector<std::pair<int, int>>();
    virt[i] = ia0;
    virt[j] = ib0;
    for (const auto& uv : tau) virt[uv.second] = cur.at(uv.second);
    for (size_t q = tau.size(); q-- > 0;) {
      const int u = tau[q].first, v = tau[q].second;
      const std::vector<int> bv = vals[virt[v]].bonds, bu = vals[virt[u]].bonds;
      std::vector<int> shv, rest, rest_u;
      for (int b : bv) (std::find(bu.begin(), bu.end(), b) != bu.end() ? shv : rest).push_back(b);
      for (int b : bu)
        if (std::find(shv.begin(), shv.end(), b) == shv.end()) rest_u.push_back(b);
      const int64_t Dsh = prod_dims(shv, dim), Drest = prod_dims(rest, dim), Du = prod_dims(rest_u, dim);
      if (Dsh > INT32_MAX || Drest > INT32_MAX || Du > INT32_MAX) return "gauge region too large";
      PView Vm = mat_view(virt[v], rest, shv, tvals);
      PView Rv = Vm;
      int64_t rrows = Drest;
      if (Drest > Dsh) {
        Rv = qr_r(Drest, Dsh, Vm);
        rrows = Dsh;
      }
      const int nb = (int)dim.size();
      dim.push_back(rrows);
      PView Um = mat_view(virt[u], shv, rest_u, tvals);
      std::vector<int> nbl = {nb};
      nbl.insert(nbl.end(), rest_u.begin(), rest_u.end());
      const int nu = new_arena_value(nbl);
      tvals.push_back(nu);
      PView C = base_view(vals[nu]);
      C.rs = Du;
      C.cs = 1;
      gemm((int)rrows, (int)Du, (int)Dsh, Rv, Um, C);
      virt[u] = nu;
    }
    // 2. R_A (rA x dab) and L_B (dab x rB) from the gauged A and B
    std::vector<int> restA, restB;
    for (int b : vals[virt[i]].bonds)
      if (std::find(sh.begin(), sh.end(), b) == sh.end()) restA.push_back(b);
    for (int b : vals[virt[j]].bonds)
      if (std::find(sh.begin(), sh.end(), b) == sh.end()) restB.push_back(b);
    const int64_t DAg = prod_dims(restA, dim), DBg = prod_dims(restB, dim);
    if (DAg > INT32_MAX || DBg > INT32_MAX) return "compression too large";
    PView RA = mat_view(virt[i], restA, sh, tvals);
    int64_t rA = DAg;
    if (DAg > dab) {
      RA = qr_r(DAg, dab, RA);
      rA = dab;
    }
    PView LB = mat_view(virt[j], sh, restB, tvals);
    int64_t rB = DBg;
    if (DBg > dab) {
      PView Bt = LB;
      std::swap(Bt.rs, Bt.cs);
      LB = qr_r(DBg, dab, Bt);
      std::swap(LB.rs, LB.cs);
      rB = dab;
    }
    const int64_t kk = std::min<int64_t>(chi, std::min(rA, rB));
    // 3. SVD of the core R_A L_B (two precisions, V kept), sorted factors
    const bool tall = rA >= rB;
    const int64_t Jm = tall ? rA : rB, Jn = tall ? rB : rA;
    PView M0 = tmp(rA * rB);
    if (tall) { M0.rs = 1; M0.cs = rA; } else { M0.rs = rB; M0.cs = 1; }
    gemm((int)rA, (int)rB, (int)dab, RA, LB, M0);
    PView M0c = M0;
    M0c.rs = 1;
    M0c.cs = Jm;
    PView G32 = tmp((Jm * Jn + 1) / 2), V32 = tmp((Jn * Jn + 1) / 2);
    {
      Step st;
      st.kind = ST_TO_F32;
      st.src = M0;
      st.dst = G32;
      st.count = Jm * Jn;
      st.fbs_dst = 2 * G32.bs;
      add(st);
      Step jst;
      jst.kind = ST_JACOBI32;
      jst.m = (int)Jm;
      jst.n = (int)Jn;
      jst.C = G32;
      jst.aux1 = V32;
      jst.fbs_src = 2 * G32.bs;
      jst.fbs_dst = 2 * V32.bs;
      add(jst);
    }
    PView Vd = tmp(Jn * Jn), V = tmp(Jn * Jn), E = tmp(Jn * Jn);
    {
      Step st;
      st.kind = ST_TO_F64;
      st.src = V32;
      st.dst = Vd;
      st.out1 = V;
      st.count = Jn * Jn;
      st.fbs_src = 2 * V32.bs;
      add(st);
    }
    PView VdT = Vd, VdN = Vd, Ec = E, Vc = V;
    VdT.rs = Jn; VdT.cs = 1;
    VdN.rs = 1; VdN.cs = Jn;
    Ec.rs = Jn; Ec.cs = 1;
    Vc.rs = 1; Vc.cs = Jn;
    gemm((int)Jn, (int)Jn, (int)Jn, VdT, VdN, Ec, 1.0, 0.0, true);
    gemm((int)Jn, (int)Jn, (int)Jn, VdN, Ec, Vc, -0.5, 1.5, true);
    {
      Step cp;
      cp.kind = ST_COPY;
      cp.src = V;
      cp.dst = Vd;
      cp.count = Jn * Jn;
      add(cp);
    }
    PView VT = V;
    VT.rs = Jn;
    VT.cs = 1;
    gemm((int)Jn, (int)Jn, (int)Jn, VT, Vc, Ec, 1.0, 0.0, true);
    gemm((int)Jn, (int)Jn, (int)Jn, VdN, Ec, Vc, -0.5, 1.5, true);
    PView G = tmp(Jm * Jn);
    G.rs = 1;
    G.cs = Jm;
    gemm((int)Jm, (int)Jn, (int)Jn, M0c, Vc, G, 1.0, 0.0, true);
    PView sig = tmp(Jn);
    {
      Step st;
      st.kind = ST_JACOBI;
      st.m = (int)Jm;
      st.n = (int)Jn;
      st.C = G;
      st.aux1 = V;
      st.aux2 = sig;
      st.init_v = 0;
      st.no_v = 0;
      st.jac_tol = 1e-8;
      st.flops = svd_flops((double)rA, (double)rB);
      plan->svd_flops += st.flops;
      add(st);
    }
    const int64_t q = Jn;
    PView U = tmp(rA * q), W = tmp(rB * q), sv = tmp(q), Us = tmp(rA * kk), Ws = tmp(rB * kk);
    {
      Step st;
      st.kind = ST_SVD_FACTORS;
      st.m = (int)Jm;
      st.n = (int)Jn;
      st.k = (int)kk;
      st.flag = tall ? 1 : 0;
      st.C = G;
      st.aux1 = V;
      st.aux2 = sig;
      st.out1 = U;
      st.out2 = W;
      st.work = sv;
      st.A = Us;
      st.B = Ws;
      add(st);
    }
    Us.rs = 1; Us.cs = rA;
    Ws.rs = 1; Ws.cs = rB;
    // 4. projectors P_L = L_B W_s (dab x k) and P_R^T = R_A^T U_s (dab x k)
    PView PL = tmp(dab * kk), PRt = tmp(dab * kk);
    PL.rs = kk; PL.cs = 1;
    PRt.rs = kk; PRt.cs = 1;
    gemm((int)dab, (int)kk, (int)rB, LB, Ws, PL);
    PView RAt = RA;
    std::swap(RAt.rs, RAt.cs);
    gemm((int)dab, (int)kk, (int)rA, RAt, Us, PRt);
    // 5. A <- A P_L, B^T <- B^T P_R^T into the new tensors (column-major, bonds [new, rest...])
    const int nbond = (int)dim.size();
    dim.push_back(kk);
    std::vector<int> bi = {nbond};
    bi.insert(bi.end(), sp.rem_i.begin(), sp.rem_i.end());
    std::vector<int> bj = {nbond};
    bj.insert(bj.end(), sp.rem_j.begin(), sp.rem_j.end());
    const int na = new_arena_value(bi), nbv = new_arena_value(bj);
    PView A = base_view(vals[ia]);
    if (la == 0) { A.rs = dab; A.cs = 1; } else { A.rs = 1; A.cs = DA; }
    PView B = base_view(vals[ib]);
    if (lb == 0) { B.rs = DB; B.cs = 1; } else { B.rs = 1; B.cs = dab; }
    PView Ab = base_view(vals[na]), Bb = base_view(vals[nbv]);
    Ab.rs = 1; Ab.cs = DA;
    Bb.rs = 1; Bb.cs = DB;
    gemm((int)DA, (int)kk, (int)dab, A, PL, Ab);
    PView Bt = B;
    std::swap(Bt.rs, Bt.cs);
    gemm((int)DB, (int)kk, (int)dab, Bt, PRt, Bb);
    plan->gemm_flops += 2.0 * DA * dab * (double)kk + 2.0 * DB * dab * (double)kk;
    rescale(na);
    rescale(nbv);
    for (auto& t : trel) rel(t.first, t.second);
    for (int t : tvals) release_value(t);
    for (int t : tmps) release_value(t);
    release_value(ia0);
    release_value(ib0);
    cur[i] = na;
    cur[j] = nbv;
    record(i, na);
    record(j, nbv);
    plan->n_compressions++;
    return "";
  }

  std::string compress(int i, int j) {
    if (gauge_r >= 0) return compress_gauged(i, j);
    int ia = cur.at(i), ib = cur.at(j);
    const int ia0 = ia, ib0 = ib;
    Split sp = split(vals[ia], vals[ib]);
    const int64_t dab = prod_dims(sp.sh_i, dim);
    if (dab <= chi) return "";
    std::vector<int> sh;
    int la, lb;
    std::vector<int> tmps;
    orient(ia, ib, sp, sh, la, lb, tmps);
    const int64_t DA = prod_dims(sp.rem_i, dim), DB = prod_dims(sp.rem_j, dim);
    if (DA > INT32_MAX || DB > INT32_MAX || dab > INT32_MAX) return "compression too large";
    const int64_t rA = std::min(DA, dab), rB = std::min(DB, dab);
    const int64_t kk = std::min<int64_t>(chi, std::min(rA, rB));
    std::vector<std::pair<int64_t, int64_t>> trel;  // temporaries (off, size)
    auto tmp = [&](int64_t size) {
      int64_t off;
      PView p = temp(size, &off);
      trel.push_back({off, size});
      return p;
    };
    PView A = base_view(vals[ia]);
    if (la == 0) { A.rs = dab; A.cs = 1; } else { A.rs = 1; A.cs = DA; }
    PView B = base_view(vals[ib]);
    if (lb == 0) { B.rs = DB; B.cs = 1; } else { B.rs = 1; B.cs = dab; }
    // R_A (rA x dab)
    PView RA, workA, workB;
    if (DA > dab) {
      PView work = tmp(DA * dab + dab);
      workA = work;
      workA.bs = DA * dab;
      RA = tmp(rA * dab);
      RA.rs = dab;
      RA.cs = 1;
      Step st;
      st.kind = ST_QR;
      st.m = (int)DA;
      st.n = (int)dab;
      st.A = A;
      st.work = work;
      st.work.bs = DA * dab;
      st.C = RA;
      st.flops = qr_flops((double)DA, (double)dab);
      st.bytes = 8.0 * (2.0 * DA * dab + (double)rA * dab);
      plan->qr_flops += st.flops;
      add(st);
    } else {
      RA = A;
    }
    // L_B (dab x rB) as the transpose of R of B^T (rB x dab)
    PView LB;
    if (DB > dab) {
      PView work = tmp(DB * dab + dab);
      workB = work;
      workB.bs = DB * dab;
      PView RBt = tmp(rB * dab);
      RBt.rs = dab;
      RBt.cs = 1;
      PView Bt = B;
      std::swap(Bt.rs, Bt.cs);
      Step st;
      st.kind = ST_QR;
      st.lane = 1;   // independent of the QR of A: overlaps it on the side stream
      st.m = (int)DB;
      st.n = (int)dab;
      st.A = Bt;
      st.work = work;
      st.work.bs = DB * dab;
      st.C = RBt;
      st.flops = qr_flops((double)DB, (double)dab);
      st.bytes = 8.0 * (2.0 * DB * dab + (double)rB * dab);
      plan->qr_flops += st.flops;
      add(st);
      LB = RBt;
      std::swap(LB.rs, LB.cs);
    } else {
      LB = B;
    }
    // core M = R_A L_B, stored so that Jacobi sees an (Jm x Jn) column-major matrix, Jm >= Jn
    // (M itself when rA >= rB, else M^T, i.e. M row-major)
    const bool tall = rA >= rB;
    const int64_t Jm = tall ? rA : rB, Jn = tall ? rB : rA;
    PView M0 = tmp(rA * rB);
    if (tall) { M0.rs = 1; M0.cs = rA; } else { M0.rs = rB; M0.cs = 1; }
    gemm((int)rA, (int)rB, (int)dab, RA, LB, M0);
    if (DB > dab) plan->steps.back().join = 1;
    PView M0c = M0;  // the same buffer as a Jm x Jn column-major view
    M0c.rs = 1;
    M0c.cs = Jm;
    // 1. FP32 preconditioner: Jacobi on a float copy from V = I
    PView G32 = tmp((Jm * Jn + 1) / 2), V32 = tmp((Jn * Jn + 1) / 2);
    {
      Step st;
      st.kind = ST_TO_F32;
      st.src = M0;
      st.dst = G32;
      st.count = Jm * Jn;
      st.fbs_dst = 2 * G32.bs;
      st.bytes = 12.0 * (double)st.count;
      add(st);
      Step j;
      j.kind = ST_JACOBI32;
      j.m = (int)Jm;
      j.n = (int)Jn;
      j.C = G32;
      j.aux1 = V32;
      j.fbs_src = 2 * G32.bs;
      j.fbs_dst = 2 * V32.bs;
      add(j);
    }
    // 2. V <- two Newton-Schulz steps on the FP64 copy: V (1.5 I - 0.5 V^T V); G = M V
    PView Vd = tmp(Jn * Jn), V = tmp(Jn * Jn), E = tmp(Jn * Jn);
    {
      Step st;
      st.kind = ST_TO_F64;
      st.src = V32;
      st.dst = Vd;
      st.out1 = V;
      st.count = Jn * Jn;
      st.fbs_src = 2 * V32.bs;
      st.bytes = 20.0 * (double)st.count;
      add(st);
    }
    PView VdT = Vd, VdN = Vd, Ec = E, Vc = V;
    VdT.rs = Jn; VdT.cs = 1;
    VdN.rs = 1; VdN.cs = Jn;
    Ec.rs = Jn; Ec.cs = 1;
    Vc.rs = 1; Vc.cs = Jn;
    // step 1: E = Vd^T Vd, V = 1.5 V - 0.5 Vd E (V == Vd on entry)
    gemm((int)Jn, (int)Jn, (int)Jn, VdT, VdN, Ec, 1.0, 0.0, /*overhead=*/true);
    gemm((int)Jn, (int)Jn, (int)Jn, VdN, Ec, Vc, -0.5, 1.5, true);
    // step 2: Vd = V, E = V^T V, V = 1.5 V - 0.5 Vd E
    {
      Step cp;
      cp.kind = ST_COPY;
      cp.src = V;
      cp.dst = Vd;
      cp.count = Jn * Jn;
      add(cp);
    }
    PView VT = V;
    VT.rs = Jn;
    VT.cs = 1;
    gemm((int)Jn, (int)Jn, (int)Jn, VT, Vc, Ec, 1.0, 0.0, true);
    gemm((int)Jn, (int)Jn, (int)Jn, VdN, Ec, Vc, -0.5, 1.5, true);
    PView G = tmp(Jm * Jn);
    G.rs = 1;
    G.cs = Jm;
    gemm((int)Jm, (int)Jn, (int)Jn, M0c, Vc, G, 1.0, 0.0, true);
    // 3. FP64 Jacobi from V: converges quadratically to the FP64 SVD.  Without
    // V (the forward pass) only the kk kept directions are used: the polish
    // still rotates every pair, but judges convergence on the pairs touching
    // the kept columns (mark_active_f64)
    PView sig = tmp(Jn);
    PView act;
    if (!keep_v) {
      act = tmp((Jn + 1) / 2);
      Step mk;
      mk.kind = ST_MARK_ACTIVE;
      mk.m = (int)Jm;
      mk.n = (int)Jn;
      mk.k = (int)kk;
      mk.C = G;
      mk.out1 = act;
      mk.bytes = 8.0 * (double)Jm * Jn;
      add(mk);
    }
    {
      Step st;
      st.kind = ST_JACOBI;
      st.work = act;
      st.m = (int)Jm;
      st.n = (int)Jn;
      st.C = G;
      st.aux1 = V;
      st.aux2 = sig;
      st.init_v = 0;
      // V_k is recovered after the sweeps from M^T U_k (a GEMM), see below; the
      // reverse pass needs every right vector accurately, so it keeps V
      st.no_v = keep_v ? 0 : 1;
      st.jac_tol = 1e-8;
      st.flops = svd_flops((double)rA, (double)rB);
      st.bytes = 8.0 * (2.0 * Jm * Jn + 2.0 * Jn * Jn);
      plan->svd_flops += st.flops;
      plan->max_jacobi_n = std::max<int64_t>(plan->max_jacobi_n, Jn);
      add(st);
    }
    // truncate + absorb (Eq. "svd"): A_bar = Q_A [U_k s^1/2; 0], B_bar^T = Q' [V_k s^1/2; 0]
    // with B^T = Q' R'.  The selected factors are written zero-padded straight into
    // the new tensors, stored column-major (D x kk), i.e. with bonds [new, rem...],
    // and the Householder products of the two QRs are applied in place.
    const int nbond = (int)dim.size();
    dim.push_back(kk);
    int na = -1, nbv = -1;
    {
      std::vector<int> bi = {nbond};
      bi.insert(bi.end(), sp.rem_i.begin(), sp.rem_i.end());
      std::vector<int> bj = {nbond};
      bj.insert(bj.end(), sp.rem_j.begin(), sp.rem_j.end());
      na = new_arena_value(bi);
      nbv = new_arena_value(bj);
      PView Ab = base_view(vals[na]), Bb = base_view(vals[nbv]);
      PView K3 = tmp(Jm * kk);
      {
        Step st;
        st.kind = ST_SELECT;
        st.m = (int)Jm;
        st.n = (int)Jn;
        st.k = (int)kk;
        st.C = G;
        st.aux1 = V;
        st.aux2 = sig;
        st.no_v = keep_v ? 0 : 1;
        st.work = K3;
        // left singular side (rows of the Jacobi matrix) and right side
        st.out1 = tall ? Ab : Bb;
        st.out2 = tall ? Bb : Ab;
        st.count = tall ? DA : DB;     // leading dimension of out1
        st.init_v = (int)(tall ? DB : DA);  // leading dimension of out2
        st.bytes = 8.0 * (double)kk * (Jm + Jn + DA + DB);
        add(st);
      }
      // right factor V_k sigma^1/2 = G0^T U_k sigma^-1/2 = G0^T K3 into rows 0..Jn-1 of out2
      if (!keep_v) {
        PView G0T = M0c, K3v = K3, R = tall ? Bb : Ab;
        G0T.rs = Jm;
        G0T.cs = 1;
        K3v.rs = 1;
        K3v.cs = Jm;
        R.rs = 1;
        R.cs = tall ? DB : DA;
        gemm((int)Jn, (int)kk, (int)Jm, G0T, K3v, R, 1.0, 0.0, true);
      }
      auto apply = [&](int64_t mm, const PView& work, const PView& X) {
        Step st;
        st.kind = ST_APPLYQ;
        st.m = (int)mm;
        st.n = (int)dab;
        st.k = (int)kk;
        st.work = work;
        st.C = X;
        st.flops = 0.0;
        st.bytes = 8.0 * (mm * dab + 2.0 * mm * kk);
        add(st);
      };
      if (DA > dab) apply(DA, workA, Ab);
      if (DB > dab) apply(DB, workB, Bb);
    }
    // the paper's absorb contractions: (D_A x r_A)(r_A x k) and (k x r_B)(r_B x D_B)
    plan->gemm_flops += 2.0 * DA * rA * (double)kk + 2.0 * kk * rB * (double)DB;
    const int slot_a = rescale(na), slot_b = rescale(nbv);
    if (grad) {
      const int my_op = op_index;
      bwd.push_back([=, this]() {
        op_index = my_op;
        compress_adjoint(ia, ib, ia0, ib0, A, B, DA, DB, dab, rA, rB, kk, tall, Jm, Jn, workA, workB, RA, LB, G, V,
                         sig, na, nbv, slot_a, slot_b);
      });
    }
    for (auto& t : trel) rel(t.first, t.second);
    for (int t : tmps) release_value(t);
    release_value(ia0);
    release_value(ib0);
    cur[i] = na;
    cur[j] = nbv;
    record(i, na);
    record(j, nbv);
    plan->n_compressions++;
    return "";
  }
};

}  // namespace

std::string validate_tree(const Structure& s, const std::vector<int32_t>& ops, int n_inputs) {
  const int nt = (int)s.bonds.size();
  if (n_inputs != nt) return "tree inputs != network tensors";
  if (ops.size() % 4) return "ops array is not a multiple of 4";
  std::unordered_set<int> live;
  for (int t = 0; t < nt; ++t) live.insert(t);
  int next = nt;
  const size_t nops = ops.size() / 4;
  for (size_t r = 0; r < nops; ++r) {
    const int kind = ops[4 * r], i = ops[4 * r + 1], j = ops[4 * r + 2], k = ops[4 * r + 3];
    if (i == j || !live.count(i) || !live.count(j))
      return "op " + std::to_string(r) + ": ids " + std::to_string(i) + ", " + std::to_string(j) +
             " are not two live tensors";
    if (kind == 0) {
      if (k != next) return "op " + std::to_string(r) + ": C must create id " + std::to_string(next);
      live.erase(i);
      live.erase(j);
      live.insert(k);
      ++next;
    } else if (kind != 1) {
      return "op " + std::to_string(r) + ": unknown kind";
    }
  }
  if (live.size() != 1) return "tree leaves " + std::to_string(live.size()) + " tensors (need 1)";
  return "";
}

namespace {

// Gradient plan with checkpointed recomputation.  Forward: the ops run with
// normal arena reuse and no tape; at the start of every segment each live
// tensor is copied to a checkpoint buffer.  Reverse, segment by segment from
// the last: the segment's ops run again from its checkpoints with every
// operand kept (its tape), the adjoints of the tensors live at its end are
// taken over from the next segment's checkpoints (or the root), its reverse
// steps run, and its tape and the next segment's checkpoints are released.
// The arena then holds the checkpoints plus one segment's tape.
std::string build_checkpointed(Builder& bld, const std::vector<int32_t>& ops, int segments) {
  Plan* out = bld.plan;
  const size_t nops = ops.size() / 4;
  std::vector<size_t> cut;
  for (int q = 0; q <= segments; ++q) cut.push_back(nops * (size_t)q / (size_t)segments);
  // per segment: tensor id -> checkpoint value (inputs are their own checkpoint in segment 0)
  std::vector<std::map<int, int>> ck(segments);
  std::vector<std::vector<std::pair<int64_t, int64_t>>> ck_alloc(segments);
  bld.grad = false;
  bld.keep = false;
  for (int sg = 0; sg < segments; ++sg) {
    for (const auto& tv : bld.cur) {
      const Value& v = bld.vals[tv.second];
      if (v.buf == BUF_INPUT || sg == 0) {
        ck[sg][tv.first] = tv.second;
        continue;
      }
      Value c = v;
      c.off = bld.arena.alloc(c.size);
      ck_alloc[sg].push_back({c.off, c.size});
      bld.vals.push_back(c);
      const int ci = (int)bld.vals.size() - 1;
      Step cp;
      cp.kind = ST_COPY;
      cp.op_index = (int)cut[sg];
      cp.src = bld.base_view(v);
      cp.dst = bld.base_view(c);
      cp.count = c.size;
      out->steps.push_back(cp);
      ck[sg][tv.first] = ci;
    }
    for (size_t r = cut[sg]; r < cut[sg + 1]; ++r) {
      bld.op_index = (int)r;
      const int kind = ops[4 * r], i = ops[4 * r + 1], j = ops[4 * r + 2], k = ops[4 * r + 3];
      std::string e = (kind == 0) ? bld.contract(i, j, k) : bld.compress(i, j);
      if (!e.empty()) return "op " + std::to_string(r) + ": " + e;
    }
  }
  if (bld.cur.size() != 1) return "tree does not end in one tensor";
  const int root = bld.cur.begin()->second;
  if (bld.vals[root].size != 1) return "final tensor has open bonds";
  out->final_scalar = bld.base_view(bld.vals[root]);
  Step fin;
  fin.kind = ST_FINAL;
  fin.C = out->final_scalar;
  out->steps.push_back(fin);
  Step fg;
  fg.kind = ST_FINAL_GRAD;
  fg.C = out->final_scalar;
  fg.out1 = bld.gview(root);
  fg.op_index = (int)nops;
  out->steps.push_back(fg);
  const int root_tensor = bld.cur.begin()->first;
  // adjoints of the tensors live at the end of the segment being processed
  std::map<int, int> end_adj = {{root_tensor, root}};
  for (int sg = segments - 1; sg >= 0; --sg) {
    // recompute the segment from its checkpoints, keeping every operand
    bld.cur.clear();
    for (const auto& tv : ck[sg]) bld.cur[tv.first] = tv.second;
    bld.bwd.clear();
    bld.grad = true;
    bld.keep = true;
    bld.in_bwd = false;
    std::vector<std::pair<int64_t, int64_t>> tape;
    bld.rec_alloc = &tape;
    for (size_t r = cut[sg]; r < cut[sg + 1]; ++r) {
      bld.op_index = (int)r;
      const int kind = ops[4 * r], i = ops[4 * r + 1], j = ops[4 * r + 2], k = ops[4 * r + 3];
      std::string e = (kind == 0) ? bld.contract(i, j, k) : bld.compress(i, j);
      if (!e.empty()) return "op " + std::to_string(r) + " (recomputed): " + e;
    }
    bld.rec_alloc = nullptr;
    // the adjoint of each tensor live at the segment's end moves onto its recomputed value
    for (const auto& tv : end_adj) {
      auto it = bld.cur.find(tv.first);
      if (it == bld.cur.end()) return "checkpoint bookkeeping: tensor missing at a segment end";
      const int vi = it->second, src = tv.second;
      if (vi == src) continue;
      if (bld.vals[vi].size != bld.vals[src].size) return "checkpoint bookkeeping: size mismatch";
      auto g = bld.gv.find(src);
      if (g == bld.gv.end()) return "checkpoint bookkeeping: missing adjoint";
      bld.gv[vi] = g->second;
      bld.gv.erase(g);
    }
    bld.keep = false;
    bld.in_bwd = true;
    for (size_t r = bld.bwd.size(); r-- > 0;) bld.bwd[r]();
    bld.in_bwd = false;
    for (auto& a : tape) bld.arena.release(a.first, a.second);
    if (sg + 1 < segments)
      for (auto& a : ck_alloc[sg + 1]) bld.arena.release(a.first, a.second);
    end_adj = ck[sg];
  }
  return "";
}

}  // namespace

std::string build_plan(const Structure& s, const std::vector<int32_t>& ops, int n_inputs, int chi,
                       int prec, Plan* out, bool grad, int segments, int gauge_r) {
  std::string err = validate_tree(s, ops, n_inputs);
  if (!err.empty()) return err;
  if (chi < 1) return "chi must be >= 1";
  if (segments < 1) return "segments must be >= 1";
  if (grad && gauge_r >= 0) return "the reverse pass is not available with the tree gauge";
  *out = Plan();
  out->chi = chi;
  out->prec = prec;
  Builder bld{s, chi, out};
  bld.dim = s.bond_dims;
  bld.grad = grad;
  bld.keep = grad;
  bld.keep_v = grad;
  bld.gauge_r = gauge_r;
  out->gauge_r = gauge_r;
  out->grad = grad;
  out->in_total = s.in_total;
  const int nt = (int)s.bonds.size();
  for (int t = 0; t < nt; ++t) {
    Value v;
    v.bonds = s.bonds[t];
    v.size = prod_dims(v.bonds, bld.dim);
    v.buf = BUF_INPUT;
    v.off = s.in_off[t];
    v.bs = s.in_total;
    bld.vals.push_back(v);
    bld.cur[t] = t;
    bld.op_index = -1;
    bld.record(t, t);
  }
  const size_t nops = ops.size() / 4;
  if (grad && segments > 1 && nops > 1) {
    out->segments = segments < (int)nops ? segments : (int)nops;
    std::string e = build_checkpointed(bld, ops, out->segments);
    if (!e.empty()) return e;
    out->arena_units = bld.arena.peak();
    return "";
  }
  for (size_t r = 0; r < nops; ++r) {
    bld.op_index = (int)r;
    const int kind = ops[4 * r], i = ops[4 * r + 1], j = ops[4 * r + 2], k = ops[4 * r + 3];
    std::string e = (kind == 0) ? bld.contract(i, j, k) : bld.compress(i, j);
    if (!e.empty()) return "op " + std::to_string(r) + ": " + e;
  }
  // the single remaining tensor must be a scalar
  if (bld.cur.size() != 1) return "tree does not end in one tensor";
  const Value& root = bld.vals[bld.cur.begin()->second];
  if (root.size != 1) return "final tensor has open bonds";
  out->final_scalar = bld.base_view(root);
  Step fin;
  fin.kind = ST_FINAL;
  fin.C = out->final_scalar;
  out->steps.push_back(fin);
  if (grad) {
    // reverse pass: d ln|x| / dx = 1 / x at the root, then every op backwards
    bld.keep = false;
    bld.in_bwd = true;
    Step fg;
    fg.kind = ST_FINAL_GRAD;
    fg.C = out->final_scalar;
    fg.out1 = bld.gview(bld.cur.begin()->second);
    fg.op_index = (int)nops;
    out->steps.push_back(fg);
    for (size_t r = bld.bwd.size(); r-- > 0;) bld.bwd[r]();
  }
  out->arena_units = bld.arena.peak();
  return "";
}

}  // namespace tnp
