// Step dispatch and structure validation shared by both executors (tn_exec.h).
#include "tn_exec.h"

#include "../../include/tn.h"

namespace tnx {

cudaError_t exec_step(const tnp::Step& stp, const ExecEnv& env, cudaStream_t s) {
  const int batch = env.batch;
  auto ptr = [&](const tnp::PView& v) { return env.ptr(v); };
  auto cview = [&](const tnp::PView& v) { return tnk::View{ptr(v), v.rs, v.cs, v.bs}; };
  auto wview = [&](const tnp::PView& v) { return tnk::ViewW{ptr(v), v.rs, v.cs, v.bs}; };
  switch (stp.kind) {
    case tnp::ST_PERMUTE:
      return tnk::permute_f64(ptr(stp.src), stp.src.bs, ptr(stp.dst), stp.dst.bs, (int)stp.in_dims.size(),
                              stp.in_dims.data(), stp.perm.data(), batch, s);
    case tnp::ST_GEMM:
      return tnk::gemm_f64(stp.m, stp.n, stp.k, stp.alpha, cview(stp.A), cview(stp.B), stp.beta, wview(stp.C),
                           batch, s);
    case tnp::ST_QR:
      return tnk::qr_r_f64(stp.m, stp.n, cview(stp.A), ptr(stp.work), stp.work.bs, wview(stp.C), batch, s);
    case tnp::ST_JACOBI:
      return tnk::jacobi_svd_f64(stp.m, stp.n, ptr(stp.C), stp.C.bs, stp.no_v ? nullptr : ptr(stp.aux1),
                                 stp.aux1.bs, ptr(stp.aux2), stp.aux2.bs, env.jac_ws, env.ds, stp.init_v, batch, s,
                                 env.sweeps64, stp.jac_tol, env.jac_max_sweeps,
                                 stp.work.bs > 0 ? reinterpret_cast<const int*>(ptr(stp.work)) : nullptr,
                                 2 * stp.work.bs);
    case tnp::ST_TO_F32:
      return tnk::convert_f64_to_f32(ptr(stp.src), stp.count, stp.src.bs, reinterpret_cast<float*>(ptr(stp.dst)),
                                     stp.fbs_dst, batch, s);
    case tnp::ST_JACOBI32:
      return tnk::jacobi_svd_f32(stp.m, stp.n, reinterpret_cast<float*>(ptr(stp.C)), stp.fbs_src,
                                 reinterpret_cast<float*>(ptr(stp.aux1)), stp.fbs_dst, env.jac_ws, env.ds, batch, s,
                                 env.sweeps32);
    case tnp::ST_COPY:
      return cudaMemcpyAsync(ptr(stp.dst), ptr(stp.src), sizeof(double) * (size_t)stp.dst.bs * batch,
                             cudaMemcpyDeviceToDevice, s);
    case tnp::ST_TO_F64:
      return tnk::convert_f32_to_f64(reinterpret_cast<const float*>(ptr(stp.src)), stp.count, stp.fbs_src,
                                     ptr(stp.dst), ptr(stp.out1), stp.dst.bs, batch, s);
    case tnp::ST_SELECT:
      return tnk::select_scale_f64(stp.m, stp.n, stp.k, ptr(stp.C), stp.C.bs, stp.no_v ? nullptr : ptr(stp.aux1),
                                   stp.aux1.bs, ptr(stp.aux2), stp.aux2.bs, ptr(stp.out1), stp.out1.bs,
                                   (int)stp.count, ptr(stp.out2), stp.out2.bs, stp.init_v, batch, s,
                                   stp.no_v ? ptr(stp.work) : nullptr, stp.work.bs);
    case tnp::ST_APPLYQ:
      return tnk::apply_q_f64(stp.m, stp.n, ptr(stp.work), stp.work.bs, ptr(stp.C), stp.C.bs, stp.k, batch, s,
                              stp.flag);
    case tnp::ST_GEMM_TC:
      return tnk::gemm_tc(stp.m, stp.n, stp.k, 1.0, cview(stp.A), cview(stp.B), wview(stp.C), batch, stp.tc_mode,
                          ptr(stp.work), sizeof(double) * (size_t)stp.work.bs * batch, env.tc_err, s,
                          env.tc_give_up);
    case tnp::ST_RESCALE:
      return tnk::rescale_f64(ptr(stp.C), stp.count, stp.C.bs, env.maxbits, env.ds, batch, s,
                              stp.slot >= 0 && env.etape ? env.etape + (size_t)stp.slot * batch : nullptr);
    case tnp::ST_FINAL:
      return tnk::finalize_f64(ptr(stp.C), stp.C.bs, env.ds, env.out_log, env.out_sign, batch, s);
    case tnp::ST_SCALE_POW2:
      if (!env.etape) return cudaErrorInvalidValue;
      return tnk::scale_pow2_f64(ptr(stp.C), stp.count, stp.C.bs, env.etape + (size_t)stp.slot * batch, batch, s);
    case tnp::ST_FINAL_GRAD:
      return tnk::final_grad_f64(ptr(stp.C), stp.C.bs, ptr(stp.out1), stp.out1.bs, batch, s);
    case tnp::ST_SVD_FACTORS:
      return tnk::svd_factors_f64(stp.m, stp.n, stp.k, stp.flag, ptr(stp.C), stp.C.bs, ptr(stp.aux1), stp.aux1.bs,
                                  ptr(stp.aux2), stp.aux2.bs, ptr(stp.out1), stp.out1.bs, ptr(stp.out2),
                                  stp.out2.bs, ptr(stp.work), stp.work.bs, ptr(stp.A), stp.A.bs, ptr(stp.B),
                                  stp.B.bs, batch, s);
    case tnp::ST_SVD_ADJ_CORE:
      return tnk::svd_adjoint_core_f64(stp.n, stp.k, ptr(stp.A), stp.A.bs, ptr(stp.B), stp.B.bs, ptr(stp.work),
                                       stp.work.bs, ptr(stp.C), stp.C.bs, batch, s);
    case tnp::ST_COPY2D:
      return tnk::copy2d_f64(stp.m, stp.n, cview(stp.A), wview(stp.C), batch, s);
    case tnp::ST_MARK_ACTIVE:
      return tnk::mark_active_f64(stp.m, stp.n, stp.k, ptr(stp.C), stp.C.bs, reinterpret_cast<int*>(ptr(stp.out1)),
                                  2 * stp.out1.bs, batch, s);
    default:
      return cudaErrorInvalidValue;
  }
}

int check_structure(int32_t n_bonds, const int64_t* bond_dims, int32_t n_tensors, const int32_t* ndims,
                    const int32_t* bond_ids, tnp::Structure* st, std::string* msg) {
  auto bad = [&](int code, const std::string& m) {
    *msg = m;
    return code;
  };
  if (n_bonds < 0 || n_tensors < 1) return bad(TN_EINVAL, "network needs >= 1 tensor");
  if (n_bonds > 0 && !bond_dims) return bad(TN_EINVAL, "bond_dims is NULL");
  if (!ndims || (n_bonds > 0 && !bond_ids)) return bad(TN_EINVAL, "ndims / bond_ids is NULL");
  st->bond_dims.assign(bond_dims, bond_dims + n_bonds);
  for (int64_t d : st->bond_dims)
    if (d < 1 || d > (1ll << 31)) return bad(TN_ESHAPE, "bond size out of range");
  std::vector<int> count(n_bonds, 0), first(n_bonds, -1);
  st->bonds.assign(n_tensors, {});
  st->in_off.assign(n_tensors, 0);
  int64_t pos = 0, off = 0;
  for (int t = 0; t < n_tensors; ++t) {
    if (ndims[t] < 0 || ndims[t] > tnk::kMaxDims)
      return bad(TN_ESHAPE, "tensor " + std::to_string(t) + ": bad number of bonds");
    double sz = 1.0;
    int64_t isz = 1;
    for (int a = 0; a < ndims[t]; ++a) {
      int b = bond_ids[pos++];
      if (b < 0 || b >= n_bonds) return bad(TN_ESHAPE, "tensor " + std::to_string(t) + ": bond id out of range");
      if (first[b] == t)
        return bad(TN_ESHAPE, "tensor " + std::to_string(t) + " lists bond " + std::to_string(b) + " twice");
      if (first[b] < 0) first[b] = t;
      count[b]++;
      st->bonds[t].push_back(b);
      sz *= (double)st->bond_dims[b];
      if (sz > 4e9) return bad(TN_ESHAPE, "tensor " + std::to_string(t) + " too large");
      isz *= st->bond_dims[b];
    }
    st->in_off[t] = off;
    off += (isz + 31) / 32 * 32;
  }
  for (int b = 0; b < n_bonds; ++b)
    if (count[b] != 2)
      return bad(TN_ESHAPE, "bond " + std::to_string(b) + " appears " + std::to_string(count[b]) + " times (need 2)");
  st->in_total = off;
  return TN_OK;
}

}  // namespace tnx
