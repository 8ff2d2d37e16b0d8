// tn_contract_approx_noalloc: the approximate contraction of one small
// instance without any device allocation.
//
// Some callers cannot call cudaMalloc: a plug-in inside a host application
// whose own allocator has already reserved the device memory (a second
// allocator would fail or fragment it), or code on a latency-critical path
// where cudaMalloc / cudaFree would synchronise the whole device.  For them
// this entry point takes every device buffer it needs -- the copied input
// tensors, the schedule's arena, the QR / Jacobi / log-norm scratch and the
// result words -- from one file-scope __device__ array of fixed size
// (kNoAllocBytes below, 8 MiB), which every GPU that loads the library holds
// until the process exits.  The kernels, the schedule and therefore the
// results are the same as tn_contract_approx's for a batch of one in the FP64
// form with the plain Q-form compressions; the network checks and the launch
// of every step are the shared ones of tn_exec.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tn.h"
#include "tn_exec.h"
#include "tn_kernels.h"
#include "tn_plan.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (in host code the symbol is only a stand-in).
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};

int set_err(char* buf, size_t cap, int code, const std::string& msg) {
  if (buf && cap) {
    std::snprintf(buf, cap, "%s", msg.c_str());
  }
  return code;
}

}  // namespace

extern "C" int tn_contract_approx_noalloc(const tn_network_desc* net, const tn_tree_desc* tree, int chi,
                                          void* cuda_stream, double* logabsz_out, int* sign_out, char* err_msg,
                                          size_t err_cap) {
  if (!net || !tree || !logabsz_out || !sign_out) return set_err(err_msg, err_cap, TN_EINVAL, "NULL argument");
  if (chi < 1) return set_err(err_msg, err_cap, TN_EINVAL, "chi must be >= 1");
  if (!net->data) return set_err(err_msg, err_cap, TN_EINVAL, "data is NULL");
  // the same structure checks as tn_load_network (every bond in exactly two
  // different tensors, sizes in range), then the same finite-entry scan
  tnp::Structure st;
  std::string why;
  const int src = tnx::check_structure(net->n_bonds, net->bond_dims, net->n_tensors, net->ndims, net->bond_ids, &st,
                                       &why);
  if (src != TN_OK) return set_err(err_msg, err_cap, src, why);
  for (int t = 0; t < net->n_tensors; ++t) {
    if (!net->data[t]) return set_err(err_msg, err_cap, TN_EINVAL, "tensor data pointer is NULL");
    int64_t size = 1;
    for (int b : st.bonds[t]) size *= st.bond_dims[b];
    for (int64_t i = 0; i < size; ++i)
      if (!std::isfinite(net->data[t][i]))
        return set_err(err_msg, err_cap, TN_ENONFINITE, "tensor " + std::to_string(t) + " has a non-finite entry");
  }
  if (tree->n_ops < 0 || (tree->n_ops > 0 && !tree->ops)) return set_err(err_msg, err_cap, TN_EINVAL, "bad tree");
  std::vector<int32_t> ops(tree->ops, tree->ops + 4 * (size_t)tree->n_ops);
  for (int32_t q = 0; q < tree->n_ops; ++q)
    if (ops[4 * q] == 1) ops[4 * q + 3] = -1;
  tnp::Plan plan;
  std::string e = tnp::build_plan(st, ops, tree->n_inputs, chi, TN_F64, &plan);
  if (!e.empty()) return set_err(err_msg, err_cap, TN_EFORMAT, "tree: " + e);

  // carve the static scratch: inputs | arena | scratch words (all 256-byte aligned)
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t in_bytes = up(sizeof(double) * (size_t)std::max<int64_t>(st.in_total, 1));
  const size_t arena_bytes = up(sizeof(double) * (size_t)std::max<int64_t>(plan.arena_units, 1));
  const size_t word_bytes = up(sizeof(long long)) + up(sizeof(int)) + up(sizeof(int) * 64) +
                            up(sizeof(unsigned long long)) + up(sizeof(double)) + up(sizeof(int)) + up(sizeof(int));
  const size_t need = in_bytes + arena_bytes + word_bytes;
  if (need > kNoAllocBytes)
    return set_err(err_msg, err_cap, TN_ENOMEM,
                   "this instance needs " + std::to_string(need) + " bytes of device scratch; the static scratch of "
                   "tn_contract_approx_noalloc holds " + std::to_string(kNoAllocBytes) + " bytes");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_err(err_msg, err_cap, TN_ECUDA, "no current CUDA device");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
      void* p = nullptr;
      cudaError_t ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (ce != cudaSuccess || !p)
        return set_err(err_msg, err_cap, TN_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
      g_ptr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_ptr[dev]);
  }
  double* inbuf = reinterpret_cast<double*>(base);
  double* arena = reinterpret_cast<double*>(base + in_bytes);
  unsigned char* w = base + in_bytes + arena_bytes;
  long long* expo = reinterpret_cast<long long*>(w);
  w += up(sizeof(long long));
  int* status = reinterpret_cast<int*>(w);
  w += up(sizeof(int));
  int* jac_ws = reinterpret_cast<int*>(w);
  w += up(sizeof(int) * 64);
  unsigned long long* maxbits = reinterpret_cast<unsigned long long*>(w);
  w += up(sizeof(unsigned long long));
  double* out_log = reinterpret_cast<double*>(w);
  w += up(sizeof(double));
  int* out_sign = reinterpret_cast<int*>(w);
  w += up(sizeof(int));
  int* tc_err = reinterpret_cast<int*>(w);

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t ce = cudaSuccess;
  for (int t = 0; t < net->n_tensors && ce == cudaSuccess; ++t) {
    int64_t size = 1;
    for (int b : st.bonds[t]) size *= st.bond_dims[b];
    ce = cudaMemcpyAsync(inbuf + st.in_off[t], net->data[t], sizeof(double) * size, cudaMemcpyHostToDevice, s);
  }
  // the array keeps the previous call's contents: zero what must start at zero
  if (ce == cudaSuccess) ce = cudaMemsetAsync(expo, 0, sizeof(long long), s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(tc_err, 0, sizeof(int), s);
  if (ce != cudaSuccess) return set_err(err_msg, err_cap, TN_ECUDA, std::string("upload: ") + cudaGetErrorString(ce));
  tnx::ExecEnv env;
  env.inbuf = inbuf;
  env.arena = arena;
  env.batch = 1;
  env.ds = tnk::DevState{expo, status};
  env.jac_ws = jac_ws;
  env.maxbits = maxbits;
  env.out_log = out_log;
  env.out_sign = out_sign;
  env.tc_err = tc_err;
  for (const tnp::Step& stp : plan.steps) {
    ce = tnx::exec_step(stp, env, s);
    if (ce != cudaSuccess) return set_err(err_msg, err_cap, TN_ECUDA, std::string("launch: ") + cudaGetErrorString(ce));
  }
  double lg = 0.0;
  int sg = 0, stv = 0;
  ce = cudaMemcpyAsync(&lg, out_log, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&sg, out_sign, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&stv, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return set_err(err_msg, err_cap, TN_ECUDA, std::string("contraction: ") + cudaGetErrorString(ce));
  if (stv == -9) return set_err(err_msg, err_cap, TN_ENOCONV, "Jacobi SVD did not converge");
  if (stv != 0) return set_err(err_msg, err_cap, TN_ENONFINITE, "non-finite intermediate");
  *logabsz_out = lg;
  *sign_out = sg;
  return set_err(err_msg, err_cap, TN_OK, "");
}
