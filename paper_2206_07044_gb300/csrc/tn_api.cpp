// C ABI (include/tn.h): contexts, network / tree loading and validation,
// batching of instances, and the step executor that launches the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <fstream>
#include <initializer_list>
#include <map>
#include <memory>
#include <sstream>
#include <string>
#include <tuple>
#include <unordered_set>
#include <vector>

#include "../../include/tn.h"
#include "tn_exec.h"
#include "tn_kernels.h"
#include "tn_plan.h"
#include "tn_tune.h"

namespace {

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct NetRec {
  tnp::Structure st;
  double* d_data = nullptr;
  uint64_t hash = 0;
};

struct InstRec {
  int net = -1;
  int n_inputs = 0;
  std::vector<int32_t> ops;
  uint64_t hash = 0;  // structure + tree
};

struct PlanKey {
  uint64_t hash;
  int chi, prec;
  int grad;  // 0: forward only; k >= 1: with the reverse pass, checkpointed in k segments
  int gauge; // tree-gauge distance of the compressions (-1: plain Q-form)
  bool operator<(const PlanKey& o) const {
    return std::tie(hash, chi, prec, grad, gauge) < std::tie(o.hash, o.chi, o.prec, o.grad, o.gauge);
  }
};

struct CachedPlan {
  int inst_proto;  // instance whose structure/tree built the plan (for exact equality checks)
  tnp::Plan plan;
};

// A captured schedule: one plan, one ordered member list, one set of device buffers.
struct GraphKey {
  uint64_t plan_serial, buf_gen;
  std::vector<int> members;
  bool operator<(const GraphKey& o) const {
    return std::tie(plan_serial, buf_gen, members) < std::tie(o.plan_serial, o.buf_gen, o.members);
  }
};
struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  bool failed = false;  // capture was refused: this key always runs eagerly
};

const char* kFamily[] = {"permute", "gemm_f64",   "qr_f64",     "jacobi_f64",  "select_scale", "rescale",
                         "finalize", "to_f32",     "jacobi_f32", "to_f64",      "copy",         "apply_q_f64",
                         "gemm_tc",  "scale_pow2", "final_grad", "svd_factors", "svd_adj_core", "copy2d",
                         "mark_active"};
static_assert(sizeof(kFamily) / sizeof(kFamily[0]) == tnp::kNumStepKinds, "one family name per step kind");
constexpr int kNumFamily = tnp::kNumStepKinds;

}  // namespace

struct tn_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  std::vector<NetRec> nets;
  std::vector<InstRec> insts;
  std::map<PlanKey, CachedPlan> plans;
  double* arena = nullptr;
  size_t arena_bytes = 0;
  double* inbuf = nullptr;
  size_t inbuf_bytes = 0;
  // reverse pass: adjoints of the inputs (input-block layout) and the rescale exponent tape
  double* ginbuf = nullptr;
  size_t ginbuf_bytes = 0;
  int* etape = nullptr;
  size_t etape_bytes = 0;
  // per-instance scratch
  int scratch_batch = 0;
  long long* expo = nullptr;
  int* status = nullptr;
  int* jac_ws = nullptr;
  unsigned long long* maxbits = nullptr;
  double* out_log = nullptr;
  int* out_sign = nullptr;
  // side stream for steps that may overlap the main stream, and fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  unsigned long long* sweeps = nullptr;  // [2] device: Jacobi sweeps run (FP32, FP64) while profiling
  int* tc_err = nullptr;                 // device: set by a tensor-core GEMM whose bounded wait ran out
  // CUDA graphs: a schedule runs eagerly on its first call (warming every launch
  // configuration), is captured on the second and replayed from then on
  int graph_mode = 1;
  int grad_segments = 0;  // tn_grad: 0 = choose from free device memory, k >= 1 = k segments
  int gauge_r = -1;       // compressions in the tree gauge of this distance (-1: plain Q-form)
  double tape_budget = 0.0;  // tn_grad: tape bytes before checkpointing (0: half the free device memory)
  int opt_max_sweeps = 0;    // > 0: FP64 Jacobi sweep cap (tests of the bounded loop)
  bool opt_tc_give_up = false;  // tests: tensor-core GEMM pipeline waits give up at once
  std::string tuner_cache;      // autotuner cache file ("" = none)
  uint64_t plan_serial = 0;
  uint64_t buf_gen = 0;  // bumped whenever a buffer a captured graph points into moves
  cudaStream_t cap = nullptr;
  std::map<GraphKey, GraphRec> graphs;
  int64_t graph_captured = 0, graph_replays = 0, graph_refused = 0;
  // concurrent groups: instances whose trees differ run as parallel branches
  // (one stream pair per group) over slices of one set of buffers
  struct Multi {
    double* arena = nullptr;
    size_t arena_bytes = 0;
    double* inbuf = nullptr;
    size_t inbuf_bytes = 0;
    long long* expo = nullptr;
    int* status = nullptr;
    int* jac_ws = nullptr;
    unsigned long long* maxbits = nullptr;
    double* out_log = nullptr;
    int* out_sign = nullptr;
    int* tc_err = nullptr;
    int cap_inst = 0, cap_groups = 0;
    std::vector<cudaStream_t> streams, sides;
    std::vector<cudaEvent_t> ev_fork, ev_join, ev_done;
    cudaEvent_t ev_start = nullptr;
    uint64_t gen = 0;
    std::map<std::vector<int>, GraphRec> graphs;  // key: (plan serial, n members, members...) per group, then gen
  } multi;
  int64_t concurrent_runs = 0;
  int concurrent_groups = 1;  // run groups with different trees as concurrent branches
  int split_batches = 1;      // > 1: each group's batch runs as this many concurrent sub-batches
  // tn_debug_tensor: where the last partial run stopped (its plan, members and
  // buffer generation), so that a later call with a later stop continues from there
  uint64_t dbg_serial = 0, dbg_gen = 0;
  std::vector<int> dbg_members;
  int dbg_stop = -2;  // -2: no partial run to continue
  // profiling
  bool profile = false;
  unsigned long long prof_sweeps[2] = {0, 0};
  int64_t prof_launches[kNumFamily] = {0};
  double prof_ms[kNumFamily] = {0};
};

namespace {

int fail(tn_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(tn_ctx* c, cudaError_t e, const char* what) {
  return fail(c, TN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T>
cudaError_t ensure(T** p, size_t* have, size_t need) {
  if (*have >= need && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), need);
  if (e == cudaSuccess) *have = need;
  return e;
}

int load_structure(tn_ctx* c, int32_t n_bonds, const int64_t* bond_dims, int32_t n_tensors,
                   const int32_t* ndims, const int32_t* bond_ids, tnp::Structure* st) {
  std::string msg;
  const int rc = tnx::check_structure(n_bonds, bond_dims, n_tensors, ndims, bond_ids, st, &msg);
  return rc == TN_OK ? TN_OK : fail(c, rc, msg);
}

uint64_t structure_hash(const tnp::Structure& st) {
  uint64_t h = 1469598103934665603ull;
  size_t nb = st.bond_dims.size();
  h = fnv(h, &nb, sizeof nb);
  h = fnv(h, st.bond_dims.data(), nb * sizeof(int64_t));
  for (auto& bl : st.bonds) {
    size_t n = bl.size();
    h = fnv(h, &n, sizeof n);
    h = fnv(h, bl.data(), n * sizeof(int));
  }
  return h;
}

int add_network(tn_ctx* c, tnp::Structure&& st, const double* const* data, bool data_on_device,
                const std::vector<double>* flat_host, int* net_id) {
  NetRec rec;
  rec.st = std::move(st);
  rec.hash = structure_hash(rec.st);
  const int nt = (int)rec.st.bonds.size();
  // finiteness check on host data
  auto tsize = [&](int t) {
    int64_t s = 1;
    for (int b : rec.st.bonds[t]) s *= rec.st.bond_dims[b];
    return s;
  };
  if (!data_on_device) {
    for (int t = 0; t < nt; ++t) {
      const double* d = flat_host ? flat_host->data() + rec.st.in_off[t] : data[t];
      if (!d) return fail(c, TN_EINVAL, "tensor data pointer is NULL");
      int64_t s = tsize(t);
      for (int64_t i = 0; i < s; ++i)
        if (!std::isfinite(d[i]))
          return fail(c, TN_ENONFINITE, "tensor " + std::to_string(t) + " has a non-finite entry");
    }
  }
  DeviceGuard g(c->device);
  cudaError_t e = cudaMalloc(&rec.d_data, sizeof(double) * std::max<int64_t>(rec.st.in_total, 1));
  if (e != cudaSuccess) return fail(c, TN_ENOMEM, "cudaMalloc network data failed");
  cudaMemsetAsync(rec.d_data, 0, sizeof(double) * std::max<int64_t>(rec.st.in_total, 1), c->stream);
  if (flat_host) {
    e = cudaMemcpyAsync(rec.d_data, flat_host->data(), sizeof(double) * rec.st.in_total,
                        cudaMemcpyHostToDevice, c->stream);
  } else {
    for (int t = 0; t < nt && e == cudaSuccess; ++t)
      e = cudaMemcpyAsync(rec.d_data + rec.st.in_off[t], data[t], sizeof(double) * tsize(t),
                          data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFree(rec.d_data);
    return cuda_fail(c, e, "copy network data");
  }
  c->nets.push_back(std::move(rec));
  *net_id = (int)c->nets.size() - 1;
  return TN_OK;
}

int add_tree(tn_ctx* c, int net_id, int32_t n_inputs, int32_t n_ops, const int32_t* ops, int* inst_id) {
  if (net_id < 0 || net_id >= (int)c->nets.size()) return fail(c, TN_EINVAL, "unknown network id");
  if (n_ops < 0 || (n_ops > 0 && !ops)) return fail(c, TN_EINVAL, "bad ops");
  InstRec r;
  r.net = net_id;
  r.n_inputs = n_inputs;
  r.ops.assign(ops, ops + 4 * (size_t)n_ops);
  for (int32_t q = 0; q < n_ops; ++q)
    if (r.ops[4 * q] == 1) r.ops[4 * q + 3] = -1;
  std::string err = tnp::validate_tree(c->nets[net_id].st, r.ops, n_inputs);
  if (!err.empty()) return fail(c, TN_EFORMAT, "tree: " + err);
  uint64_t h = c->nets[net_id].hash;
  h = fnv(h, &n_inputs, sizeof n_inputs);
  h = fnv(h, r.ops.data(), r.ops.size() * sizeof(int32_t));
  r.hash = h;
  c->insts.push_back(std::move(r));
  *inst_id = (int)c->insts.size() - 1;
  return TN_OK;
}

bool same_group(const tn_ctx* c, int a, int b) {
  const InstRec &x = c->insts[a], &y = c->insts[b];
  if (x.hash != y.hash || x.ops != y.ops || x.n_inputs != y.n_inputs) return false;
  const tnp::Structure &s = c->nets[x.net].st, &t = c->nets[y.net].st;
  return s.bond_dims == t.bond_dims && s.bonds == t.bonds;
}

int ensure_scratch(tn_ctx* c, int batch) {
  if (c->scratch_batch >= batch) return TN_OK;
  // null every pointer once freed: a failed allocation below must not leave
  // one that the next call (or tn_destroy) would free a second time
  for (void** p : {(void**)&c->expo, (void**)&c->status, (void**)&c->jac_ws, (void**)&c->maxbits,
                   (void**)&c->out_log, (void**)&c->out_sign}) {
    cudaFree(*p);
    *p = nullptr;
  }
  c->scratch_batch = 0;
  if (cudaMalloc(&c->expo, sizeof(long long) * batch) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(int) * batch) != cudaSuccess ||
      cudaMalloc(&c->jac_ws, sizeof(int) * 64 * batch) != cudaSuccess ||
      cudaMalloc(&c->maxbits, sizeof(unsigned long long) * batch) != cudaSuccess ||
      cudaMalloc(&c->out_log, sizeof(double) * batch) != cudaSuccess ||
      cudaMalloc(&c->out_sign, sizeof(int) * batch) != cudaSuccess)
    return fail(c, TN_ENOMEM, "scratch allocation failed");
  c->scratch_batch = batch;
  return TN_OK;
}

// grad: 0 forward only, k >= 1 with the reverse pass in k checkpointed segments
const tnp::Plan* get_plan(tn_ctx* c, int inst, int chi, int prec, int* rc, int grad = 0) {
  PlanKey key{c->insts[inst].hash, chi, prec, grad, grad > 0 ? -1 : c->gauge_r};
  auto it = c->plans.find(key);
  if (it != c->plans.end() && same_group(c, it->second.inst_proto, inst)) return &it->second.plan;
  CachedPlan cp;
  cp.inst_proto = inst;
  const InstRec& r = c->insts[inst];
  std::string err = tnp::build_plan(c->nets[r.net].st, r.ops, r.n_inputs, chi, prec, &cp.plan, grad > 0,
                                    grad > 0 ? grad : 1, grad > 0 ? -1 : c->gauge_r);
  if (!err.empty()) {
    *rc = fail(c, TN_EFORMAT, "plan: " + err);
    return nullptr;
  }
  cp.plan.serial = ++c->plan_serial;
  if (it != c->plans.end()) {
    // the cached plan of this key is replaced: its captured graphs can never run again
    const uint64_t old_serial = it->second.plan.serial;
    for (auto g = c->graphs.begin(); g != c->graphs.end();) {
      if (g->first.plan_serial == old_serial) {
        if (g->second.exec) cudaGraphExecDestroy(g->second.exec);
        g = c->graphs.erase(g);
      } else {
        ++g;
      }
    }
  }
  auto res = c->plans.insert_or_assign(key, std::move(cp));
  return &res.first->second.plan;
}

// Forget every captured graph (a buffer they point into has moved).
void drop_graphs(tn_ctx* c) {
  for (auto& g : c->graphs)
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
  c->graphs.clear();
  ++c->buf_gen;
}

// Capture one pass of `enqueue` on the context's capture stream and
// instantiate it.  On any refusal the key is marked failed and keeps running
// eagerly (the same kernels, launched one by one).
template <typename F>
void capture_graph(tn_ctx* c, GraphRec* gr, F& enqueue) {
  gr->failed = true;
  if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ++c->graph_refused;
    return;
  }
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    ++c->graph_refused;
    return;
  }
  const std::string saved = c->err;
  const int rc = enqueue(c->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  c->err = saved;
  cudaGraphExec_t ex = nullptr;
  if (rc == TN_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&ex, g, 0);
  if (g) cudaGraphDestroy(g);
  if (rc != TN_OK || e != cudaSuccess || !ex) {
    cudaGetLastError();
    ++c->graph_refused;
    return;
  }
  gr->exec = ex;
  gr->failed = false;
  ++c->graph_captured;
}

// Run the plan on a batch.  With stop_op >= 0, only the steps of tree ops
// 0..stop_op run (no final read-out) and the call returns after syncing; the
// arena then holds every tensor alive after that op.  resume_after >= -1
// (with stop_op >= 0): the device already holds the state after tree op
// resume_after of this same plan and batch, so the input gather and the steps
// of ops 0..resume_after are skipped.
int run_group(tn_ctx* c, const tnp::Plan& plan, const std::vector<int>& members, double* logabs,
              int* sign, int stop_op = -1, int resume_after = -2) {
  const int batch = (int)members.size();
  if (batch > 65535) return fail(c, TN_EINVAL, "more than 65535 instances in one batch");
  c->dbg_stop = -2;  // any run overwrites the state a partial debug run left
  const tnp::Structure& st = c->nets[c->insts[members[0]].net].st;
  cudaError_t e;
  const void* before[5] = {c->arena, c->inbuf, c->expo, c->ginbuf, c->etape};
  const size_t arena_need = sizeof(double) * (size_t)std::max<int64_t>(plan.arena_units, 1) * batch;
  if ((e = ensure(&c->arena, &c->arena_bytes, arena_need)) != cudaSuccess)
    return fail(c, TN_ENOMEM, "arena allocation of " + std::to_string(arena_need) + " bytes failed");
  const size_t in_need = sizeof(double) * (size_t)std::max<int64_t>(st.in_total, 1) * batch;
  if ((e = ensure(&c->inbuf, &c->inbuf_bytes, in_need)) != cudaSuccess)
    return fail(c, TN_ENOMEM, "input buffer allocation failed");
  if (plan.grad) {
    const size_t g_need = sizeof(double) * (size_t)std::max<int64_t>(plan.in_total, 1) * batch;
    if ((e = ensure(&c->ginbuf, &c->ginbuf_bytes, g_need)) != cudaSuccess)
      return fail(c, TN_ENOMEM, "input-adjoint buffer allocation failed");
    const size_t t_need = sizeof(int) * (size_t)std::max(plan.n_slots, 1) * batch;
    if ((e = ensure(&c->etape, &c->etape_bytes, t_need)) != cudaSuccess)
      return fail(c, TN_ENOMEM, "exponent tape allocation failed");
  }
  int rc = ensure_scratch(c, batch);
  if (rc != TN_OK) return rc;
  if (!c->side) {
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return fail(c, TN_ECUDA, "side stream creation failed");
  }
  if (!c->tc_err && cudaMalloc(&c->tc_err, sizeof(int)) != cudaSuccess) return fail(c, TN_ENOMEM, "error word");
  if (c->profile && !c->sweeps && cudaMalloc(&c->sweeps, 2 * sizeof(unsigned long long)) != cudaSuccess)
    return fail(c, TN_ENOMEM, "profiling counters");
  if (before[0] != c->arena || before[1] != c->inbuf || before[2] != c->expo || before[3] != c->ginbuf ||
      before[4] != c->etape)
    drop_graphs(c);
  tnx::ExecEnv env;
  env.inbuf = c->inbuf;
  env.arena = c->arena;
  env.ginbuf = c->ginbuf;
  env.batch = batch;
  env.ds = tnk::DevState{c->expo, c->status};
  env.jac_ws = c->jac_ws;
  env.maxbits = c->maxbits;
  env.out_log = c->out_log;
  env.out_sign = c->out_sign;
  env.tc_err = c->tc_err;
  env.etape = c->etape;
  env.sweeps32 = c->profile ? c->sweeps : nullptr;
  env.sweeps64 = c->profile ? c->sweeps + 1 : nullptr;
  env.jac_max_sweeps = c->opt_max_sweeps;
  env.tc_give_up = c->opt_tc_give_up;

  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
  std::vector<int> ev_family;
  // Every stream operation of one pass (gather, resets, steps), issued on s0.
  // Under capture nothing runs; the side stream joins the capture through the
  // fork event and is joined back before the pass ends.
  auto enqueue = [&](cudaStream_t s0) -> int {
  cudaStream_t s = s0;
  cudaError_t e = cudaSuccess;
  const bool resuming = stop_op >= 0 && resume_after >= -1;
  for (int b = 0; b < batch && e == cudaSuccess && !resuming; ++b) {
    const NetRec& nr = c->nets[c->insts[members[b]].net];
    e = cudaMemcpyAsync(c->inbuf + (size_t)b * st.in_total, nr.d_data, sizeof(double) * st.in_total,
                        cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess && !resuming) e = cudaMemsetAsync(c->expo, 0, sizeof(long long) * batch, s);
  if (e == cudaSuccess && !resuming) e = cudaMemsetAsync(c->status, 0, sizeof(int) * batch, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->tc_err, 0, sizeof(int), s);
  if (e == cudaSuccess && c->profile) e = cudaMemsetAsync(c->sweeps, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "gather inputs");
  bool side_open = false;
  for (const tnp::Step& stp : plan.steps) {
    if (stop_op >= 0 && (stp.op_index > stop_op || stp.kind == tnp::ST_FINAL)) break;
    if (resuming && stp.op_index <= resume_after) continue;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stp.join && side_open) {
      cudaStreamWaitEvent(s, c->ev_join, 0);
      side_open = false;
    }
    // a side-lane step forks from the main stream; profiling keeps everything on one stream
    const bool on_side = stp.lane == 1 && !c->profile;
    cudaStream_t ms = s;
    if (on_side) {
      cudaEventRecord(c->ev_fork, s);
      cudaStreamWaitEvent(c->side, c->ev_fork, 0);
      s = c->side;
    }
    if (c->profile) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
    }
    e = tnx::exec_step(stp, env, s);
    if (e != cudaSuccess) {
      return fail(c, TN_ECUDA, std::string("launch of ") + kFamily[stp.kind] + " (tree op " +
                                   std::to_string(stp.op_index) + ") failed: " + cudaGetErrorString(e));
    }
    if (c->profile) {
      cudaEventRecord(e1, s);
      evs.push_back({e0, e1});
      ev_family.push_back(stp.kind);
    }
    if (on_side) {
      cudaEventRecord(c->ev_join, s);
      s = ms;
      side_open = true;
    }
  }
  if (side_open) cudaStreamWaitEvent(s, c->ev_join, 0);
  return TN_OK;
  };

  cudaStream_t s = c->stream;
  const bool graphable = c->graph_mode && !c->profile && stop_op < 0;
  GraphRec* gr = nullptr;
  if (graphable) {
    GraphKey key{plan.serial, c->buf_gen, members};
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
      c->graphs.emplace(key, GraphRec{});  // first call: eager; captured on the next
    } else {
      gr = &it->second;
      if (!gr->exec && !gr->failed) capture_graph(c, gr, enqueue);
    }
  }
  if (gr && gr->exec) {
    e = cudaGraphLaunch(gr->exec, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    ++c->graph_replays;
  } else {
    rc = enqueue(s);
    if (rc != TN_OK) return rc;
  }
  if (stop_op >= 0) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "partial run");
    return TN_OK;
  }
  std::vector<double> hl(batch);
  std::vector<int> hs(batch), hst(batch);
  e = cudaMemcpyAsync(hl.data(), c->out_log, sizeof(double) * batch, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), c->out_sign, sizeof(int) * batch, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), c->status, sizeof(int) * batch, cudaMemcpyDeviceToHost, s);
  unsigned long long hsw[2] = {0, 0};
  int htc = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&htc, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && c->profile)
    e = cudaMemcpyAsync(hsw, c->sweeps, sizeof(hsw), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "contraction");
  c->prof_sweeps[0] += hsw[0];
  c->prof_sweeps[1] += hsw[1];
  if (htc) return fail(c, TN_ETIMEOUT, "a tensor-core GEMM's bounded wait ran out");
  for (size_t q = 0; q < evs.size(); ++q) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, evs[q].first, evs[q].second);
    c->prof_ms[ev_family[q]] += ms;
    c->prof_launches[ev_family[q]] += 1;
    cudaEventDestroy(evs[q].first);
    cudaEventDestroy(evs[q].second);
  }
  int worst = 0;
  for (int b = 0; b < batch; ++b) {
    logabs[b] = hl[b];
    sign[b] = hs[b];
    if (hst[b] != 0 && worst == 0) worst = hst[b];
  }
  if (worst == -9) return fail(c, TN_ENOCONV, "Jacobi SVD did not converge");
  if (worst == -7) return fail(c, TN_ENONFINITE, "non-finite intermediate");
  if (worst != 0) return fail(c, TN_ECUDA, "device status " + std::to_string(worst));
  return TN_OK;
}

// Forward passes of several groups (instances whose network structure and
// tree differ between groups) as concurrent branches: every group gets a
// slice of one arena / input block / scratch set and its own stream pair; the
// main stream forks to all of them and joins them back.  With graph mode the
// whole multi-group pass is captured on the second call (one graph whose
// branches are the groups' schedules) and replayed after.  The kernels, shapes
// and data of each group are those of run_group, so results are identical to
// running the groups one after the other.
int run_groups_concurrent(tn_ctx* c, const std::vector<const tnp::Plan*>& plans,
                          const std::vector<std::vector<int>>& groups, std::vector<std::vector<double>>* logabs,
                          std::vector<std::vector<int>>* sign) {
  auto& M = c->multi;
  const int G = (int)groups.size();
  c->dbg_stop = -2;
  std::vector<int64_t> a_off(G), i_off(G), o_off(G);
  int64_t a_tot = 0, i_tot = 0, o_tot = 0;
  for (int g = 0; g < G; ++g) {
    const int batch = (int)groups[g].size();
    if (batch > 65535) return fail(c, TN_EINVAL, "more than 65535 instances in one batch");
    const tnp::Structure& st = c->nets[c->insts[groups[g][0]].net].st;
    a_off[g] = a_tot;
    i_off[g] = i_tot;
    o_off[g] = o_tot;
    a_tot += (std::max<int64_t>(plans[g]->arena_units, 1) * batch + 31) / 32 * 32;
    i_tot += (std::max<int64_t>(st.in_total, 1) * batch + 31) / 32 * 32;
    o_tot += batch;
  }
  cudaError_t e;
  const void* before[3] = {M.arena, M.inbuf, M.expo};
  if ((e = ensure(&M.arena, &M.arena_bytes, sizeof(double) * (size_t)a_tot)) != cudaSuccess)
    return fail(c, TN_ENOMEM, "arena allocation of " + std::to_string(8 * a_tot) + " bytes failed");
  if ((e = ensure(&M.inbuf, &M.inbuf_bytes, sizeof(double) * (size_t)i_tot)) != cudaSuccess)
    return fail(c, TN_ENOMEM, "input buffer allocation failed");
  if (M.cap_inst < o_tot || M.cap_groups < G) {
    for (void** p : {(void**)&M.expo, (void**)&M.status, (void**)&M.jac_ws, (void**)&M.maxbits,
                     (void**)&M.out_log, (void**)&M.out_sign, (void**)&M.tc_err}) {
      cudaFree(*p);
      *p = nullptr;
    }
    M.cap_inst = M.cap_groups = 0;
    const size_t n = (size_t)o_tot;
    if (cudaMalloc(&M.expo, sizeof(long long) * n) != cudaSuccess ||
        cudaMalloc(&M.status, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(&M.jac_ws, sizeof(int) * 64 * n) != cudaSuccess ||
        cudaMalloc(&M.maxbits, sizeof(unsigned long long) * n) != cudaSuccess ||
        cudaMalloc(&M.out_log, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&M.out_sign, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(&M.tc_err, sizeof(int) * (size_t)G) != cudaSuccess)
      return fail(c, TN_ENOMEM, "scratch allocation failed");
    M.cap_inst = (int)o_tot;
    M.cap_groups = G;
  }
  if (before[0] != M.arena || before[1] != M.inbuf || before[2] != M.expo) {
    for (auto& gx : M.graphs)
      if (gx.second.exec) cudaGraphExecDestroy(gx.second.exec);
    M.graphs.clear();
    ++M.gen;
  }
  while ((int)M.streams.size() < G) {
    cudaStream_t a = nullptr, b = nullptr;
    cudaEvent_t f = nullptr, j = nullptr, d = nullptr;
    if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d, cudaEventDisableTiming) != cudaSuccess)
      return fail(c, TN_ECUDA, "stream creation failed");
    M.streams.push_back(a);
    M.sides.push_back(b);
    M.ev_fork.push_back(f);
    M.ev_join.push_back(j);
    M.ev_done.push_back(d);
  }
  if (!M.ev_start && cudaEventCreateWithFlags(&M.ev_start, cudaEventDisableTiming) != cudaSuccess)
    return fail(c, TN_ECUDA, "event creation failed");

  auto enqueue = [&](cudaStream_t s0) -> int {
    if (cudaEventRecord(M.ev_start, s0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "fork");
    for (int g = 0; g < G; ++g) {
      const tnp::Plan& plan = *plans[g];
      const std::vector<int>& members = groups[g];
      const int batch = (int)members.size();
      const tnp::Structure& st = c->nets[c->insts[members[0]].net].st;
      tnx::ExecEnv env;
      env.inbuf = M.inbuf + i_off[g];
      env.arena = M.arena + a_off[g];
      env.batch = batch;
      env.ds = tnk::DevState{M.expo + o_off[g], M.status + o_off[g]};
      env.jac_ws = M.jac_ws + 64 * o_off[g];
      env.maxbits = M.maxbits + o_off[g];
      env.out_log = M.out_log + o_off[g];
      env.out_sign = M.out_sign + o_off[g];
      env.tc_err = M.tc_err + g;
      env.jac_max_sweeps = c->opt_max_sweeps;
      env.tc_give_up = c->opt_tc_give_up;
      cudaStream_t s = M.streams[g];
      cudaError_t e2 = cudaStreamWaitEvent(s, M.ev_start, 0);
      for (int b = 0; b < batch && e2 == cudaSuccess; ++b) {
        const NetRec& nr = c->nets[c->insts[members[b]].net];
        e2 = cudaMemcpyAsync(env.inbuf + (size_t)b * st.in_total, nr.d_data, sizeof(double) * st.in_total,
                             cudaMemcpyDeviceToDevice, s);
      }
      if (e2 == cudaSuccess) e2 = cudaMemsetAsync(env.ds.expo, 0, sizeof(long long) * batch, s);
      if (e2 == cudaSuccess) e2 = cudaMemsetAsync(env.ds.status, 0, sizeof(int) * batch, s);
      if (e2 == cudaSuccess) e2 = cudaMemsetAsync(env.tc_err, 0, sizeof(int), s);
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "gather inputs");
      bool side_open = false;
      for (const tnp::Step& stp : plan.steps) {
        if (stp.join && side_open) {
          cudaStreamWaitEvent(s, M.ev_join[g], 0);
          side_open = false;
        }
        cudaStream_t ss = s;
        if (stp.lane == 1) {
          cudaEventRecord(M.ev_fork[g], s);
          cudaStreamWaitEvent(M.sides[g], M.ev_fork[g], 0);
          ss = M.sides[g];
        }
        e2 = tnx::exec_step(stp, env, ss);
        if (e2 != cudaSuccess)
          return fail(c, TN_ECUDA, std::string("launch of ") + kFamily[stp.kind] + " (tree op " +
                                       std::to_string(stp.op_index) + ") failed: " + cudaGetErrorString(e2));
        if (stp.lane == 1) {
          cudaEventRecord(M.ev_join[g], ss);
          side_open = true;
        }
      }
      if (side_open) cudaStreamWaitEvent(s, M.ev_join[g], 0);
      cudaEventRecord(M.ev_done[g], s);
      if (cudaStreamWaitEvent(s0, M.ev_done[g], 0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "join");
    }
    return TN_OK;
  };

  cudaStream_t s = c->stream;
  GraphRec* gr = nullptr;
  if (c->graph_mode) {
    std::vector<int> key;
    for (int g = 0; g < G; ++g) {
      key.push_back((int)plans[g]->serial);
      key.push_back((int)groups[g].size());
      key.insert(key.end(), groups[g].begin(), groups[g].end());
    }
    key.push_back((int)M.gen);
    auto it = M.graphs.find(key);
    if (it == M.graphs.end()) {
      M.graphs.emplace(key, GraphRec{});  // first call: eager (still concurrent); captured on the next
    } else {
      gr = &it->second;
      if (!gr->exec && !gr->failed) capture_graph(c, gr, enqueue);
    }
  }
  if (gr && gr->exec) {
    e = cudaGraphLaunch(gr->exec, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    ++c->graph_replays;
  } else {
    const int rc = enqueue(s);
    if (rc != TN_OK) return rc;
  }
  ++c->concurrent_runs;
  std::vector<double> hl(o_tot);
  std::vector<int> hs(o_tot), hst(o_tot), htc(G);
  e = cudaMemcpyAsync(hl.data(), M.out_log, sizeof(double) * o_tot, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), M.out_sign, sizeof(int) * o_tot, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), M.status, sizeof(int) * o_tot, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(htc.data(), M.tc_err, sizeof(int) * G, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "contraction");
  for (int g = 0; g < G; ++g)
    if (htc[g]) return fail(c, TN_ETIMEOUT, "a tensor-core GEMM's bounded wait ran out");
  int worst = 0;
  logabs->assign(G, {});
  sign->assign(G, {});
  for (int g = 0; g < G; ++g)
    for (size_t b = 0; b < groups[g].size(); ++b) {
      (*logabs)[g].push_back(hl[o_off[g] + b]);
      (*sign)[g].push_back(hs[o_off[g] + b]);
      if (hst[o_off[g] + b] != 0 && worst == 0) worst = hst[o_off[g] + b];
    }
  if (worst == -9) return fail(c, TN_ENOCONV, "Jacobi SVD did not converge");
  if (worst == -7) return fail(c, TN_ENONFINITE, "non-finite intermediate");
  if (worst != 0) return fail(c, TN_ECUDA, "device status " + std::to_string(worst));
  return TN_OK;
}

bool read_file(const char* path, std::string* out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  std::ostringstream ss;
  ss << f.rdbuf();
  *out = ss.str();
  return true;
}

}  // namespace

namespace {

// Time `launch` (one launch per call) on stream s: one untimed launch, then the
// fastest of two timed ones (ms); a negative value if a launch failed.
template <typename F>
double time_launch(cudaStream_t s, F launch) {
  if (launch() != cudaSuccess) {
    cudaGetLastError();
    return -1.0;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = -1.0;
  for (int r = 0; r < 2; ++r) {
    cudaEventRecord(e0, s);
    const cudaError_t e = launch();
    cudaEventRecord(e1, s);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      best = -1.0;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0 || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

void fill_random(std::vector<double>& h, uint64_t seed) {
  uint64_t x = seed * 0x9E3779B97F4A7C15ull + 1;
  for (double& v : h) {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    v = (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

struct TuneKey {
  int kernel, m, n, k;
  bool operator<(const TuneKey& o) const {
    return std::tie(kernel, m, n, k) < std::tie(o.kernel, o.m, o.n, o.k);
  }
};

}  // namespace

extern "C" {

const char* tn_version(void) { return "tn-gb300 0.1"; }

void tn_options_default(tn_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->struct_size = (int32_t)sizeof(tn_options);
  opt->graph_mode = 1;
}

int tn_create(tn_ctx** out, int device, const tn_options* opt) {
  if (!out) return TN_EINVAL;
  *out = nullptr;
  tn_options o;
  tn_options_default(&o);
  if (opt) {
    if (opt->struct_size < (int32_t)sizeof(tn_options)) return TN_EINVAL;
    o = *opt;
  }
  if (o.graph_mode < 0 || o.graph_mode > 1 || o.grad_segments < 0 || o.debug_max_sweeps < 0 ||
      !(o.tape_budget_bytes >= 0.0) || o.debug_tc_give_up < 0 || o.debug_tc_give_up > 1 ||
      o.sequential_groups < 0 || o.sequential_groups > 1 || o.split_batches < 0 || o.split_batches > 64)
    return TN_EINVAL;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TN_ECUDA;
  tn_ctx* c = new (std::nothrow) tn_ctx();
  if (!c) return TN_ENOMEM;
  c->device = device;
  c->graph_mode = o.graph_mode;
  c->grad_segments = o.grad_segments;
  c->tape_budget = o.tape_budget_bytes;
  c->opt_max_sweeps = o.debug_max_sweeps;
  c->opt_tc_give_up = o.debug_tc_give_up != 0;
  c->concurrent_groups = o.sequential_groups ? 0 : 1;
  c->split_batches = o.split_batches > 0 ? o.split_batches : 1;
  if (o.tuner_cache && *o.tuner_cache) {
    c->tuner_cache = o.tuner_cache;
    DeviceGuard g(device);
    const std::string e = tnk::tune_load(c->tuner_cache);
    if (!e.empty()) {
      delete c;
      return TN_EFORMAT;
    }
  }
  *out = c;
  return TN_OK;
}

void tn_destroy(tn_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  for (auto& n : c->nets) cudaFree(n.d_data);
  cudaFree(c->arena);
  cudaFree(c->inbuf);
  cudaFree(c->ginbuf);
  cudaFree(c->etape);
  cudaFree(c->expo);
  cudaFree(c->status);
  cudaFree(c->jac_ws);
  cudaFree(c->maxbits);
  cudaFree(c->out_log);
  cudaFree(c->out_sign);
  cudaFree(c->sweeps);
  cudaFree(c->tc_err);
  for (auto& gx : c->graphs)
    if (gx.second.exec) cudaGraphExecDestroy(gx.second.exec);
  {
    auto& M = c->multi;
    for (auto& gx : M.graphs)
      if (gx.second.exec) cudaGraphExecDestroy(gx.second.exec);
    cudaFree(M.arena);
    cudaFree(M.inbuf);
    cudaFree(M.expo);
    cudaFree(M.status);
    cudaFree(M.jac_ws);
    cudaFree(M.maxbits);
    cudaFree(M.out_log);
    cudaFree(M.out_sign);
    cudaFree(M.tc_err);
    for (auto x : M.streams) cudaStreamDestroy(x);
    for (auto x : M.sides) cudaStreamDestroy(x);
    for (auto x : M.ev_fork) cudaEventDestroy(x);
    for (auto x : M.ev_join) cudaEventDestroy(x);
    for (auto x : M.ev_done) cudaEventDestroy(x);
    if (M.ev_start) cudaEventDestroy(M.ev_start);
  }
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

int tn_set_graph_mode(tn_ctx* c, int mode) {
  if (!c || mode < 0 || mode > 1) return fail(c, TN_EINVAL, "graph mode must be 0 or 1");
  c->graph_mode = mode;
  return TN_OK;
}

int tn_graph_info(const tn_ctx* c, int64_t* captured, int64_t* replays, int64_t* refused) {
  if (!c) return TN_EINVAL;
  if (captured) *captured = c->graph_captured;
  if (replays) *replays = c->graph_replays;
  if (refused) *refused = c->graph_refused;
  return TN_OK;
}

int tn_set_stream(tn_ctx* c, void* stream) {
  if (!c) return TN_EINVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  return TN_OK;
}

int tn_load_network(tn_ctx* c, const tn_network_desc* d, int* net_id) {
  if (!c || !d || !net_id) return fail(c, TN_EINVAL, "NULL argument");
  if (!d->data) return fail(c, TN_EINVAL, "data is NULL");
  tnp::Structure st;
  int rc = load_structure(c, d->n_bonds, d->bond_dims, d->n_tensors, d->ndims, d->bond_ids, &st);
  if (rc != TN_OK) return rc;
  return add_network(c, std::move(st), d->data, false, nullptr, net_id);
}

int tn_load_network_file(tn_ctx* c, const char* path, int* net_id) {
  if (!c || !path || !net_id) return fail(c, TN_EINVAL, "NULL argument");
  std::string buf;
  if (!read_file(path, &buf)) return fail(c, TN_EINVAL, std::string("cannot read ") + path);
  size_t off = 0;
  auto need = [&](size_t n) { return off + n <= buf.size(); };
  auto rd64 = [&](int64_t* v) {
    if (!need(8)) return false;
    std::memcpy(v, buf.data() + off, 8);
    off += 8;
    return true;
  };
  if (!need(8) || std::memcmp(buf.data(), "TNNET1\0\0", 8) != 0) return fail(c, TN_EFORMAT, "not a TNNET1 file");
  off = 8;
  int64_t nb, nt;
  if (!rd64(&nb) || !rd64(&nt) || nb < 0 || nt < 1 || nb > (1 << 28) || nt > (1 << 28))
    return fail(c, TN_EFORMAT, "bad header");
  std::vector<int64_t> dims(nb);
  for (auto& d : dims)
    if (!rd64(&d)) return fail(c, TN_EFORMAT, "truncated bond sizes");
  std::vector<int32_t> ndims(nt), ids;
  for (int64_t t = 0; t < nt; ++t) {
    int64_t nd;
    if (!rd64(&nd) || nd < 0 || nd > tnk::kMaxDims) return fail(c, TN_EFORMAT, "bad tensor header");
    ndims[t] = (int32_t)nd;
    for (int64_t a = 0; a < nd; ++a) {
      int64_t b;
      if (!rd64(&b) || b < 0 || b >= nb) return fail(c, TN_EFORMAT, "bad bond id");
      ids.push_back((int32_t)b);
    }
  }
  tnp::Structure st;
  int rc = load_structure(c, (int32_t)nb, dims.data(), (int32_t)nt, ndims.data(), ids.data(), &st);
  if (rc != TN_OK) return rc;
  std::vector<double> flat((size_t)std::max<int64_t>(st.in_total, 1), 0.0);
  for (int64_t t = 0; t < nt; ++t) {
    int64_t s = 1;
    for (int b : st.bonds[t]) s *= st.bond_dims[b];
    if (!need(8 * (size_t)s)) return fail(c, TN_EFORMAT, "truncated tensor data");
    std::memcpy(flat.data() + st.in_off[t], buf.data() + off, 8 * (size_t)s);
    off += 8 * (size_t)s;
  }
  return add_network(c, std::move(st), nullptr, false, &flat, net_id);
}

int tn_set_network_data(tn_ctx* c, int net_id, const double* const* data, int on_device) {
  if (!c || !data) return fail(c, TN_EINVAL, "NULL argument");
  if (net_id < 0 || net_id >= (int)c->nets.size()) return fail(c, TN_EINVAL, "unknown network id");
  NetRec& nr = c->nets[net_id];
  DeviceGuard g(c->device);
  for (size_t t = 0; t < nr.st.bonds.size(); ++t) {
    int64_t s = 1;
    for (int b : nr.st.bonds[t]) s *= nr.st.bond_dims[b];
    if (!data[t]) return fail(c, TN_EINVAL, "tensor data pointer is NULL");
    if (!on_device)
      for (int64_t i = 0; i < s; ++i)
        if (!std::isfinite(data[t][i]))
          return fail(c, TN_ENONFINITE, "tensor " + std::to_string(t) + " has a non-finite entry");
    cudaError_t e = cudaMemcpyAsync(nr.d_data + nr.st.in_off[t], data[t], sizeof(double) * s,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set network data");
  }
  return TN_OK;
}

int tn_load_tree(tn_ctx* c, int net_id, const tn_tree_desc* d, int* inst_id) {
  if (!c || !d || !inst_id) return fail(c, TN_EINVAL, "NULL argument");
  return add_tree(c, net_id, d->n_inputs, d->n_ops, d->ops, inst_id);
}

int tn_load_tree_file(tn_ctx* c, int net_id, const char* path, int* inst_id) {
  if (!c || !path || !inst_id) return fail(c, TN_EINVAL, "NULL argument");
  std::string buf;
  if (!read_file(path, &buf)) return fail(c, TN_EINVAL, std::string("cannot read ") + path);
  std::istringstream in(buf);
  std::string line;
  int n_inputs = -1, ln = 0;
  std::vector<int32_t> ops;
  while (std::getline(in, line)) {
    ++ln;
    size_t h = line.find('#');
    if (h != std::string::npos) line.resize(h);
    std::istringstream ls(line);
    std::string tok;
    if (!(ls >> tok)) continue;
    if (tok == "tntree") continue;
    if (tok == "inputs") {
      if (!(ls >> n_inputs)) return fail(c, TN_EFORMAT, "tree line " + std::to_string(ln) + ": bad inputs");
    } else if (tok == "C") {
      int i, j, k;
      if (!(ls >> i >> j >> k)) return fail(c, TN_EFORMAT, "tree line " + std::to_string(ln) + ": bad C op");
      ops.insert(ops.end(), {0, i, j, k});
    } else if (tok == "S") {
      int i, j;
      if (!(ls >> i >> j)) return fail(c, TN_EFORMAT, "tree line " + std::to_string(ln) + ": bad S op");
      ops.insert(ops.end(), {1, i, j, -1});
    } else {
      return fail(c, TN_EFORMAT, "tree line " + std::to_string(ln) + ": unknown token " + tok);
    }
  }
  if (n_inputs < 0) return fail(c, TN_EFORMAT, "tree file has no inputs line");
  return add_tree(c, net_id, n_inputs, (int32_t)(ops.size() / 4), ops.data(), inst_id);
}

int tn_contract_approx(tn_ctx* c, int n_inst, const int* inst_ids, int chi, int prec, double* logabsz_out,
                       int* sign_out) {
  if (!c || !inst_ids || !logabsz_out || !sign_out || n_inst < 1) return fail(c, TN_EINVAL, "bad arguments");
  if (chi < 1) return fail(c, TN_EINVAL, "chi must be >= 1");
  if (prec < TN_F64 || prec > TN_TF32X3) return fail(c, TN_EINVAL, "unknown precision form");
  for (int q = 0; q < n_inst; ++q)
    if (inst_ids[q] < 0 || inst_ids[q] >= (int)c->insts.size()) return fail(c, TN_EINVAL, "unknown instance id");
  DeviceGuard g(c->device);
  std::vector<bool> done(n_inst, false);
  std::vector<std::vector<int>> groups, poss;
  std::vector<const tnp::Plan*> plans;
  for (int q = 0; q < n_inst; ++q) {
    if (done[q]) continue;
    std::vector<int> members, pos;
    for (int r = q; r < n_inst; ++r)
      if (!done[r] && same_group(c, inst_ids[q], inst_ids[r])) {
        members.push_back(inst_ids[r]);
        pos.push_back(r);
        done[r] = true;
      }
    int rc = TN_OK;
    const tnp::Plan* plan = get_plan(c, inst_ids[q], chi, prec, &rc);
    if (!plan) return rc;
    groups.push_back(members);
    poss.push_back(pos);
    plans.push_back(plan);
  }
  // (two groups could share one cached plan slot only through a hash
  // collision of their structures and trees; they then run one after the other)
  bool distinct = true;
  for (size_t a = 0; a < plans.size(); ++a)
    for (size_t b = a + 1; b < plans.size(); ++b) distinct = distinct && plans[a] != plans[b];
  // tn_options.split_batches: each group's batch runs as that many concurrent
  // sub-batches (they share the group's plan, which is read-only)
  if (distinct && c->split_batches > 1 && !c->profile && c->concurrent_groups) {
    std::vector<std::vector<int>> g2, p2;
    std::vector<const tnp::Plan*> pl2;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      const int nb = (int)groups[gi].size();
      const int parts = std::min(c->split_batches, nb);
      for (int q = 0; q < parts; ++q) {
        const int lo = nb * q / parts, hi = nb * (q + 1) / parts;
        g2.emplace_back(groups[gi].begin() + lo, groups[gi].begin() + hi);
        p2.emplace_back(poss[gi].begin() + lo, poss[gi].begin() + hi);
        pl2.push_back(plans[gi]);
      }
    }
    groups.swap(g2);
    poss.swap(p2);
    plans.swap(pl2);
  }
  if (groups.size() >= 2 && !c->profile && c->concurrent_groups && (distinct || c->split_batches > 1)) {
    std::vector<std::vector<double>> lg;
    std::vector<std::vector<int>> sg;
    const int rc = run_groups_concurrent(c, plans, groups, &lg, &sg);
    if (rc != TN_OK) return rc;
    for (size_t gi = 0; gi < groups.size(); ++gi)
      for (size_t m = 0; m < groups[gi].size(); ++m) {
        logabsz_out[poss[gi][m]] = lg[gi][m];
        sign_out[poss[gi][m]] = sg[gi][m];
      }
    return TN_OK;
  }
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    std::vector<double> lg(groups[gi].size());
    std::vector<int> sg(groups[gi].size());
    const int rc = run_group(c, *plans[gi], groups[gi], lg.data(), sg.data());
    if (rc != TN_OK) return rc;
    for (size_t m = 0; m < groups[gi].size(); ++m) {
      logabsz_out[poss[gi][m]] = lg[m];
      sign_out[poss[gi][m]] = sg[m];
    }
  }
  return TN_OK;
}

int tn_grad(tn_ctx* c, int n_inst, const int* inst_ids, int chi, int prec, double* logabsz_out, int* sign_out,
            double* const* grad_out, int on_device) {
  if (!c || !inst_ids || !logabsz_out || !sign_out || !grad_out || n_inst < 1)
    return fail(c, TN_EINVAL, "bad arguments");
  if (c->gauge_r >= 0) return fail(c, TN_EINVAL, "tn_grad is not available with the tree gauge (tn_set_tree_gauge)");
  if (chi < 1) return fail(c, TN_EINVAL, "chi must be >= 1");
  if (prec < TN_F64 || prec > TN_TF32X3) return fail(c, TN_EINVAL, "unknown precision form");
  for (int q = 0; q < n_inst; ++q) {
    if (inst_ids[q] < 0 || inst_ids[q] >= (int)c->insts.size()) return fail(c, TN_EINVAL, "unknown instance id");
    if (!grad_out[q]) return fail(c, TN_EINVAL, "grad_out has a NULL entry");
  }
  DeviceGuard g(c->device);
  std::vector<bool> done(n_inst, false);
  int zero_at = -1;
  for (int q = 0; q < n_inst; ++q) {
    if (done[q]) continue;
    std::vector<int> members, pos;
    for (int r = q; r < n_inst; ++r)
      if (!done[r] && same_group(c, inst_ids[q], inst_ids[r])) {
        members.push_back(inst_ids[r]);
        pos.push_back(r);
        done[r] = true;
      }
    int rc = TN_OK;
    int segs = c->grad_segments > 0 ? c->grad_segments : 1;
    const tnp::Plan* plan = get_plan(c, inst_ids[q], chi, prec, &rc, segs);
    if (!plan) return rc;
    if (c->grad_segments == 0) {
      // the whole tape does not fit in the budget (default half the free device memory): checkpoint
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
      }
      const double need = 8.0 * (double)plan->arena_units * (double)members.size();
      const size_t nops = c->insts[inst_ids[q]].ops.size() / 4;
      const double budget = c->tape_budget > 0.0 ? c->tape_budget : 0.5 * (double)free_b;
      if ((c->tape_budget > 0.0 || free_b) && need > budget && nops > 1) {
        segs = (int)std::ceil(std::sqrt((double)nops));
        plan = get_plan(c, inst_ids[q], chi, prec, &rc, segs);
        if (!plan) return rc;
      }
    }
    std::vector<double> lg(members.size());
    std::vector<int> sg(members.size());
    rc = run_group(c, *plan, members, lg.data(), sg.data());
    if (rc != TN_OK) return rc;
    // the adjoint block is padded like the input block; hand it out packed
    const tnp::Structure& st = c->nets[c->insts[members[0]].net].st;
    const int64_t nt = plan->in_total;
    for (size_t m = 0; m < members.size(); ++m) {
      logabsz_out[pos[m]] = lg[m];
      sign_out[pos[m]] = sg[m];
      if (sg[m] == 0 && zero_at < 0) zero_at = pos[m];
      int64_t packed = 0;
      for (size_t t = 0; t < st.bonds.size(); ++t) {
        int64_t sz = 1;
        for (int b : st.bonds[t]) sz *= st.bond_dims[b];
        cudaError_t e = cudaMemcpyAsync(grad_out[pos[m]] + packed, c->ginbuf + (size_t)m * nt + st.in_off[t],
                                        sizeof(double) * sz,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "gradient copy-out");
        packed += sz;
      }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "gradient copy-out");
  }
  if (zero_at >= 0)
    return fail(c, TN_ENONFINITE, "Z = 0 for instance " + std::to_string(zero_at) + ": log|Z| has no gradient");
  return TN_OK;
}

int tn_set_tree_gauge(tn_ctx* c, int r) {
  if (!c || r < -1) return fail(c, TN_EINVAL, "tree-gauge distance must be >= -1");
  c->gauge_r = r;
  return TN_OK;
}

int tn_set_grad_segments(tn_ctx* c, int segments) {
  if (!c || segments < 0) return fail(c, TN_EINVAL, "segments must be >= 0");
  c->grad_segments = segments;
  return TN_OK;
}

int tn_plan_describe(const tn_network_desc* d, const tn_tree_desc* t, int chi, int prec, int grad, int gauge_r,
                     char* buf, size_t cap, size_t* need) {
  if (!d || !t || !need) return TN_EINVAL;
  if (chi < 1 || prec < TN_F64 || prec > TN_TF32X3 || t->n_ops < 0 || (t->n_ops > 0 && !t->ops)) return TN_EINVAL;
  tnp::Structure st;
  int rc = load_structure(nullptr, d->n_bonds, d->bond_dims, d->n_tensors, d->ndims, d->bond_ids, &st);
  if (rc != TN_OK) return rc;
  std::vector<int32_t> ops(t->ops, t->ops + 4 * (size_t)t->n_ops);
  tnp::Plan plan;
  std::string err;
  try {
    err = tnp::build_plan(st, ops, t->n_inputs, chi, prec, &plan, grad != 0, grad > 1 ? grad : 1, gauge_r);
  } catch (...) {
    return TN_ENOMEM;
  }
  if (!err.empty()) return TN_EFORMAT;
  std::ostringstream o;
  o.precision(17);
  auto view = [&](const tnp::PView& v) {
    o << "[" << v.buf << "," << v.off << "," << v.rs << "," << v.cs << "," << v.bs << "," << v.eo << "]";
  };
  o << "{\"arena_units\":" << plan.arena_units << ",\"n_slots\":" << plan.n_slots << ",\"in_total\":" << st.in_total
    << ",\"grad\":" << (plan.grad ? 1 : 0) << ",\"segments\":" << plan.segments << ",\"in_off\":[";
  for (size_t q = 0; q < st.in_off.size(); ++q) o << (q ? "," : "") << st.in_off[q];
  o << "],\"steps\":[";
  for (size_t q = 0; q < plan.steps.size(); ++q) {
    const tnp::Step& x = plan.steps[q];
    o << (q ? "," : "") << "{\"kind\":" << x.kind << ",\"op\":" << x.op_index << ",\"m\":" << x.m << ",\"n\":" << x.n
      << ",\"k\":" << x.k << ",\"flag\":" << x.flag << ",\"slot\":" << x.slot << ",\"no_v\":" << x.no_v
      << ",\"init_v\":" << x.init_v << ",\"count\":" << x.count << ",\"fbs_src\":" << x.fbs_src
      << ",\"fbs_dst\":" << x.fbs_dst << ",\"alpha\":" << x.alpha << ",\"beta\":" << x.beta << ",\"tc_mode\":" << x.tc_mode;
    const char* names[] = {"A", "B", "C", "src", "dst", "work", "aux1", "aux2", "out1", "out2"};
    const tnp::PView* vs[] = {&x.A, &x.B, &x.C, &x.src, &x.dst, &x.work, &x.aux1, &x.aux2, &x.out1, &x.out2};
    for (int w = 0; w < 10; ++w) {
      o << ",\"" << names[w] << "\":";
      view(*vs[w]);
    }
    o << ",\"in_dims\":[";
    for (size_t a = 0; a < x.in_dims.size(); ++a) o << (a ? "," : "") << x.in_dims[a];
    o << "],\"perm\":[";
    for (size_t a = 0; a < x.perm.size(); ++a) o << (a ? "," : "") << x.perm[a];
    o << "]}";
  }
  o << "]}";
  const std::string js = o.str();
  *need = js.size() + 1;
  if (!buf) return TN_OK;
  if (cap < js.size() + 1) return TN_EINVAL;
  std::memcpy(buf, js.c_str(), js.size() + 1);
  return TN_OK;
}

int tn_debug_tensor(tn_ctx* c, int n_inst, const int* inst_ids, int which, int chi, int prec, int stop_op,
                    int tensor_id, double* out, int64_t cap, int32_t* ndim_out, int32_t* bond_ids_out,
                    int64_t* dims_out) {
  if (!c || !inst_ids || !ndim_out || n_inst < 1 || which < 0 || which >= n_inst)
    return fail(c, TN_EINVAL, "bad arguments");
  if (chi < 1) return fail(c, TN_EINVAL, "chi must be >= 1");
  if (prec < TN_F64 || prec > TN_TF32X3) return fail(c, TN_EINVAL, "unknown precision form");
  for (int q = 0; q < n_inst; ++q) {
    if (inst_ids[q] < 0 || inst_ids[q] >= (int)c->insts.size()) return fail(c, TN_EINVAL, "unknown instance id");
    if (!same_group(c, inst_ids[0], inst_ids[q])) return fail(c, TN_EINVAL, "instances do not share a tree and structure");
  }
  DeviceGuard g(c->device);
  int rc = TN_OK;
  const tnp::Plan* plan = get_plan(c, inst_ids[0], chi, prec, &rc);
  if (!plan) return rc;
  const tnp::TensorRec* rec = nullptr;
  for (const auto& r : plan->records)
    if (r.tensor_id == tensor_id && r.op_index <= stop_op) rec = &r;
  if (!rec) return fail(c, TN_EINVAL, "tensor does not exist after that op");
  for (const auto& cs : plan->consumed)
    if (cs.second == tensor_id && cs.first > rec->op_index && cs.first <= stop_op)
      return fail(c, TN_EINVAL, "tensor was contracted away before that op");
  int64_t size = 1;
  for (int64_t d : rec->dims) size *= d;
  *ndim_out = (int32_t)rec->bonds.size();
  if (bond_ids_out)
    for (size_t a = 0; a < rec->bonds.size() && a < (size_t)tnk::kMaxDims; ++a) bond_ids_out[a] = rec->bonds[a];
  if (dims_out)
    for (size_t a = 0; a < rec->dims.size() && a < (size_t)tnk::kMaxDims; ++a) dims_out[a] = rec->dims[a];
  if (!out) return TN_OK;  // shape query only
  if (cap < size) return fail(c, TN_EINVAL, "output buffer too small");
  std::vector<int> members(inst_ids, inst_ids + n_inst);
  std::vector<double> lg(n_inst);
  std::vector<int> sg(n_inst);
  const int stop = stop_op < 0 ? INT32_MAX : stop_op;
  // the previous call left this plan's state after op dbg_stop on the same batch: continue from there
  const bool cont = c->dbg_stop >= -1 && c->dbg_serial == plan->serial && c->dbg_members == members &&
                    c->dbg_gen == c->buf_gen && stop >= c->dbg_stop && stop != INT32_MAX;
  if (!(cont && stop == c->dbg_stop)) {
    const int prev = cont ? c->dbg_stop : -2;
    rc = run_group(c, *plan, members, lg.data(), sg.data(), stop, prev);
    if (rc != TN_OK) return rc;
    if (stop != INT32_MAX) {
      c->dbg_serial = plan->serial;
      c->dbg_gen = c->buf_gen;
      c->dbg_members = members;
      c->dbg_stop = stop;
    }
  }
  const int batch = n_inst;
  const double* base = rec->view.buf == tnp::BUF_INPUT ? c->inbuf + rec->view.off : c->arena + rec->view.off * batch;
  cudaError_t e = cudaMemcpy(out, base + (int64_t)which * rec->view.bs, sizeof(double) * size, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "fetch tensor");
  return TN_OK;
}

int tn_autotune(tn_ctx* c, int n_inst, const int* inst_ids, int chi, int prec, int* n_tuned) {
  if (!c || !inst_ids || n_inst < 1) return fail(c, TN_EINVAL, "bad arguments");
  if (chi < 1) return fail(c, TN_EINVAL, "chi must be >= 1");
  if (prec < TN_F64 || prec > TN_TF32X3) return fail(c, TN_EINVAL, "unknown precision form");
  for (int q = 0; q < n_inst; ++q)
    if (inst_ids[q] < 0 || inst_ids[q] >= (int)c->insts.size()) return fail(c, TN_EINVAL, "unknown instance id");
  DeviceGuard g(c->device);
  c->dbg_stop = -2;
  int tuned = 0;
  std::vector<bool> done(n_inst, false);
  for (int q = 0; q < n_inst; ++q) {
    if (done[q]) continue;
    int batch = 0;
    for (int r = q; r < n_inst; ++r)
      if (!done[r] && same_group(c, inst_ids[q], inst_ids[r])) {
        done[r] = true;
        ++batch;
      }
    int rc = TN_OK;
    const tnp::Plan* plan = get_plan(c, inst_ids[q], chi, prec, &rc);
    if (!plan) return rc;
    // distinct launch shapes; GEMMs by their share of the plan's GEMM flops
    std::map<TuneKey, double> work;
    std::map<TuneKey, bool> with_v;
    for (const tnp::Step& st : plan->steps) {
      if (st.kind == tnp::ST_QR) work[{tnk::TK_QR, st.m, st.n, 0}] += 1.0;
      if (st.kind == tnp::ST_JACOBI) {
        work[{tnk::TK_JAC64, st.m, st.n, 0}] += 1.0;
        with_v[{tnk::TK_JAC64, st.m, st.n, 0}] = !st.no_v;
      }
      if (st.kind == tnp::ST_JACOBI32) work[{tnk::TK_JAC32, st.m, st.n, 0}] += 1.0;
      if (st.kind == tnp::ST_GEMM) work[{tnk::TK_GEMM64, st.m, st.n, st.k}] += 2.0 * st.m * st.n * (double)st.k;
      if (st.kind == tnp::ST_GEMM_TC) work[{tnk::TK_GEMMTC, st.m, st.n, st.k}] += 2.0 * st.m * st.n * (double)st.k;
    }
    std::vector<std::pair<double, TuneKey>> gemms;
    double gemm_total = 0.0;
    for (const auto& w : work)
      if (w.first.kernel == tnk::TK_GEMM64 || w.first.kernel == tnk::TK_GEMMTC) {
        gemms.push_back({w.second, w.first});
        gemm_total += w.second;
      }
    std::sort(gemms.begin(), gemms.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<TuneKey> keys;
    for (const auto& w : work)
      if (w.first.kernel != tnk::TK_GEMM64 && w.first.kernel != tnk::TK_GEMMTC) keys.push_back(w.first);
    double covered = 0.0;
    for (const auto& gk : gemms) {  // the GEMM shapes that carry 98% of the GEMM flops (64 shapes at most in all)
      if (covered >= 0.98 * gemm_total || (int)keys.size() >= 64) break;
      keys.push_back(gk.second);
      covered += gk.first;
    }
    cudaStream_t s = c->stream;
    for (const TuneKey& key : keys) {
      const int m = key.m, n = key.n, k = key.k;
      // scratch operands of one launch of this shape (random entries)
      size_t elems = 0, aux = 0;
      if (key.kernel == tnk::TK_QR) elems = (size_t)m * n, aux = (size_t)m * n + n + (size_t)std::min(m, n) * n;
      if (key.kernel == tnk::TK_JAC64 || key.kernel == tnk::TK_JAC32)
        elems = (size_t)m * n, aux = (size_t)n * n + n;
      if (key.kernel == tnk::TK_GEMM64 || key.kernel == tnk::TK_GEMMTC)
        elems = (size_t)m * k + (size_t)k * n, aux = (size_t)m * n;
      struct Scratch {  // freed on every exit from this shape's iteration
        double* in = nullptr;
        double* aux = nullptr;
        void* ws = nullptr;
        ~Scratch() {
          cudaFree(in);
          cudaFree(aux);
          cudaFree(ws);
        }
      } sc;
      double*& d_in = sc.in;
      double*& d_aux = sc.aux;
      void*& d_ws = sc.ws;
      size_t ws_bytes = 0;
      if (key.kernel == tnk::TK_GEMMTC) ws_bytes = tnk::gemm_tc_workspace_bytes(m, n, k, prec == 1 ? 0 : (prec == 2 ? 1 : 2), batch);
      if (cudaMalloc(&d_in, sizeof(double) * elems * batch) != cudaSuccess ||
          cudaMalloc(&d_aux, sizeof(double) * aux * batch) != cudaSuccess ||
          (ws_bytes && cudaMalloc(&d_ws, ws_bytes) != cudaSuccess)) {
        cudaGetLastError();
        return fail(c, TN_ENOMEM, "autotune scratch allocation failed");
      }
      {
        std::vector<double> h(elems * batch);
        fill_random(h, (uint64_t)(m * 131 + n * 7 + k));
        if (key.kernel == tnk::TK_JAC32) {  // the FP32 pass reads floats
          std::vector<float> hf(h.begin(), h.end());
          cudaMemcpy(d_in, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice);
        } else {
          cudaMemcpy(d_in, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
        }
      }
      const void* old_scratch = c->expo;
      rc = ensure_scratch(c, batch);
      if (rc != TN_OK) return rc;
      if (old_scratch != c->expo) drop_graphs(c);  // captured graphs point at the old scratch
      if (!c->tc_err && cudaMalloc(&c->tc_err, sizeof(int)) != cudaSuccess) return fail(c, TN_ENOMEM, "error word");
      tnk::DevState ds{c->expo, c->status};
      std::vector<int> cands;
      if (key.kernel == tnk::TK_QR || key.kernel == tnk::TK_JAC64 || key.kernel == tnk::TK_JAC32) {
        for (int P : {1, 2, 3, 4, 6, 8, 10, 12, 14, 16})
          if (P * 8 <= std::max(8, n)) cands.push_back(P);
      } else if (key.kernel == tnk::TK_GEMM64) {
        cands = {1, 2, 3, 4};
      } else {
        cands = {64, 128};
        if (prec != TN_TF32X3) cands.push_back(256);
      }
      const int saved = tnk::tune_get(key.kernel, m, n, k, batch);
      int best = 0;
      double best_ms = -1.0;
      for (int cand : cands) {
        tnk::tune_set(key.kernel, m, n, k, batch, cand);
        auto launch = [&]() -> cudaError_t {
          switch (key.kernel) {
            case tnk::TK_QR:
              return tnk::qr_r_f64(m, n, tnk::View{d_in, 1, m, (int64_t)m * n}, d_aux, (int64_t)m * n,
                                   tnk::ViewW{d_aux + ((size_t)m * n + n) * batch, n, 1, (int64_t)std::min(m, n) * n},
                                   batch, s);
            case tnk::TK_JAC64:
              return tnk::jacobi_svd_f64(m, n, d_in, (int64_t)m * n, with_v[key] ? d_aux : nullptr, (int64_t)n * n,
                                         d_aux + (size_t)n * n * batch, n, c->jac_ws, ds, 1, batch, s, nullptr,
                                         1e-300, 2);
            case tnk::TK_JAC32:
              return tnk::jacobi_svd_f32(m, n, reinterpret_cast<float*>(d_in), (int64_t)m * n,
                                         reinterpret_cast<float*>(d_aux), (int64_t)n * n, c->jac_ws, ds, batch, s,
                                         nullptr, 2);
            case tnk::TK_GEMM64:
              return tnk::gemm_f64(m, n, k, 1.0, tnk::View{d_in, k, 1, (int64_t)m * k},
                                   tnk::View{d_in + (size_t)m * k * batch, n, 1, (int64_t)k * n}, 0.0,
                                   tnk::ViewW{d_aux, n, 1, (int64_t)m * n}, batch, s);
            default:
              return tnk::gemm_tc(m, n, k, 1.0, tnk::View{d_in, k, 1, (int64_t)m * k},
                                  tnk::View{d_in + (size_t)m * k * batch, n, 1, (int64_t)k * n},
                                  tnk::ViewW{d_aux, n, 1, (int64_t)m * n}, batch,
                                  prec == 1 ? 0 : (prec == 2 ? 1 : 2), d_ws, ws_bytes, c->tc_err, s);
          }
        };
        const double ms = time_launch(s, launch);
        if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
          best_ms = ms;
          best = cand;
        }
      }
      tnk::tune_set(key.kernel, m, n, k, batch, best > 0 ? best : saved);
      if (best > 0) ++tuned;
      // the scratch runs may have flagged statuses (capped sweeps): clear them
      cudaMemsetAsync(c->status, 0, sizeof(int) * batch, s);
      cudaMemsetAsync(c->tc_err, 0, sizeof(int), s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "autotune");
    }
  }
  if (n_tuned) *n_tuned = tuned;
  drop_graphs(c);  // recapture with the tuned launch shapes
  if (!c->tuner_cache.empty()) {
    const std::string e = tnk::tune_save(c->tuner_cache);
    if (!e.empty()) return fail(c, TN_EINVAL, "tuner cache: " + e);
  }
  return TN_OK;
}

int tn_tuned_choices(tn_ctx* c, int cap, int32_t* rows) {
  if (!c || cap < 0 || (cap > 0 && !rows)) return fail(c, TN_EINVAL, "bad arguments");
  DeviceGuard g(c->device);
  const auto e = tnk::tune_entries();
  for (int i = 0; i < cap && i < (int)e.size(); ++i)
    for (int j = 0; j < 6; ++j) rows[6 * i + j] = e[i][j];
  return (int)e.size();
}

int tn_plan_stats_get(tn_ctx* c, int inst_id, int chi, int prec, tn_plan_stats* out) {
  if (!c || !out) return fail(c, TN_EINVAL, "NULL argument");
  if (inst_id < 0 || inst_id >= (int)c->insts.size()) return fail(c, TN_EINVAL, "unknown instance id");
  if (chi < 1) return fail(c, TN_EINVAL, "chi must be >= 1");
  int rc = TN_OK;
  const tnp::Plan* p = get_plan(c, inst_id, chi, prec, &rc);
  if (!p) return rc;
  out->n_contractions = p->n_contractions;
  out->n_compressions = p->n_compressions;
  out->gemm_flops = p->gemm_flops;
  out->qr_flops = p->qr_flops;
  out->svd_flops = p->svd_flops;
  out->permute_bytes = p->permute_bytes;
  out->peak_bytes = 8.0 * (double)p->arena_units;
  int64_t launches = 0;
  for (auto& s : p->steps)  // rescale = max + scale kernels; copies are not kernels
    launches += (s.kind == tnp::ST_RESCALE || s.kind == tnp::ST_JACOBI32 || s.kind == tnp::ST_JACOBI)
                    ? (s.kind == tnp::ST_RESCALE ? 2 : 1)
                    : (s.kind == tnp::ST_COPY ? 0 : (s.kind == tnp::ST_GEMM_TC ? 3 : 1));  // TC: 2 staging + GEMM
  out->kernel_launches = launches;
  return TN_OK;
}

int tn_profile_enable(tn_ctx* c, int enable) {
  if (!c) return TN_EINVAL;
  c->profile = enable != 0;
  for (int f = 0; f < kNumFamily; ++f) {
    c->prof_launches[f] = 0;
    c->prof_ms[f] = 0.0;
  }
  c->prof_sweeps[0] = c->prof_sweeps[1] = 0;
  return TN_OK;
}

int tn_kernel_times(tn_ctx* c, int cap, const char** names, int64_t* launches, double* total_ms) {
  if (!c) return TN_EINVAL;
  int n = 0;
  for (int f = 0; f < kNumFamily; ++f) {
    if (c->prof_launches[f] == 0) continue;
    if (n < cap) {
      if (names) names[n] = kFamily[f];
      if (launches) launches[n] = c->prof_launches[f];
      if (total_ms) total_ms[n] = c->prof_ms[f];
    }
    ++n;
  }
  // pseudo-families: Jacobi sweeps run (launches = sweeps summed over matrices, time 0)
  const char* sw_names[2] = {"sweeps:jacobi_f32", "sweeps:jacobi_f64"};
  for (int q = 0; q < 2; ++q) {
    if (!c->prof_sweeps[q]) continue;
    if (n < cap) {
      if (names) names[n] = sw_names[q];
      if (launches) launches[n] = (int64_t)c->prof_sweeps[q];
      if (total_ms) total_ms[n] = 0.0;
    }
    ++n;
  }
  return n;
}

const char* tn_last_error(const tn_ctx* c) {
  if (!c) return "NULL context";
  return c->err.c_str();
}

}  // extern "C"
