// One launch of one schedule step, and the validation of a network's
// structure: shared by the context executor (tn_api.cpp) and the
// allocation-free entry point (tn_noalloc.cu), so that both run every step
// kind with the same arguments and accept exactly the same networks.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "tn_kernels.h"
#include "tn_plan.h"

namespace tnx {

// Device buffers of one batch as the executor laid them out (arena buffers
// at offset * batch, inputs and input adjoints at their element offsets).
struct ExecEnv {
  double* inbuf = nullptr;
  double* arena = nullptr;
  double* ginbuf = nullptr;      // reverse-pass plans only
  int batch = 1;
  tnk::DevState ds{nullptr, nullptr};
  int* jac_ws = nullptr;         // 64 ints per instance
  unsigned long long* maxbits = nullptr;
  double* out_log = nullptr;
  int* out_sign = nullptr;
  int* tc_err = nullptr;         // tensor-core GEMMs: set when a bounded wait ran out
  int* etape = nullptr;          // reverse-pass plans: rescale exponents, [slots][batch]
  unsigned long long* sweeps32 = nullptr;  // optional Jacobi sweep counters
  unsigned long long* sweeps64 = nullptr;
  int jac_max_sweeps = 0;        // > 0: cap on the Jacobi sweep loops (0: the kernels' default)
  bool tc_give_up = false;       // tests: the tensor-core GEMM's pipeline waits give up at once

  double* ptr(const tnp::PView& v) const {
    double* base = v.buf == tnp::BUF_INPUT ? inbuf + v.off
                   : v.buf == tnp::BUF_GIN ? ginbuf + v.off
                                           : arena + v.off * batch;
    return base + v.eo;
  }
};

// Launch the kernels of one step on stream s.
cudaError_t exec_step(const tnp::Step& stp, const ExecEnv& env, cudaStream_t s);

// Validate a network's bond structure (every bond in exactly two different
// tensors, sizes in range) and fill *st.  Returns TN_OK or a tn_status with
// the reason in *msg.
int check_structure(int32_t n_bonds, const int64_t* bond_dims, int32_t n_tensors, const int32_t* ndims,
                    const int32_t* bond_ids, tnp::Structure* st, std::string* msg);

}  // namespace tnx
