// Householder QR of one side of a compression: A = Q_A R_A with A = T_i as
// (D_A x D_AB), and LQ of B via QR of B^T (Sec. "Bond compression
// strategies").  The kernel writes R and keeps the reflectors (v_j below the
// diagonal of the working copy, tau_j after it) for the Q-form absorb.
//
// One thread-block cluster of P CTAs factors one matrix.  Columns are dealt
// out cyclically (column c belongs to CTA c mod P); the working copy lives
// column-major in global scratch (L2-resident at these sizes).  Step j:
//   the owner of column j builds the reflector (v, tau) in place,
//   a cluster barrier (release / acquire) publishes it,
//   every CTA applies H_j = I - tau v v^T to its own columns c > j,
//   one warp per column (dot product by warp shuffles, then the axpy).
// GB300's FP64 pipe (2 DFMA / clock / SM) bounds the update, so spreading one
// matrix over P SMs is what sets the speed.
#include <cooperative_groups.h>

#include "tn_cluster.h"
#include "tn_kernels.h"
#include "tn_tune.h"

namespace cg = cooperative_groups;

namespace tnk {
namespace {

constexpr int kThreads = 256;
constexpr int kVSmem = 8192;  // stage v in shared memory up to this many rows

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ double block_sum(double x, double* red) {
  x = warp_sum(x);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < (blockDim.x >> 5)) t = red[threadIdx.x];
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// kSmem: this CTA's columns live in shared memory for the whole factorisation
// (reflectors are also written to global memory for the other CTAs and for
// apply_q); otherwise they are updated in place in the global working copy.
template <bool kSmem>
__global__ void __launch_bounds__(kThreads) qr_cluster_kernel(int m, int n, View A, double* work,
                                                              int64_t work_bs, double* taus,
                                                              ViewW R) {
  cg::cluster_group cl = cg::this_cluster();
  const int P = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int b = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  double* W = work + (int64_t)b * work_bs;
  double* tau_b = taus + (int64_t)b * n;
  const double* a = A.p + (int64_t)b * A.bs;
  extern __shared__ double sm[];
  __shared__ double red[32];
  const int nc_max = (n + P - 1) / P;
  double* colbuf = sm;                                       // kSmem: nc_max columns of length m
  double* vs = kSmem ? sm + (size_t)nc_max * m : sm;         // reflector staging (m <= kVSmem)
  const bool stage_v = kSmem || (m <= kVSmem);
  auto col_of = [&](int c) -> double* {
    return kSmem ? colbuf + (size_t)((c - rank) / P) * m : W + (int64_t)c * m;
  };

  // working copy of this CTA's columns
  for (int c = rank; c < n; c += P) {
    double* dst = col_of(c);
    for (int r = tid; r < m; r += blockDim.x) dst[r] = a[(int64_t)r * A.rs + (int64_t)c * A.cs];
  }
  __syncthreads();

  const int rmin = m < n ? m : n;
  for (int j = 0; j < rmin; ++j) {
    if (j % P == rank) {
      double* x = col_of(j);
      double part = 0.0;
      for (int r = j + 1 + tid; r < m; r += blockDim.x) part += x[r] * x[r];
      const double sigma = block_sum(part, red);
      const double alpha = x[j];
      double tau = 0.0;
      if (sigma > 0.0) {
        const double nrm = sqrt(alpha * alpha + sigma);
        const double beta = (alpha <= 0.0) ? nrm : -nrm;
        tau = (beta - alpha) / beta;
        const double scale = 1.0 / (alpha - beta);
        double* g = W + (int64_t)j * m;
        for (int r = j + 1 + tid; r < m; r += blockDim.x) {
          const double v = x[r] * scale;
          x[r] = v;
          if (kSmem) g[r] = v;   // publish the reflector
        }
        __syncthreads();
        if (tid == 0) x[j] = beta;
      }
      if (tid == 0) tau_b[j] = tau;
    }
    cl.sync();
    const double tau = __ldcg(tau_b + j);
    if (tau != 0.0) {
      const double* v = W + (int64_t)j * m;
      const int len = m - j;
      if (stage_v) {
        for (int r = tid; r < len; r += blockDim.x) vs[r] = (r == 0) ? 1.0 : __ldcg(v + j + r);
        __syncthreads();
      }
      // first own column > j
      int c0 = j + 1 + ((rank - (j + 1)) % P + P) % P;
      int ncol = (c0 < n) ? (n - 1 - c0) / P + 1 : 0;
      for (int q = warp; q < ncol; q += nwarps) {
        double* col = col_of(c0 + q * P) + j;
        double d = 0.0;
        if (stage_v) {
          for (int r = lane; r < len; r += 32) d = fma(vs[r], col[r], d);
        } else {
          for (int r = lane; r < len; r += 32) d = fma(r == 0 ? 1.0 : __ldcg(v + j + r), col[r], d);
        }
        d = warp_sum(d) * tau;
        if (stage_v) {
          for (int r = lane; r < len; r += 32) col[r] -= d * vs[r];
        } else {
          for (int r = lane; r < len; r += 32) col[r] -= d * (r == 0 ? 1.0 : __ldcg(v + j + r));
        }
      }
    }
    __syncthreads();
  }
  // R: rows 0..rmin-1 of this CTA's columns (the diagonal holds beta); with
  // kSmem the columns (R above, reflectors below the diagonal) go back to W
  double* rr = R.p + (int64_t)b * R.bs;
  for (int c = rank; c < n; c += P) {
    const double* col = col_of(c);
    for (int i = tid; i < rmin; i += blockDim.x)
      rr[(int64_t)i * R.rs + (int64_t)c * R.cs] = (i <= c) ? col[i] : 0.0;
    if (kSmem) {
      double* g = W + (int64_t)c * m;
      for (int r = tid; r < m; r += blockDim.x) g[r] = col[r];
    }
  }
}

// X <- Q X with Q = H_0 H_1 ... H_{r-1} the Householder product left in
// `work` by qr_cluster_kernel (v_j below the diagonal of column j, implicit
// unit at j; tau_j in `taus`).  This is the Q-form absorb of Eq. "svd":
// A_bar = Q_A (U_k sigma^1/2), applied reflector by reflector in reverse so
// the orthogonal factor is never formed.  X is m x k column-major; each warp
// owns one column of X, and each reflector is staged once per CTA in shared
// memory.
__global__ void __launch_bounds__(kThreads) apply_q_kernel(int m, int n, const double* Wall,
                                                           int64_t w_bs, const double* taus,
                                                           double* Xall, int64_t x_bs, int k, int trans) {
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const double* W = Wall + (int64_t)b * w_bs;
  const double* tau = taus + (int64_t)b * n;
  double* X = Xall + (int64_t)b * x_bs;
  const int col = blockIdx.x * nwarps + warp;
  extern __shared__ double vs[];
  const bool stage_v = (m <= kVSmem);
  const int rmin = m < n ? m : n;
  // Q = H_0 H_1 ... H_{r-1}: Q X applies H_{r-1} first, Q^T X applies H_0 first
  for (int it = 0; it < rmin; ++it) {
    const int j = trans ? it : rmin - 1 - it;
    const double t = tau[j];
    if (t == 0.0) continue;
    const double* v = W + (int64_t)j * m;
    if (stage_v) {
      __syncthreads();
      for (int r = j + threadIdx.x; r < m; r += blockDim.x) vs[r] = (r == j) ? 1.0 : v[r];
      __syncthreads();
    }
    if (col < k) {
      double* x = X + (int64_t)col * m;
      double d = 0.0;
      for (int r = j + lane; r < m; r += 32) d = fma(stage_v ? vs[r] : (r == j ? 1.0 : v[r]), x[r], d);
      d = warp_sum(d) * t;
      for (int r = j + lane; r < m; r += 32) x[r] -= d * (stage_v ? vs[r] : (r == j ? 1.0 : v[r]));
    }
  }
}

}  // namespace

cudaError_t apply_q_f64(int m, int n, const double* work, int64_t work_bs, double* X, int64_t x_bs, int k,
                        int batch, cudaStream_t s, int trans) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  const double* taus = work + (int64_t)batch * work_bs;
  size_t smem = (m <= kVSmem) ? (size_t)m * sizeof(double) : 0;
  cudaError_t ae = once_per_device((const void*)apply_q_kernel, [] {
    return cudaFuncSetAttribute(apply_q_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kVSmem * (int)sizeof(double));
  });
  if (ae != cudaSuccess) return ae;
  const int per_cta = kThreads / 32;
  dim3 grid((k + per_cta - 1) / per_cta, batch);
  apply_q_kernel<<<grid, kThreads, smem, s>>>(m, n, work, work_bs, taus, X, x_bs, k, trans);
  return cudaGetLastError();
}

namespace {

constexpr size_t kQrSmemCap = 210 * 1024;

cudaError_t ensure_qr_attrs() {
  return once_per_device((const void*)qr_cluster_kernel<true>, [] {
    cudaError_t e =
        cudaFuncSetAttribute(qr_cluster_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQrSmemCap);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(qr_cluster_kernel<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(qr_cluster_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kVSmem * (int)sizeof(double));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(qr_cluster_kernel<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
  });
}

template <bool kSmem>
cudaError_t launch_qr(int P, int m, int n, View A, double* work, int64_t work_bs, double* taus, ViewW R,
                      int batch, cudaStream_t s, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P, batch, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, qr_cluster_kernel<kSmem>, m, n, A, work, work_bs, taus, R);
}

}  // namespace

cudaError_t qr_r_f64(int m, int n, View A, double* work, int64_t work_bs, ViewW R, int batch,
                     cudaStream_t s) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  cudaError_t ae = ensure_qr_attrs();
  if (ae != cudaSuccess) return ae;
  // tau scratch sits after the batch of working copies
  double* taus = work + (int64_t)batch * work_bs;
  // cluster size: at least ~16 columns per CTA and at most 16 CTAs (non-portable
  // size); within [pmax/2, pmax] the size with the fewest waves per CTA of work
  int pmax = (n + 15) / 16;
  if (pmax > 16) pmax = 16;
  if (pmax < 1) pmax = 1;
  const int pmin = pmax / 2 > 0 ? pmax / 2 : 1;
  auto smem_cols = [&](int q) {
    const int nc = (n + q - 1) / q;
    const size_t b = ((size_t)nc * m + (size_t)m) * sizeof(double);
    return b <= kQrSmemCap ? b : (size_t)-1;
  };
  const size_t gsm = (m <= kVSmem) ? (size_t)m * sizeof(double) : 0;
  // a measured choice (tn_autotune) first
  const int tp = tune_get(TK_QR, m, n, 0, batch);
  if (tp >= 1 && tp <= 16) {
    if (smem_cols(tp) != (size_t)-1) return launch_qr<true>(tp, m, n, A, work, work_bs, taus, R, batch, s, smem_cols(tp));
    return launch_qr<false>(tp, m, n, A, work, work_bs, taus, R, batch, s, gsm);
  }
  auto even = [](int) { return 1.0; };
  int P = choose_cluster((const void*)qr_cluster_kernel<true>, kThreads, batch, pmin, pmax, smem_cols, even);
  if (P > 0) return launch_qr<true>(P, m, n, A, work, work_bs, taus, R, batch, s, smem_cols(P));
  // columns do not fit in shared memory: update them in global memory
  P = choose_cluster((const void*)qr_cluster_kernel<false>, kThreads, batch, pmin, pmax, [&](int) { return gsm; },
                     even);
  if (P < 1) P = pmax < 8 ? pmax : 8;
  return launch_qr<false>(P, m, n, A, work, work_bs, taus, R, batch, s, gsm);
}

}  // namespace tnk
