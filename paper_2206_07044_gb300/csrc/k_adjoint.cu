// Kernels of the reverse pass: d log|Z| / d (every input tensor).
//
// The reverse pass walks the forward schedule backwards.  Matrix-product
// adjoints are plain GEMMs (gemm_f64 / the tensor-core GEMM with transposed
// views); the kernels here are the pieces that are not products:
//   * the adjoint of the exact power-of-two rescale (multiply by 2^-e),
//   * the adjoint of ln|x| at the root (1 / x),
//   * the sorted singular factors of the compression core (from the Jacobi
//     outputs), and
//   * the core matrix of the truncated-SVD adjoint (the Lorentzian-broadened
//     F-terms and the singular-value adjoint), one element per thread.
// The compression adjoint follows the SVD of X = A B written in the bases of
// the forward QRs: with Q_A^T A_bar' = [dU; W_A] and Q_B^T B_bar'^T = [dV; W_B],
//   D11 = U C W^T + (dU - U P) Ws^T + Us (dV - W Q)^T,   P = U^T dU, Q = W^T dV,
//   dA  = Q_A [D11 L_B^T; W_A Ws^T L_B^T],  dB^T = Q_B [D11^T R_A; W_B Us^T R_A],
// which the plan issues as GEMMs around the two kernels below.
#include "tn_kernels.h"

namespace tnk {
namespace {

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_isum(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

int grid1(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

__global__ void scale_pow2_kernel(double* __restrict__ X, int64_t n, int64_t bs, const int* __restrict__ e) {
  const int b = blockIdx.y;
  const double sc = ldexp(1.0, -e[b]);
  double* x = X + (int64_t)b * bs;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= sc;
}

__global__ void final_grad_kernel(const double* x, int64_t xbs, double* g, int64_t gbs, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) g[(int64_t)b * gbs] = 1.0 / x[(int64_t)b * xbs];
}

constexpr int kFacThreads = 128;

// One block per (source column i, instance): rank of sigma_i, then the column
// of each factor at that rank.
__global__ void __launch_bounds__(kFacThreads) svd_factors_kernel(
    int m, int n, int k, int tall, const double* Gall, int64_t g_bs, const double* Vall, int64_t v_bs,
    const double* sigall, int64_t sig_bs, double* Uall, int64_t u_bs, double* Wall, int64_t w_bs, double* sall,
    int64_t s_bs, double* Usall, int64_t us_bs, double* Wsall, int64_t ws_bs) {
  const int i = blockIdx.x, b = blockIdx.y;
  const double* sig = sigall + (int64_t)b * sig_bs;
  const double si = sig[i];
  double mx = 0.0;
  int r = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double sj = sig[j];
    mx = fmax(mx, sj);
    r += (sj > si) || (sj == si && j < i);
  }
  __shared__ double smx[kFacThreads / 32];
  __shared__ int srk[kFacThreads / 32];
  mx = warp_max(mx);
  r = warp_isum(r);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    smx[warp] = mx;
    srk[warp] = r;
  }
  __syncthreads();
  double smax = 0.0;
  int p = 0;
  for (int w = 0; w < kFacThreads / 32; ++w) {
    smax = fmax(smax, smx[w]);
    p += srk[w];
  }
  const bool nz = si > 1e-13 * smax && si > 0.0;
  const double inv = nz ? 1.0 / si : 0.0;
  const double isq = nz ? 1.0 / sqrt(si) : 0.0;
  const int rows_u = tall ? m : n, rows_w = tall ? n : m;
  double* U = Uall + (int64_t)b * u_bs + (int64_t)p * rows_u;
  double* W = Wall + (int64_t)b * w_bs + (int64_t)p * rows_w;
  double* Us = Usall + (int64_t)b * us_bs + (int64_t)p * rows_u;
  double* Ws = Wsall + (int64_t)b * ws_bs + (int64_t)p * rows_w;
  const double* g = Gall + (int64_t)b * g_bs + (int64_t)i * m;
  const double* v = Vall + (int64_t)b * v_bs + (int64_t)i * n;
  // the G column is sigma_i times a left vector of J; the V column a right vector
  double* gdst = tall ? U : W;
  double* gdst_s = tall ? Us : Ws;
  double* vdst = tall ? W : U;
  double* vdst_s = tall ? Ws : Us;
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const double x = g[q] * inv;
    gdst[q] = x;
    if (p < k) gdst_s[q] = x * isq;
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const double x = v[q];
    vdst[q] = x;
    if (p < k) vdst_s[q] = x * isq;
  }
  if (threadIdx.x == 0) sall[(int64_t)b * s_bs + p] = si;
}

__global__ void svd_adjoint_core_kernel(int q, int k, const double* Pall, int64_t p_bs, const double* Qall,
                                        int64_t q_bs, const double* sall, int64_t s_bs, double* Call,
                                        int64_t c_bs) {
  const int b = blockIdx.y;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)q * q) return;
  const int i = (int)(idx % q), j = (int)(idx / q);
  const double* s = sall + (int64_t)b * s_bs;
  const double* P = Pall + (int64_t)b * p_bs;
  const double* Q = Qall + (int64_t)b * q_bs;
  const double s0 = s[0];
  const double si = s[i], sj = s[j];
  double c = 0.0;
  if (i != j) {
    const double d = sj * sj - si * si;
    const double F = d / (d * d + 1e-12 * s0 * s0);
    const double aij = j < k ? P[i + (int64_t)j * q] * sqrt(sj) : 0.0;
    const double aji = i < k ? P[j + (int64_t)i * q] * sqrt(si) : 0.0;
    const double bij = j < k ? Q[i + (int64_t)j * q] * sqrt(sj) : 0.0;
    const double bji = i < k ? Q[j + (int64_t)i * q] * sqrt(si) : 0.0;
    c = F * (aij - aji) * sj + si * F * (bij - bji);
  } else if (i < k) {
    const double isq = (si > 1e-13 * s0 && si > 0.0) ? 1.0 / sqrt(si) : 0.0;
    c = 0.5 * isq * (P[i + (int64_t)i * q] + Q[i + (int64_t)i * q]);
  }
  Call[(int64_t)b * c_bs + idx] = c;
}

__global__ void copy2d_kernel(int m, int n, View X, ViewW Y) {
  const int b = blockIdx.y;
  const int64_t total = (int64_t)m * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % m, c = t / m;
    Y.p[(int64_t)b * Y.bs + r * Y.rs + c * Y.cs] = X.p[(int64_t)b * X.bs + r * X.rs + c * X.cs];
  }
}

}  // namespace

cudaError_t scale_pow2_f64(double* X, int64_t n, int64_t bs, const int* e, int batch, cudaStream_t s) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  scale_pow2_kernel<<<dim3(grid1(n), batch), 256, 0, s>>>(X, n, bs, e);
  return cudaGetLastError();
}

cudaError_t final_grad_f64(const double* x, int64_t xbs, double* g, int64_t gbs, int batch, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  final_grad_kernel<<<(batch + 127) / 128, 128, 0, s>>>(x, xbs, g, gbs, batch);
  return cudaGetLastError();
}

cudaError_t svd_factors_f64(int m, int n, int k, int tall, const double* G, int64_t g_bs, const double* V,
                            int64_t v_bs, const double* sig, int64_t sig_bs, double* U, int64_t u_bs, double* W,
                            int64_t w_bs, double* s_out, int64_t s_bs, double* Us, int64_t us_bs, double* Ws,
                            int64_t ws_bs, int batch, cudaStream_t s) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535 || m < n || k > n) return cudaErrorInvalidValue;
  svd_factors_kernel<<<dim3(n, batch), kFacThreads, 0, s>>>(m, n, k, tall, G, g_bs, V, v_bs, sig, sig_bs, U, u_bs,
                                                            W, w_bs, s_out, s_bs, Us, us_bs, Ws, ws_bs);
  return cudaGetLastError();
}

cudaError_t svd_adjoint_core_f64(int q, int k, const double* P, int64_t p_bs, const double* Q, int64_t q_bs,
                                 const double* s, int64_t s_bs, double* C, int64_t c_bs, int batch, cudaStream_t st) {
  if (q <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535 || k > q) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)q * q;
  svd_adjoint_core_kernel<<<dim3((unsigned)((total + 255) / 256), batch), 256, 0, st>>>(q, k, P, p_bs, Q, q_bs, s,
                                                                                       s_bs, C, c_bs);
  return cudaGetLastError();
}

cudaError_t copy2d_f64(int m, int n, View X, ViewW Y, int batch, cudaStream_t s) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  copy2d_kernel<<<dim3(grid1((int64_t)m * n), batch), 256, 0, s>>>(m, n, X, Y);
  return cudaGetLastError();
}

}  // namespace tnk
