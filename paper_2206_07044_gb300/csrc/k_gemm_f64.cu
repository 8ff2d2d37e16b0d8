// FP64 GEMM on the CUDA cores: C = alpha * A * B for the pairwise
// contractions (A = T_i as (left x shared), B = T_j as (shared x right)), the
// R_A L_B core and the Newton-Schulz / preconditioning products of the core SVD.
//
// GB300 runs FP64 at 2 DFMA / clock / SM (about 1.2 TFLOP/s for the chip), so
// these products are FP64-pipe bound at any realistic size; the kernel keeps
// 16 independent DFMAs per thread per k-step and stages 64 x 16 / 16 x 64
// operand tiles through shared memory with coalesced loads for either
// operand orientation (the schedule passes row- or column-major views
// instead of permuting).
#include "tn_kernels.h"

namespace tnk {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(int m, int n, int k, double alpha, View A,
                                                       View B, double beta, ViewW C) {
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const double* a = A.p + (int64_t)blockIdx.z * A.bs;
  const double* b = B.p + (int64_t)blockIdx.z * B.bs;
  double* c = C.p + (int64_t)blockIdx.z * C.bs;
  const bool a_kcontig = (A.cs == 1);
  const bool b_ncontig = (B.cs == 1);

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  auto load_regs = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int l = tid + q * 256;
      int mm, kk;
      if (a_kcontig) { kk = l & 15; mm = l >> 4; } else { mm = l & 63; kk = l >> 6; }
      int gm = m0 + mm, gk = k0 + kk;
      ra[q] = (gm < m && gk < k) ? a[(int64_t)gm * A.rs + (int64_t)gk * A.cs] : 0.0;
      int nn, kb;
      if (b_ncontig) { nn = l & 63; kb = l >> 6; } else { kb = l & 15; nn = l >> 4; }
      int gn = n0 + nn, gkb = k0 + kb;
      rb[q] = (gn < n && gkb < k) ? b[(int64_t)gkb * B.rs + (int64_t)gn * B.cs] : 0.0;
    }
  };
  auto store_regs = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int l = tid + q * 256;
      int mm, kk;
      if (a_kcontig) { kk = l & 15; mm = l >> 4; } else { mm = l & 63; kk = l >> 6; }
      As[buf][kk][mm] = ra[q];
      int nn, kb;
      if (b_ncontig) { nn = l & 63; kb = l >> 6; } else { kb = l & 15; nn = l >> 4; }
      Bs[buf][kb][nn] = rb[q];
    }
  };

  const int nk = (k + BK - 1) / BK;
  load_regs(0);
  store_regs(0);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load_regs((t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double fa[4], fb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) fa[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) fb[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(fa[i], fb[j], acc[i][j]);
    }
    if (t + 1 < nk) store_regs(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn < n) {
        double* dst = c + (int64_t)gm * C.rs + (int64_t)gn * C.cs;
        *dst = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *dst);
      }
    }
  }
}

}  // namespace

cudaError_t gemm_f64(int m, int n, int k, double alpha, View A, View B, double beta, ViewW C,
                     int batch, cudaStream_t s) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  if ((m + BM - 1) / BM > 65535) return cudaErrorInvalidValue;
  dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM, batch);
  gemm_f64_kernel<<<grid, 256, 0, s>>>(m, n, k, alpha, A, B, beta, C);
  return cudaGetLastError();
}

}  // namespace tnk
