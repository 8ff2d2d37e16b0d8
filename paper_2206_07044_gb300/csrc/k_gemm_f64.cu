// FP64 GEMM on the CUDA cores: C = alpha * A * B for the pairwise
// contractions (A = T_i as (left x shared), B = T_j as (shared x right)), the
// R_A L_B core and the Newton-Schulz / preconditioning products of the core SVD.
//
// GB300 runs FP64 at 2 DFMA / clock / SM (about 1.2 TFLOP/s for the chip), so
// these products are FP64-pipe bound at any realistic size; the kernel keeps
// TM x TN independent DFMAs per thread per k-step and stages the operand
// tiles through shared memory with coalesced loads for either operand
// orientation (the schedule passes row- or column-major views instead of
// permuting).
#include "tn_kernels.h"
#include "tn_tune.h"

namespace tnk {
namespace {

constexpr int BK = 16;

// One CTA of 256 threads (16 x 16) computes a BM x BN tile, TM x TN outputs
// per thread (BM = 16 TM, BN = 16 TN); operand tiles BM x BK and BK x BN are
// double-buffered in shared memory (under the 48 KB static limit).  Variants
// (tn_autotune picks one per shape): 64 x 64 (4 x 4), 32 x 32 (2 x 2) for
// small products, 128 x 32 (8 x 2) and 128 x 16 (8 x 1) for tall products
// with few columns (the row absorptions of a boundary contraction).
template <int TM, int TN>
__global__ void __launch_bounds__(256) gemm_f64_kernel(int m, int n, int k, double alpha, View A,
                                                       View B, double beta, ViewW C) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;  // elements per thread per tile
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

  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  double ra[LA], rb[LB];
  // coalesced loads along whichever index is contiguous in memory
  auto a_idx = [&](int l, int& mm, int& kk) {
    if (a_kcontig) { kk = l % BK; mm = l / BK; } else { mm = l % BM; kk = l / BM; }
  };
  auto b_idx = [&](int l, int& nn, int& kb) {
    if (b_ncontig) { nn = l % BN; kb = l / BN; } else { kb = l % BK; nn = l / BK; }
  };
  auto load_regs = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      int mm, kk;
      a_idx(tid + q * 256, mm, kk);
      const int gm = m0 + mm, gk = k0 + kk;
      ra[q] = (gm < m && gk < k) ? a[(int64_t)gm * A.rs + (int64_t)gk * A.cs] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      int nn, kb;
      b_idx(tid + q * 256, nn, kb);
      const int gn = n0 + nn, gkb = k0 + kb;
      rb[q] = (gn < n && gkb < k) ? b[(int64_t)gkb * B.rs + (int64_t)gn * B.cs] : 0.0;
    }
  };
  auto store_regs = [&](int buf) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      int mm, kk;
      a_idx(tid + q * 256, mm, kk);
      As[buf][kk][mm] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      int nn, kb;
      b_idx(tid + q * 256, nn, kb);
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
      double fa[TM], fb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) fa[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) fb[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(fa[i], fb[j], acc[i][j]);
    }
    if (t + 1 < nk) store_regs(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= m) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn < n) {
        double* dst = c + (int64_t)gm * C.rs + (int64_t)gn * C.cs;
        *dst = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *dst);
      }
    }
  }
}

template <int TM, int TN>
cudaError_t launch_gemm(int m, int n, int k, double alpha, View A, View B, double beta, ViewW C, int batch,
                        cudaStream_t s) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  if ((m + BM - 1) / BM > 65535) return cudaErrorInvalidValue;
  dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM, batch);
  gemm_f64_kernel<TM, TN><<<grid, 256, 0, s>>>(m, n, k, alpha, A, B, beta, C);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_f64(int m, int n, int k, double alpha, View A, View B, double beta, ViewW C,
                     int batch, cudaStream_t s) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  switch (tune_get(TK_GEMM64, m, n, k, batch)) {
    case 2:
      return launch_gemm<2, 2>(m, n, k, alpha, A, B, beta, C, batch, s);
    case 3:
      return launch_gemm<8, 2>(m, n, k, alpha, A, B, beta, C, batch, s);
    case 4:
      return launch_gemm<8, 1>(m, n, k, alpha, A, B, beta, C, batch, s);
    default:
      return launch_gemm<4, 4>(m, n, k, alpha, A, B, beta, C, batch, s);
  }
}

}  // namespace tnk
