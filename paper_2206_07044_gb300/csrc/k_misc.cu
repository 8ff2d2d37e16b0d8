// Running log-norm and final read-out.
//
// After every op each output X is divided by 2^e, e the binary exponent of
// max|X| (max|X| = f 2^e with f in [0.5, 1)), and e is added to the
// instance's exponent E.  Scaling by a power of two is exact, so this changes
// no rounding anywhere; it only keeps intermediates inside the double range
// (log Z of the largest networks is far beyond 709).  At the end
// log|Z| = ln|x| + E ln 2 for the final scalar x.
#include <cmath>

#include "tn_kernels.h"

namespace tnk {
namespace {

__global__ void absmax_kernel(const double* __restrict__ X, int64_t n, int64_t bs,
                              unsigned long long* maxbits) {
  const int b = blockIdx.y;
  const double* x = X + (int64_t)b * bs;
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(x[i]);
    m = (a > m || a != a) ? a : m;  // keeps a NaN (its bit pattern dominates below)
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, m, o);
    m = (t > m || t != t) ? t : m;
  }
  __shared__ double red[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = (red[i] > m || red[i] != red[i]) ? red[i] : m;
    // non-negative doubles (and NaN with the sign bit clear) order like their bit patterns
    atomicMax(maxbits + b, (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void scale_kernel(double* __restrict__ X, int64_t n, int64_t bs,
                             const unsigned long long* maxbits, long long* expo, int* status, int* e_out) {
  const int b = blockIdx.y;
  const double m = __longlong_as_double((long long)maxbits[b]);
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  if (!isfinite(m)) {
    if (lead) {
      atomicExch(status + b, -7);
      if (e_out) e_out[b] = 0;
    }
    return;
  }
  if (m == 0.0) {
    if (lead && e_out) e_out[b] = 0;
    return;
  }
  int e;
  frexp(m, &e);
  if (lead && e_out) e_out[b] = e;
  const double sc = ldexp(1.0, -e);
  double* x = X + (int64_t)b * bs;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= sc;
  if (blockIdx.x == 0 && threadIdx.x == 0) expo[b] += e;
}

__global__ void finalize_kernel(const double* x, int64_t bs, const long long* expo,
                                const int* status, double* out_log, int* out_sign, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const double v = x[(int64_t)b * bs];
  if (status[b] != 0 || !isfinite(v)) {
    out_log[b] = NAN;
    out_sign[b] = 0;
  } else if (v == 0.0) {
    out_log[b] = -INFINITY;
    out_sign[b] = 0;
  } else {
    out_log[b] = log(fabs(v)) + (double)expo[b] * 0.69314718055994530942;
    out_sign[b] = v > 0.0 ? 1 : -1;
  }
}

__global__ void identity_kernel(double* V, int n, int64_t bs) {
  double* v = V + (int64_t)blockIdx.y * bs;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n * n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (i % (n + 1) == 0) ? 1.0 : 0.0;
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t rescale_f64(double* X, int64_t n, int64_t bs, unsigned long long* maxbits, DevState st,
                        int batch, cudaStream_t s, int* e_out) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long) * batch, s);
  if (e != cudaSuccess) return e;
  dim3 grid(grid_for(n), batch);
  absmax_kernel<<<grid, 256, 0, s>>>(X, n, bs, maxbits);
  scale_kernel<<<grid, 256, 0, s>>>(X, n, bs, maxbits, st.expo, st.status, e_out);
  return cudaGetLastError();
}

cudaError_t finalize_f64(const double* x, int64_t bs, DevState st, double* out_log, int* out_sign,
                         int batch, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  finalize_kernel<<<(batch + 127) / 128, 128, 0, s>>>(x, bs, st.expo, st.status, out_log, out_sign,
                                                      batch);
  return cudaGetLastError();
}

cudaError_t set_identity_f64(double* V, int n, int64_t bs, int batch, cudaStream_t s) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid(grid_for((int64_t)n * n), batch);
  identity_kernel<<<grid, 256, 0, s>>>(V, n, bs);
  return cudaGetLastError();
}

}  // namespace tnk
