// SVD of the compression core R_AB = R_A L_B (Eq. "svd"): one-sided (Hestenes)
// Jacobi.  Columns of G are rotated pairwise until mutually orthogonal; then
// G = U diag(sigma) and the accumulated rotations are V.
//
// GB300 runs FP32 58x faster than FP64 (measured 69.7 vs 1.19 TFLOP/s), so the
// core SVD runs in two precisions:
//   1. FP32 Jacobi on a float copy of the core, from V = I, until every pair's
//      relative off-diagonal is below 3e-4 (pairs below 4 m eps32 are skipped
//      on the way), then one finishing sweep that rotates every pair above
//      16 eps32: it takes the off-diagonals from ~1e-4 to the FP32 rounding
//      level, which saves the FP64 stage one of its sweeps;
//   2. (host schedule) V is re-orthonormalised in FP64 by two Newton-Schulz
//      steps V <- V (3 I - V^T V) / 2 (from ~1e-5 to below 1e-16) and
//      G = M V is formed in FP64;
//   3. FP64 Jacobi on that G, starting from V, which converges quadratically in
//      about 2 sweeps to FP64 accuracy.
// The FP64 result is the exact-arithmetic fixed point of step 3; step 1 only
// supplies the starting basis.
//
// Parallel layout: one thread-block cluster of P CTAs per matrix.  The columns
// are cut into 2P blocks; a sweep is 2P-1 rounds of the round-robin "circle"
// pairing of blocks, one block pair per CTA.  The CTA stages its two blocks of
// G and V in shared memory and orthogonalises the pair there (every column
// pair within the union in round 0, the cross pairs in later rounds), so
// cluster barriers separate rounds, not rotations.  Column norms are cached in
// shared memory, computed exactly at every load and after every rotation
// (fused into the rotation loop: the analytic update alpha' = alpha - t gamma
// loses a small column to cancellation).  Columns whose norm is at the
// rounding floor of the matrix (|g| <= floor_rel |G|_F) are left unrotated:
// they carry no direction, and their singular values fall below the
// truncation's zero cut anyway.
//
// A sweep counts the pairs whose relative off-diagonal |gamma| / sqrt(alpha
// beta) exceeded `sig_tol` when visited (they are rotated all the same); the
// matrix has converged when a sweep counts none, since the sweep's own
// rotations then leave off-diagonals of about sig_tol^2 / gap.  The sweep loop is bounded: a matrix that has not
// converged after max_sweeps reports TN_ENOCONV (-9) in its status word.
#include <cooperative_groups.h>

#include <cfloat>

#include "tn_cluster.h"
#include "tn_kernels.h"
#include "tn_tune.h"

namespace cg = cooperative_groups;

namespace tnk {
namespace {

constexpr int kThreads = 256;      // pair_jacobi_kernel and the small kernels
constexpr int kMaxJacThreads = 512; // block_jacobi_kernel: one warp per column of a block, 8..16 warps
constexpr int kWsInts = 64;   // per-matrix scratch: counters + 16 per-CTA double partials

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ void circle_pair(int rnd, int k, int np, int& a, int& b) {
  const int mmod = np - 1;
  if (k == 0) {
    a = np - 1;
    b = rnd % mmod;
  } else {
    a = (rnd + k) % mmod;
    b = (rnd - k + mmod) % mmod;
  }
}

template <typename T>
struct JacArgs {
  int m, n;
  T* G;
  int64_t g_bs;
  T* V;
  int64_t v_bs;
  double* sig;      // optional FP64 column norms out (may be null)
  int64_t sig_bs;
  int* ws;          // kWsInts per matrix: 3 sweep counters, then (from int 8) one double per CTA
  int* status;
  int init_v;
  int max_sweeps;
  T tol;            // rotate iff |gamma| > tol * sqrt(alpha beta)
  T sig_tol;        // ... and the pair is not yet converged iff |gamma| > sig_tol * sqrt(alpha beta)
  T floor_rel;      // columns with |g| <= floor_rel * |G|_F are left alone
  T fin_tol;        // > 0: after convergence, one more sweep rotating every pair above fin_tol
  T floor2;         // (set in the kernel) floor_rel^2 * |G|_F^2
  T tol2, sig_tol2; // (set in the kernel) tol^2, sig_tol^2
  T noise2;         // (set in the kernel) (64 eps |G|_F)^2: the matrix's rounding floor for an off-diagonal
  unsigned long long* sweep_ctr;  // optional: total sweeps run, summed over matrices
  const int* active;  // optional, n ints per matrix (stride act_bs): convergence is judged on pairs
  int64_t act_bs;     //   with at least one active column (every pair is still rotated)
};

// Squared Frobenius norm of G.  Each CTA writes its partial sum to its own
// scratch slot and every CTA adds the P slots in rank order, so the value is
// bit-identical run to run (the truncated contraction can be chaotic in
// rounding, so the whole path avoids order-dependent floating-point atomics).
template <typename T>
__device__ T cluster_fro2(cg::cluster_group& cl, const T* G, int m, int n, int rank, int P, double* slots) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ double wpart[32];
  double part = 0.0;
  for (int c = warp; c < n; c += nwarps) {
    if (c % P != rank) continue;
    const T* gc = G + (int64_t)c * m;
    double s2 = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double x = (double)__ldcg(gc + r);
      s2 = fma(x, x, s2);
    }
    part += warp_sum(s2);
  }
  if (lane == 0) wpart[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nwarps; ++w) t += wpart[w];
    slots[rank] = t;
  }
  cl.sync();
  double tot = 0.0;
  for (int r = 0; r < P; ++r) tot += __ldcg(slots + r);
  return (T)tot;
}

template <typename T>
__device__ __forceinline__ T ab_max(T a, T b) {
  return a > b ? a : b;
}

template <typename T, bool kGlobal>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (kGlobal) return __ldcg(p); else return *p;
}

// Rotate columns x, y (length len, contiguous) by (c, s): x' = c x - s y, y' = s x + c y.
template <typename T, bool kGlobal>
__device__ __forceinline__ void rot_cols_g(T* x, T* y, int len, T c, T s, int lane) {
  for (int r = lane; r < len; r += 32) {
    const T a = ld<T, kGlobal>(x + r), b = ld<T, kGlobal>(y + r);
    x[r] = c * a - s * b;
    y[r] = s * a + c * b;
  }
}

// Same, and return the exact squared norms of the rotated columns (analytic
// norm updates lose the small column to cancellation when alpha >> beta).
template <typename T, bool kGlobal>
__device__ __forceinline__ void rot_cols_norms(T* x, T* y, int len, T c, T s, int lane, T& nx, T& ny) {
  T ax = T(0), ay = T(0);
  for (int r = lane; r < len; r += 32) {
    const T a = ld<T, kGlobal>(x + r), b = ld<T, kGlobal>(y + r);
    const T xa = c * a - s * b, yb = s * a + c * b;
    x[r] = xa;
    y[r] = yb;
    ax = fma(xa, xa, ax);
    ay = fma(yb, yb, ay);
  }
  nx = warp_sum(ax);
  ny = warp_sum(ay);
}

// Returns true if the pair was rotated significantly.  kGlobal: the columns
// live in global memory written by other CTAs (loads bypass L1).
template <typename T, bool kGlobal = false>
__device__ __forceinline__ bool jacobi_pair(T* gx, T* gy, T* vx, T* vy, int m, int n, T& al, T& be,
                                            const JacArgs<T>& p, int lane) {
  // columns at the rounding floor of the matrix carry no direction: leave them
  if (!(al > p.floor2) || !(be > p.floor2)) return false;
  T ga = T(0);
  for (int r = lane; r < m; r += 32) ga = fma(ld<T, kGlobal>(gx + r), ld<T, kGlobal>(gy + r), ga);
  ga = warp_sum(ga);
  // The tests |gamma| > tol sqrt(alpha beta) are made on squares (no square
  // root or division), and the rotation takes one square root, one division
  // and one reciprocal square root: every lane of the warp evaluates these
  // scalars, and on the FP64 pipe they cost more than the column updates.
  //   t = tan(theta) = sgn(d) h / (|d| + sqrt(d^2 + h^2)),  d = beta - alpha, h = 2 gamma
  // (the smaller root of t^2 + 2 (d / h) t - 1 = 0), c = 1 / sqrt(1 + t^2), s = c t.
  const T g2 = ga * ga, ab = al * be;
  if (!(g2 > p.tol2 * ab)) return false;
  const T d = be - al, h = T(2) * ga;
  const T t = (d >= T(0) ? h : -h) / (fabs(d) + sqrt(d * d + h * h));
  const T c = rsqrt(T(1) + t * t);
  const T s = c * t;
  const T mx = ab_max(al, be);
  __syncwarp();
  rot_cols_norms<T, kGlobal>(gx, gy, m, c, s, lane, al, be);
  if (vx) rot_cols_g<T, kGlobal>(vx, vy, n, c, s, lane);
  // Not yet converged: the relative off-diagonal exceeds sig_tol, and the
  // off-diagonal itself is above the rounding floor of the matrix.  A column
  // of norm |y| << |G|_F receives rounding of order eps |G|_F from every
  // rotation against a large column, so its relative off-diagonals stall near
  // eps |G|_F / |y|; such a pair can only turn the large column by ~eps and is
  // counted as converged.
  return g2 > p.sig_tol2 * ab && g2 > p.noise2 * mx;
}

template <typename T>
__global__ void __launch_bounds__(kMaxJacThreads) block_jacobi_kernel(JacArgs<T> p) {
  cg::cluster_group cl = cg::this_cluster();
  const int P = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int bidx = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int m = p.m, n = p.n;
  const int nblk = 2 * P;
  const int b = (n + nblk - 1) / nblk;
  T* G = p.G + (int64_t)bidx * p.g_bs;
  const bool has_v = (p.V != nullptr);  // without V only G is rotated
  T* V = has_v ? p.V + (int64_t)bidx * p.v_bs : nullptr;
  int* cnt = p.ws + kWsInts * bidx;
  {
    const T fro2 = cluster_fro2(cl, G, m, n, rank, P, reinterpret_cast<double*>(cnt + 8));
    // the rounding-floor test serves the FP64 polish; the FP32 preconditioner
    // keeps the plain relative test (its floor would be far coarser)
    const T eps64 = sizeof(T) == sizeof(double) ? T(64) * T(DBL_EPSILON) : T(0);
    p.floor2 = p.floor_rel * p.floor_rel * fro2;
    p.noise2 = eps64 * eps64 * fro2;
  }
  p.tol2 = p.tol * p.tol;
  p.sig_tol2 = p.sig_tol * p.sig_tol;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Gs = reinterpret_cast<T*>(smem_raw);                  // 2b columns of length m
  T* Vs = Gs + (size_t)2 * b * m;                          // 2b columns of length n (if V)
  T* nrm = Vs + (has_v ? (size_t)2 * b * n : 0);           // 2b cached squared norms
  int* col = reinterpret_cast<int*>(nrm + 2 * b);          // global column of each slot (-1 = pad)
  int* act = col + 2 * b;                                  // 1 if the slot's column is active
  const int* active = p.active ? p.active + (int64_t)bidx * p.act_bs : nullptr;
  __shared__ int sig_rot_s;

  if (has_v && p.init_v) {
    for (int c = rank; c < n; c += P)
      for (int r = threadIdx.x; r < n; r += blockDim.x) V[(int64_t)c * n + r] = (r == c) ? T(1) : T(0);
  }
  if (rank == 0 && threadIdx.x < 3) cnt[threadIdx.x] = 0;
  cl.sync();

  bool converged = (n < 2), finishing = false;
  int sweeps_run = 0;
  const int sweep_cap = p.max_sweeps + (p.fin_tol > T(0) ? 1 : 0);
  for (int sweep = 0; sweep < sweep_cap && !converged; ++sweep) {
    ++sweeps_run;
    if (rank == 0 && threadIdx.x == 0) cnt[(sweep + 1) % 3] = 0;
    if (threadIdx.x == 0) sig_rot_s = 0;
    int sig_rot = 0;
    for (int rnd = 0; rnd < nblk - 1; ++rnd) {
      int pa, pb;
      circle_pair(rnd, rank, nblk, pa, pb);
      // stage blocks pa (slots 0..b-1) and pb (slots b..2b-1)
      for (int s = threadIdx.x; s < 2 * b; s += blockDim.x) {
        const int gc = (s < b ? pa : pb) * b + (s % b);
        col[s] = gc < n ? gc : -1;
        act[s] = (gc < n && (!active || active[gc])) ? 1 : 0;
      }
      __syncthreads();
      for (int s = warp; s < 2 * b; s += nwarps) {
        const int gc = col[s];
        T* gs = Gs + (size_t)s * m;
        T acc = T(0);
        if (gc >= 0) {
          const T* gg = G + (int64_t)gc * m;
          for (int r = lane; r < m; r += 32) {
            const T x = __ldcg(gg + r);
            gs[r] = x;
            acc = fma(x, x, acc);
          }
          if (has_v) {
            T* vs = Vs + (size_t)s * n;
            const T* vv = V + (int64_t)gc * n;
            for (int r = lane; r < n; r += 32) vs[r] = __ldcg(vv + r);
          }
        }
        acc = warp_sum(acc);
        if (lane == 0) nrm[s] = acc;
      }
      __syncthreads();
      if (rnd == 0) {
        // every pair of the 2b columns: circle over 2b players
        const int np = 2 * b;
        for (int ir = 0; ir < np - 1; ++ir) {
          for (int k = warp; k < np / 2; k += nwarps) {
            int x, y;
            circle_pair(ir, k, np, x, y);
            if (col[x] < 0 || col[y] < 0) continue;
            if (x > y) { int t = x; x = y; y = t; }
            T al = nrm[x], be = nrm[y];
            if (jacobi_pair(Gs + (size_t)x * m, Gs + (size_t)y * m, has_v ? Vs + (size_t)x * n : nullptr,
                            has_v ? Vs + (size_t)y * n : nullptr, m, n, al, be, p, lane) &&
                (act[x] | act[y]))
              sig_rot += (lane == 0);
            if (lane == 0) { nrm[x] = al; nrm[y] = be; }
          }
          __syncthreads();
        }
      } else {
        // cross pairs only: (i, b + (i + t) mod b)
        for (int t = 0; t < b; ++t) {
          for (int i = warp; i < b; i += nwarps) {
            const int x = i, y = b + (i + t) % b;
            if (col[x] < 0 || col[y] < 0) continue;
            T al = nrm[x], be = nrm[y];
            if (jacobi_pair(Gs + (size_t)x * m, Gs + (size_t)y * m, has_v ? Vs + (size_t)x * n : nullptr,
                            has_v ? Vs + (size_t)y * n : nullptr, m, n, al, be, p, lane) &&
                (act[x] | act[y]))
              sig_rot += (lane == 0);
            if (lane == 0) { nrm[x] = al; nrm[y] = be; }
          }
          __syncthreads();
        }
      }
      // write the pair back
      for (int s = warp; s < 2 * b; s += nwarps) {
        const int gc = col[s];
        if (gc < 0) continue;
        T* gg = G + (int64_t)gc * m;
        const T* gs = Gs + (size_t)s * m;
        for (int r = lane; r < m; r += 32) gg[r] = gs[r];
        if (has_v) {
          T* vv = V + (int64_t)gc * n;
          const T* vs = Vs + (size_t)s * n;
          for (int r = lane; r < n; r += 32) vv[r] = vs[r];
        }
      }
      cl.sync();
    }
    sig_rot = __reduce_add_sync(0xffffffffu, sig_rot);
    if (lane == 0 && sig_rot) atomicAdd(&sig_rot_s, sig_rot);
    __syncthreads();
    if (threadIdx.x == 0 && sig_rot_s) atomicAdd(cnt + (sweep % 3), sig_rot_s);
    cl.sync();
    converged = (__ldcg(cnt + (sweep % 3)) == 0);
    if (finishing) {
      converged = true;
    } else if (converged && p.fin_tol > T(0)) {
      converged = false;
      finishing = true;
      p.tol2 = p.fin_tol * p.fin_tol;
    }
  }
  if (!converged && p.status && rank == 0 && threadIdx.x == 0) atomicExch(p.status + bidx, -9);
  if (p.sweep_ctr && rank == 0 && threadIdx.x == 0) atomicAdd(p.sweep_ctr, (unsigned long long)sweeps_run);
  if (p.sig) {
    double* sig = p.sig + (int64_t)bidx * p.sig_bs;
    for (int c = rank * nwarps + warp; c < n; c += P * nwarps) {
      const T* gc = G + (int64_t)c * m;
      double s2 = 0.0;
      for (int r = lane; r < m; r += 32) {
        const double x = (double)__ldcg(gc + r);
        s2 = fma(x, x, s2);
      }
      s2 = warp_sum(s2);
      if (lane == 0) sig[c] = sqrt(s2);
    }
  }
}

// Fallback for matrices whose block pairs do not fit in shared memory: one
// column pair per warp straight from global memory (L2), a cluster barrier
// per round of the circle ordering.
template <typename T>
__global__ void __launch_bounds__(kThreads) pair_jacobi_kernel(JacArgs<T> p) {
  cg::cluster_group cl = cg::this_cluster();
  const int P = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int bidx = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int m = p.m, n = p.n;
  T* G = p.G + (int64_t)bidx * p.g_bs;
  T* V = p.V ? p.V + (int64_t)bidx * p.v_bs : nullptr;
  int* cnt = p.ws + kWsInts * bidx;
  {
    const T fro2 = cluster_fro2(cl, G, m, n, rank, P, reinterpret_cast<double*>(cnt + 8));
    // the rounding-floor test serves the FP64 polish; the FP32 preconditioner
    // keeps the plain relative test (its floor would be far coarser)
    const T eps64 = sizeof(T) == sizeof(double) ? T(64) * T(DBL_EPSILON) : T(0);
    p.floor2 = p.floor_rel * p.floor_rel * fro2;
    p.noise2 = eps64 * eps64 * fro2;
  }
  p.tol2 = p.tol * p.tol;
  p.sig_tol2 = p.sig_tol * p.sig_tol;
  const int np = n + (n & 1);
  const int gw = rank * nwarps + warp, nw = P * nwarps;
  if (V && p.init_v) {
    for (int c = rank; c < n; c += P)
      for (int r = threadIdx.x; r < n; r += blockDim.x) V[(int64_t)c * n + r] = (r == c) ? T(1) : T(0);
  }
  if (rank == 0 && threadIdx.x < 3) cnt[threadIdx.x] = 0;
  cl.sync();
  bool converged = (n < 2), finishing = false;
  int sweeps_run = 0;
  const int sweep_cap = p.max_sweeps + (p.fin_tol > T(0) ? 1 : 0);
  for (int sweep = 0; sweep < sweep_cap && !converged; ++sweep) {
    ++sweeps_run;
    if (rank == 0 && threadIdx.x == 0) cnt[(sweep + 1) % 3] = 0;
    int sig_rot = 0;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int k = gw; k < np / 2; k += nw) {
        int a, bb;
        circle_pair(rnd, k, np, a, bb);
        if (a >= n || bb >= n) continue;
        const int i = a < bb ? a : bb, j = a < bb ? bb : a;
        T* gi = G + (int64_t)i * m;
        T* gj = G + (int64_t)j * m;
        T al = T(0), be = T(0);
        for (int r = lane; r < m; r += 32) {
          const T x = __ldcg(gi + r), y = __ldcg(gj + r);
          al = fma(x, x, al);
          be = fma(y, y, be);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        __syncwarp();
        const bool counted = !p.active || p.active[(int64_t)bidx * p.act_bs + i] | p.active[(int64_t)bidx * p.act_bs + j];
        if (jacobi_pair<T, true>(gi, gj, V ? V + (int64_t)i * n : nullptr, V ? V + (int64_t)j * n : nullptr, m, n,
                                 al, be, p, lane) && counted)
          sig_rot += (lane == 0);
      }
      cl.sync();
    }
    sig_rot = __reduce_add_sync(0xffffffffu, sig_rot);
    if (lane == 0 && sig_rot) atomicAdd(cnt + (sweep % 3), sig_rot);
    cl.sync();
    converged = (__ldcg(cnt + (sweep % 3)) == 0);
    if (finishing) {
      converged = true;
    } else if (converged && p.fin_tol > T(0)) {
      converged = false;
      finishing = true;
      p.tol2 = p.fin_tol * p.fin_tol;
    }
  }
  if (!converged && p.status && rank == 0 && threadIdx.x == 0) atomicExch(p.status + bidx, -9);
  if (p.sweep_ctr && rank == 0 && threadIdx.x == 0) atomicAdd(p.sweep_ctr, (unsigned long long)sweeps_run);
  if (p.sig) {
    double* sig = p.sig + (int64_t)bidx * p.sig_bs;
    for (int c = gw; c < n; c += nw) {
      const T* gc = G + (int64_t)c * m;
      double s2 = 0.0;
      for (int r = lane; r < m; r += 32) {
        const double x = (double)__ldcg(gc + r);
        s2 = fma(x, x, s2);
      }
      s2 = warp_sum(s2);
      if (lane == 0) sig[c] = sqrt(s2);
    }
  }
}

template <typename T>
size_t block_smem(int m, int n, int P, bool has_v) {
  const int b = (n + 2 * P - 1) / (2 * P);
  return (size_t)2 * b * (m + (has_v ? n : 0)) * sizeof(T) + (size_t)2 * b * (sizeof(T) + 2 * sizeof(int)) + 16;
}

constexpr size_t kSmemCap = 200 * 1024;

template <typename T>
cudaError_t launch_jacobi(const JacArgs<T>& a, int batch, cudaStream_t s) {
  if (a.n <= 0 || batch <= 0) return cudaSuccess;
  if (a.m < a.n || batch > 65535) return cudaErrorInvalidValue;
  cudaError_t ze = cudaMemsetAsync(a.ws, 0, sizeof(int) * kWsInts * (size_t)batch, s);
  if (ze != cudaSuccess) return ze;
  // cluster size: at most one block pair of 8 columns per CTA and 16 CTAs
  // (non-portable size); within [pmax/2, pmax] the size with the fewest
  // waves per CTA of work for this batch
  int pmax = a.n / 16;
  if (pmax > 16) pmax = 16;
  if (pmax < 1) pmax = 1;
  cudaError_t ae = once_per_device((const void*)block_jacobi_kernel<T>, [] {
    cudaError_t e = cudaFuncSetAttribute(block_jacobi_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(block_jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    return e;
  });
  if (ae != cudaSuccess) return ae;
  const bool has_v = a.V != nullptr;
  auto smem_of = [&](int q) {
    const size_t sm = block_smem<T>(a.m, a.n, q, has_v);
    return sm <= kSmemCap ? sm : (size_t)-1;
  };
  // a round pairs b = n / 2P columns with b others: b pairs per inner step, one
  // per warp; the CTA gets b warps (8 at least, 16 at most)
  auto warps_of = [&](int q) {
    const int b = (a.n + 2 * q - 1) / (2 * q);
    return b < 8 ? 8 : (b > kMaxJacThreads / 32 ? kMaxJacThreads / 32 : b);
  };
  auto threads_of = [&](int q) { return 32 * warps_of(q); };
  auto imbalance = [&](int q) {
    const int b = (a.n + 2 * q - 1) / (2 * q);
    const int nw = warps_of(q);
    return (double)((b + nw - 1) / nw * nw) / b;
  };
  // The FP64 polish is bound by the SM's FP64 pipe, so a wave counts clusters
  // whose CTAs each own an SM; the FP32 pass is latency-bound and shares SMs well.
  const bool fp64 = sizeof(T) == sizeof(double);
  // a measured choice (tn_autotune) first, else the residency rule
  const int tp = tune_get(fp64 ? TK_JAC64 : TK_JAC32, a.m, a.n, 0, batch);
  int P = (tp >= 1 && tp <= 16 && smem_of(tp) != (size_t)-1)
              ? tp
              : choose_cluster((const void*)block_jacobi_kernel<T>, batch, pmax / 2 > 0 ? pmax / 2 : 1, pmax, smem_of,
                               imbalance, threads_of, fp64);
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(P > 0 ? threads_of(P) : kThreads, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (P > 0) {
    cfg.gridDim = dim3(P, batch, 1);
    attr[0].val.clusterDim.x = P;
    cfg.dynamicSmemBytes = smem_of(P);
    return cudaLaunchKernelEx(&cfg, block_jacobi_kernel<T>, a);
  }
  // block pairs do not fit in shared memory: column pairs from global memory
  P = a.n / 64;
  if (P > 8) P = 8;
  if (P < 1) P = 1;
  cfg.gridDim = dim3(P, batch, 1);
  attr[0].val.clusterDim.x = P;
  cfg.dynamicSmemBytes = 0;
  return cudaLaunchKernelEx(&cfg, pair_jacobi_kernel<T>, a);
}

// Pick the k largest sigma and write the truncated factors of Eq. "svd" with
// sigma^1/2 absorbed on each side: left column p = g_i / sqrt(sigma_i)
// (= u_i sigma_i^1/2, since G's columns are sigma_i u_i) and right column p =
// v_i sigma_i^1/2.  Outputs are column-major with leading dimensions ldl / ldr;
// rows m..ldl-1 (n..ldr-1) are zero-filled so that a Householder product can
// be applied to them directly.  Ties keep the lower index first.
//
// Without V (the polish did not accumulate it), the right factor is recovered
// afterwards as v_i sigma_i^1/2 = M^T g_i / sigma_i^3/2 by a GEMM: this kernel
// writes K3[:, p] = g_i / sigma_i^3/2 and only zero-fills rows n..ldr-1 of R.
// Components with sigma_i <= 1e-13 sigma_max are dropped on both sides there:
// M^T g_i / sigma_i^3/2 carries an error of eps |M| / sqrt(sigma_i), which
// must stay small next to the true sqrt(sigma_i).
__global__ void select_scale_kernel(int m, int n, int k, const double* Gall, int64_t g_bs,
                                    const double* Vall, int64_t v_bs, const double* sigall,
                                    int64_t sig_bs, double* Lall, int64_t l_bs, int ldl, double* Rall,
                                    int64_t r_bs, int ldr, double* K3all, int64_t k3_bs) {
  const int b = blockIdx.x;
  const double* G = Gall + (int64_t)b * g_bs;
  const double* V = Vall ? Vall + (int64_t)b * v_bs : nullptr;
  const double* sig = sigall + (int64_t)b * sig_bs;
  double* L = Lall + (int64_t)b * l_bs;
  double* R = Rall + (int64_t)b * r_bs;
  double* K3 = K3all ? K3all + (int64_t)b * k3_bs : nullptr;
  extern __shared__ int rank_of[];
  __shared__ double smax;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, sig[i]);
    smax = mx;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = sig[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const double sj = sig[j];
      r += (sj > si) || (sj == si && j < i);
    }
    rank_of[i] = r;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int i = warp; i < n; i += nwarps) {
    const int p = rank_of[i];
    if (p >= k) continue;
    const double si = sig[i];
    const double rs = sqrt(si);
    if (V) {
      const double sl = si > 0.0 ? 1.0 / rs : 0.0;
      for (int r = lane; r < ldl; r += 32) L[(int64_t)p * ldl + r] = r < m ? G[(int64_t)i * m + r] * sl : 0.0;
      for (int r = lane; r < ldr; r += 32) R[(int64_t)p * ldr + r] = r < n ? V[(int64_t)i * n + r] * rs : 0.0;
    } else {
      const bool keep = si > 1e-13 * smax && si > 0.0;
      const double sl = keep ? 1.0 / rs : 0.0, s3 = keep ? 1.0 / (si * rs) : 0.0;
      for (int r = lane; r < ldl; r += 32) L[(int64_t)p * ldl + r] = r < m ? G[(int64_t)i * m + r] * sl : 0.0;
      for (int r = lane; r < m; r += 32) K3[(int64_t)p * m + r] = G[(int64_t)i * m + r] * s3;
      for (int r = n + lane; r < ldr; r += 32) R[(int64_t)p * ldr + r] = 0.0;
    }
  }
}

// Active columns of the FP64 polish (one CTA per matrix).  G (m x n, column
// major) is the FP64 product M V with V the re-orthonormalised FP32 basis, so
// its column norms are the singular values to FP32 accuracy.  Only the k
// largest enter the truncation (Eq. "svd"), so the polish judges convergence
// on the pairs that touch them: it still rotates every pair (skipping pairs
// would let the coupling of two skipped columns flow back into kept ones), but
// a pair of two inactive columns no longer keeps the sweep loop alive.  Column
// i is active when its rank is below k + 16 or its norm is at least half the
// k-th largest.  When the k-th norm is within 1e-4 of |G|_F (where the FP32
// ordering is not trusted) or k + 16 >= n, every column is active.
__global__ void mark_active_kernel(int m, int n, int k, const double* Gall, int64_t g_bs, int* act_all,
                                   int64_t act_bs) {
  const int b = blockIdx.x;
  const double* G = Gall + (int64_t)b * g_bs;
  int* act = act_all + (int64_t)b * act_bs;
  extern __shared__ double nrm2[];
  __shared__ double fro2_s, kth_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int c = warp; c < n; c += nwarps) {
    double s2 = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double x = G[(int64_t)c * m + r];
      s2 = fma(x, x, s2);
    }
    s2 = warp_sum(s2);
    if (lane == 0) nrm2[c] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int c = 0; c < n; ++c) f += nrm2[c];
    fro2_s = f;
    kth_s = -1.0;
  }
  __syncthreads();
  // the k-th largest: the column of rank k - 1 (ties by index)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = nrm2[i];
    int r = 0;
    for (int j = 0; j < n; ++j) r += (nrm2[j] > si) || (nrm2[j] == si && j < i);
    if (r == k - 1) kth_s = si;
    act[i] = r;  // rank, replaced by the flag below
  }
  __syncthreads();
  const double kth = kth_s;
  const bool all = (k + 16 >= n) || !(kth >= 1e-8 * fro2_s);
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    act[i] = (all || act[i] < k + 16 || nrm2[i] >= 0.25 * kth) ? 1 : 0;
}

constexpr int kMarkMaxN = 6144;  // n doubles of shared memory within the 48 KB default

__global__ void all_active_kernel(int n, int* act_all, int64_t act_bs) {
  int* act = act_all + (int64_t)blockIdx.x * act_bs;
  for (int i = threadIdx.x; i < n; i += blockDim.x) act[i] = 1;
}

__global__ void to_f32_kernel(const double* __restrict__ x, int64_t n, int64_t xbs, float* __restrict__ y,
                              int64_t ybs) {
  const int b = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[(int64_t)b * ybs + i] = (float)x[(int64_t)b * xbs + i];
}

__global__ void to_f64_kernel(const float* __restrict__ x, int64_t n, int64_t xbs, double* __restrict__ y1,
                              double* __restrict__ y2, int64_t ybs) {
  const int b = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[(int64_t)b * xbs + i];
    y1[(int64_t)b * ybs + i] = v;
    if (y2) y2[(int64_t)b * ybs + i] = v;
  }
}

int grid1d(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 1024 ? 1024 : (g < 1 ? 1 : g));
}

}  // namespace

cudaError_t jacobi_svd_f32(int m, int n, float* G, int64_t g_bs, float* V, int64_t v_bs, int* ws,
                           DevState st, int batch, cudaStream_t s, unsigned long long* sweep_ctr, int max_sweeps) {
  // a preconditioner: running out of sweeps is not an error (the FP64 stage decides)
  JacArgs<float> a{m, n, G, g_bs, V, v_bs, nullptr, 0, ws, nullptr, 1, max_sweeps > 0 ? max_sweeps : 60,
                   4.0f * (float)m * FLT_EPSILON, 3e-4f, 1e-6f, 16.0f * FLT_EPSILON, 0.0f, 0.0f, 0.0f, 0.0f,
                   sweep_ctr, nullptr, 0};
  return launch_jacobi(a, batch, s);
}

cudaError_t jacobi_svd_f64(int m, int n, double* G, int64_t g_bs, double* V, int64_t v_bs, double* sig,
                           int64_t sig_bs, int* ws, DevState st, int init_v, int batch, cudaStream_t s,
                           unsigned long long* sweep_ctr, double sig_tol, int max_sweeps, const int* active,
                           int64_t act_bs) {
  // rotate down to sqrt(m) eps (the cut's subspace error is that over the gap);
  // convergence is judged by the looser sig_tol, so rounding-level rotations
  // never keep the sweep loop alive
  const double rt = sqrt((double)(m > 16 ? m : 16));
  JacArgs<double> a{m, n, G, g_bs, V, v_bs, sig, sig_bs, ws, st.status, init_v, max_sweeps > 0 ? max_sweeps : 60,
                    rt * DBL_EPSILON, sig_tol, 1e-14, 0.0, 0.0, 0.0, 0.0, 0.0, sweep_ctr, active, act_bs};
  return launch_jacobi(a, batch, s);
}

cudaError_t select_scale_f64(int m, int n, int k, const double* G, int64_t g_bs, const double* V,
                             int64_t v_bs, const double* sig, int64_t sig_bs, double* L, int64_t l_bs,
                             int ldl, double* R, int64_t r_bs, int ldr, int batch, cudaStream_t s,
                             double* K3, int64_t k3_bs) {
  if (batch <= 0 || k <= 0) return cudaSuccess;
  if (n > 8192 || ldl < m || ldr < n || (!V && !K3)) return cudaErrorInvalidValue;
  select_scale_kernel<<<batch, 256, (size_t)n * sizeof(int), s>>>(m, n, k, G, g_bs, V, v_bs, sig, sig_bs, L,
                                                                   l_bs, ldl, R, r_bs, ldr, K3, k3_bs);
  return cudaGetLastError();
}

cudaError_t mark_active_f64(int m, int n, int k, const double* G, int64_t g_bs, int* act, int64_t act_bs, int batch,
                            cudaStream_t s) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  if (k < 1 || batch > 65535) return cudaErrorInvalidValue;
  if (n > kMarkMaxN) {  // too wide for the shared-memory ranking: every column counts
    all_active_kernel<<<batch, 256, 0, s>>>(n, act, act_bs);
    return cudaGetLastError();
  }
  mark_active_kernel<<<batch, 256, (size_t)n * sizeof(double), s>>>(m, n, k, G, g_bs, act, act_bs);
  return cudaGetLastError();
}

cudaError_t convert_f64_to_f32(const double* x, int64_t n, int64_t xbs, float* y, int64_t ybs, int batch,
                               cudaStream_t s) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  to_f32_kernel<<<dim3(grid1d(n), batch), 256, 0, s>>>(x, n, xbs, y, ybs);
  return cudaGetLastError();
}

cudaError_t convert_f32_to_f64(const float* x, int64_t n, int64_t xbs, double* y1, double* y2, int64_t ybs,
                               int batch, cudaStream_t s) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  to_f64_kernel<<<dim3(grid1d(n), batch), 256, 0, s>>>(x, n, xbs, y1, y2, ybs);
  return cudaGetLastError();
}

}  // namespace tnk
