// Reduced-precision GEMM on the 5th-generation tensor cores (tcgen05 + TMEM),
// fed by TMA: the pairwise-contraction products of the mixed forms (TF32,
// BF16 or split TF32 inputs, FP32 accumulation; QR, SVD and the Q-form absorb
// stay FP64).
//
//   C (m x n, FP64, any strides) = alpha * A (m x k) * B (k x n)
//
// Operands are first staged by `stage_operand` into K-major, zero-padded
// buffers (A as Mp x Kp, B^T as Np x Kp, rows of 128 bytes per K-block): that
// is the canonical 128-byte-swizzled K-major layout the tensor core reads,
// every TMA box starts on a 128-byte boundary, and ragged m, n, k need no
// special cases in the main loop.  One CTA computes a 128 x BN tile:
//   warp 0 lane 0   issues the TMA loads of a 4-stage ring (mbarrier expect-tx);
//   warp 1 lane 0   issues tcgen05.mma (kind::tf32 K=8 or kind::f16 K=16, M=128)
//                   into a TMEM accumulator of BN FP32 columns, and
//                   tcgen05.commit frees each stage / signals the epilogue;
//   warps 0-3       read the accumulator with tcgen05.ld (lane = row) and
//                   write alpha * D to C in FP64.
// Every mbarrier wait is bounded: after a poll budget the kernel records an
// error in *err, skips its remaining work and still releases its TMEM.  The
// pipeline waits (a free stage for the producer, a loaded stage for the MMA
// issuer) use `pipe_spin` polls (kSpinLimit normally; 0 when a test asks the
// kernel to give up at once); the drain waits that must end before the CTA
// exits -- the TMA copies still in flight, the MMAs still writing TMEM --
// always use kSpinLimit, so an early give-up never leaves asynchronous work
// running behind an exited CTA.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>

#include "tn_cluster.h"
#include "tn_kernels.h"
#include "tn_tune.h"

namespace tnk {
namespace {

constexpr int kTcThreads = 128;
constexpr int kStages = 4;
constexpr int kBM = 128;
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait on phase `parity`; returns false if `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)(16 >> 4) << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)2 << 61;                           // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D = F32, A/B format (TF32 = 2, BF16 = 1), both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t ab_fmt, int n) {
  return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

// kMode: 0 = TF32, 1 = BF16, 2 = split TF32 (A_hi B_hi + A_hi B_lo + A_lo B_hi)
template <int kMode, int BN>
__global__ void __launch_bounds__(kTcThreads) gemm_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                                                             const __grid_constant__ CUtensorMap mapB, int m,
                                                             int n, int kblocks, double alpha, ViewW C,
                                                             int64_t a_rows_per_batch, int64_t b_rows_per_batch,
                                                             int64_t a_lo_row, int64_t b_lo_row, int* err,
                                                             uint32_t pipe_spin) {
  constexpr bool kBF16 = (kMode == 1);
  constexpr bool kSplit = (kMode == 2);
  constexpr int kStages = kSplit ? 3 : ::tnk::kStages;
  // K-block of 128 bytes per row: 32 TF32 or 64 BF16 elements
  constexpr int kElemBytes = kBF16 ? 2 : 4;
  constexpr int kBK = 128 / kElemBytes;
  constexpr int kMmaK = kBF16 ? 16 : 8;
  // a split stage holds the hi tiles then the lo tiles
  constexpr uint32_t kABytes = kBM * 128 * (kSplit ? 2 : 1), kBBytes = BN * 128 * (kSplit ? 2 : 1);
  constexpr uint32_t kAHalf = kBM * 128, kBHalf = BN * 128;
  constexpr uint32_t kIdesc = make_idesc(kBF16 ? 1u : 2u, BN);
  constexpr int kTmemCols = BN < 32 ? 32 : BN;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzle atoms
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;
  unsigned char* sB = base + kStages * kABytes;
  __shared__ uint64_t full_bar[4], empty_bar[4], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile_n = blockIdx.x, tile_m = blockIdx.y, b = blockIdx.z;
  const int ya = (int)(b * a_rows_per_batch) + tile_m * kBM;
  const int yb = (int)(b * b_rows_per_batch) + tile_n * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer: TMA ring
    int issued = 0;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages) {
        if (!mbar_wait(&empty_bar[s], ((kb / kStages) - 1) & 1, pipe_spin)) {
          atomicExch(&abort_flag, 1);
          break;
        }
      }
      if (abort_flag) break;
      mbar_expect_tx(&full_bar[s], kABytes + kBBytes);
      tma_load_2d(sA + s * kABytes, &mapA, &full_bar[s], kb * kBK, ya);
      tma_load_2d(sB + s * kBBytes, &mapB, &full_bar[s], kb * kBK, yb);
      if (kSplit) {
        // lo parts live in the second half of the staged rows (row offset = rows per batch x batch count)
        tma_load_2d(sA + s * kABytes + kAHalf, &mapA, &full_bar[s], kb * kBK, ya + (int)a_lo_row);
        tma_load_2d(sB + s * kBBytes + kBHalf, &mapB, &full_bar[s], kb * kBK, yb + (int)b_lo_row);
      }
      issued = kb + 1;
    }
    // Before the CTA can exit, every copy issued must have landed.  The last
    // kStages loads are the only ones the MMA issuer may not have waited for
    // (it can lag by at most the ring's depth), so wait for exactly those, on
    // every path: after a normal run they completed long ago and the test
    // returns at once; after a give-up on either side (possibly decided after
    // this loop ended) they may still be in flight.
    for (int kb = (issued > kStages ? issued - kStages : 0); kb < issued; ++kb)
      mbar_wait(&full_bar[kb % kStages], (kb / kStages) & 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % kStages;
      if (!mbar_wait(&full_bar[s], (kb / kStages) & 1, pipe_spin)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
      for (int kk = 0; kk < kBK / kMmaK; ++kk) {
        const uint64_t ad = sw128_desc(a0 + kk * kMmaK * kElemBytes);
        const uint64_t bd = sw128_desc(b0 + kk * kMmaK * kElemBytes);
        const uint32_t accum = (kb > 0 || kk > 0) ? 1u : 0u;
        if (kSplit) {
          const uint64_t adl = sw128_desc(a0 + kAHalf + kk * kMmaK * kElemBytes);
          const uint64_t bdl = sw128_desc(b0 + kBHalf + kk * kMmaK * kElemBytes);
          asm volatile(
              "{\n .reg .pred p, q;\n setp.ne.u32 p, %6, 0;\n setp.eq.u32 q, %6, %6;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %5, p;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %3, %5, q;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %4, %2, %5, q;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "l"(bdl), "l"(adl), "r"(kIdesc), "r"(accum)
              : "memory");
        } else if (kBF16) {
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(kIdesc), "r"(accum)
              : "memory");
        } else {
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(kIdesc), "r"(accum)
              : "memory");
        }
      }
      // the stage is free once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty_bar[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&done_bar))
                 : "memory");
  }
  // epilogue: every warp reads its 32 TMEM lanes (= rows of the tile)
  const bool ok = mbar_wait(&done_bar, 0);
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) atomicExch(&abort_flag, 1);
  __syncthreads();
  if (!abort_flag) {
    const int row = tile_m * kBM + warp * 32 + lane;
    double* c = C.p + (int64_t)b * C.bs;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < m) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int col = tile_n * BN + c0 + q;
          if (col < n) c[(int64_t)row * C.rs + (int64_t)col * C.cs] = alpha * (double)__uint_as_float(v[q]);
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
  return t;
}

// FP64 strided view -> K-major padded FP32 / BF16 rows: out[r][kk] = src(r, kk)
// (rows = m of A or n of B), zero outside the logical matrix.  Split TF32
// also writes lo = tf32(x - hi) `lo_off` elements further on.
template <int kMode>
__global__ void stage_operand_kernel(const double* __restrict__ src, int64_t rs, int64_t cs, int64_t bs, int rows,
                                     int cols, int rows_p, int cols_p, void* dst, int64_t lo_off) {
  constexpr bool kBF16 = (kMode == 1);
  const int b = blockIdx.y;
  const int64_t total = (int64_t)rows_p * cols_p;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols_p), k = (int)(i % cols_p);
    const double x = (r < rows && k < cols) ? src[(int64_t)b * bs + (int64_t)r * rs + (int64_t)k * cs] : 0.0;
    if (kBF16) {
      reinterpret_cast<__nv_bfloat16*>(dst)[(int64_t)b * total + i] = __float2bfloat16_rn((float)x);
    } else {
      // round to the nearest TF32 value (the tensor core reads the top 19 bits)
      const float xf = (float)x;
      const uint32_t hi = to_tf32(xf);
      reinterpret_cast<uint32_t*>(dst)[(int64_t)b * total + i] = hi;
      if (kMode == 2)
        reinterpret_cast<uint32_t*>(dst)[lo_off + (int64_t)b * total + i] = to_tf32(xf - __uint_as_float(hi));
    }
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

// 2-D map over a K-major buffer of `rows` rows x `kp` elements; box = box_rows x 128 bytes.
bool make_map(CUtensorMap* map, void* ptr, bool bf16, int64_t rows, int64_t kp, int box_rows) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  const int eb = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(kp * eb)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / eb), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int kMode, int BN>
cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, int m, int n, int kblocks, double alpha,
                      ViewW C, int64_t arows, int64_t brows, int64_t alo, int64_t blo, int tiles_m, int tiles_n,
                      int batch, int* err, cudaStream_t s, uint32_t pipe_spin) {
  const int stages = kMode == 2 ? 3 : kStages;
  const int split = kMode == 2 ? 2 : 1;
  const size_t smem = 1024 + (size_t)stages * split * (kBM * 128 + BN * 128);
  cudaError_t ae = once_per_device((const void*)gemm_tc_kernel<kMode, BN>, [&] {
    return cudaFuncSetAttribute(gemm_tc_kernel<kMode, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (ae != cudaSuccess) return ae;
  dim3 grid(tiles_n, tiles_m, batch);
  gemm_tc_kernel<kMode, BN><<<grid, kTcThreads, smem, s>>>(ma, mb, m, n, kblocks, alpha, C, arows, brows, alo, blo,
                                                           err, pipe_spin);
  return cudaGetLastError();
}

int pick_bn(int n, int mode) {
  if (mode == 2) return n <= 64 ? 64 : 128;
  return n <= 64 ? 64 : (n <= 128 ? 128 : 256);
}

}  // namespace

size_t gemm_tc_workspace_bytes(int m, int n, int k, int mode, int batch) {
  const int eb = mode == 1 ? 2 : 4, bk = 128 / eb, split = mode == 2 ? 2 : 1;
  // B^T padded to a multiple of the largest N tile, so any tile choice fits
  const int64_t mp = (int64_t)(m + kBM - 1) / kBM * kBM, np = (int64_t)(n + 255) / 256 * 256;
  const int64_t kp = (int64_t)((k > 0 ? k : 1) + bk - 1) / bk * bk;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  return (size_t)(up(mp * kp * eb * batch * split) + up(np * kp * eb * batch * split) + 256);
}

cudaError_t gemm_tc(int m, int n, int k, double alpha, View A, View B, ViewW C, int batch, int mode,
                    void* workspace, size_t ws_bytes, int* err, cudaStream_t s, bool give_up_at_once) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  const uint32_t spin = give_up_at_once ? 0u : kSpinLimit;
  if (mode < 0 || mode > 2) return cudaErrorInvalidValue;
  if (batch > 65535 || ws_bytes < gemm_tc_workspace_bytes(m, n, k, mode, batch)) return cudaErrorInvalidValue;
  const bool bf16 = mode == 1;
  const int eb = bf16 ? 2 : 4, bk = 128 / eb, split = mode == 2 ? 2 : 1;
  // a measured N tile (tn_autotune) first; split TF32 has no 256-wide variant
  int bn = tune_get(TK_GEMMTC, m, n, k, batch);
  if (!(bn == 64 || bn == 128 || (bn == 256 && mode != 2))) bn = pick_bn(n, mode);
  const int64_t mp = (int64_t)(m + kBM - 1) / kBM * kBM, np = (int64_t)(n + bn - 1) / bn * bn;
  const int64_t kp = (int64_t)((k > 0 ? k : 1) + bk - 1) / bk * bk;
  if (mp * batch * split > INT32_MAX || np * batch * split > INT32_MAX) return cudaErrorInvalidValue;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  void* a_st = ws;
  void* b_st = ws + up(mp * kp * eb * batch * split);
  // stage A (m x k) and B^T (n x k) K-major, zero padded; split TF32 stores the
  // lo rows after all the hi rows (one tensor map covers both)
  {
    int64_t tot = mp * kp;
    int g = (int)((tot + 255) / 256 > 2048 ? 2048 : (tot + 255) / 256);
    const int64_t alo = mp * kp * batch, blo = np * kp * batch;
    if (mode == 1)
      stage_operand_kernel<1><<<dim3(g, batch), 256, 0, s>>>(A.p, A.rs, A.cs, A.bs, m, k, (int)mp, (int)kp, a_st, 0);
    else if (mode == 2)
      stage_operand_kernel<2><<<dim3(g, batch), 256, 0, s>>>(A.p, A.rs, A.cs, A.bs, m, k, (int)mp, (int)kp, a_st, alo);
    else
      stage_operand_kernel<0><<<dim3(g, batch), 256, 0, s>>>(A.p, A.rs, A.cs, A.bs, m, k, (int)mp, (int)kp, a_st, 0);
    tot = np * kp;
    g = (int)((tot + 255) / 256 > 2048 ? 2048 : (tot + 255) / 256);
    // B^T(r = col of B, kk) = B(kk, r): rows stride = B.cs, k stride = B.rs
    if (mode == 1)
      stage_operand_kernel<1><<<dim3(g, batch), 256, 0, s>>>(B.p, B.cs, B.rs, B.bs, n, k, (int)np, (int)kp, b_st, 0);
    else if (mode == 2)
      stage_operand_kernel<2><<<dim3(g, batch), 256, 0, s>>>(B.p, B.cs, B.rs, B.bs, n, k, (int)np, (int)kp, b_st, blo);
    else
      stage_operand_kernel<0><<<dim3(g, batch), 256, 0, s>>>(B.p, B.cs, B.rs, B.bs, n, k, (int)np, (int)kp, b_st, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, a_st, bf16, mp * batch * split, kp, kBM) || !make_map(&mb, b_st, bf16, np * batch * split, kp, bn))
    return cudaErrorInvalidValue;
  const int kblocks = (int)(kp / bk);
  const int tm = (int)(mp / kBM), tn = (int)(np / bn);
  const int64_t alo_row = mp * batch, blo_row = np * batch;
  if (mode == 2) {
    if (bn == 64) return launch_tc<2, 64>(ma, mb, m, n, kblocks, alpha, C, mp, np, alo_row, blo_row, tm, tn, batch, err, s, spin);
    return launch_tc<2, 128>(ma, mb, m, n, kblocks, alpha, C, mp, np, alo_row, blo_row, tm, tn, batch, err, s, spin);
  }
  if (bf16) {
    if (bn == 64) return launch_tc<1, 64>(ma, mb, m, n, kblocks, alpha, C, mp, np, 0, 0, tm, tn, batch, err, s, spin);
    if (bn == 128) return launch_tc<1, 128>(ma, mb, m, n, kblocks, alpha, C, mp, np, 0, 0, tm, tn, batch, err, s, spin);
    return launch_tc<1, 256>(ma, mb, m, n, kblocks, alpha, C, mp, np, 0, 0, tm, tn, batch, err, s, spin);
  }
  if (bn == 64) return launch_tc<0, 64>(ma, mb, m, n, kblocks, alpha, C, mp, np, 0, 0, tm, tn, batch, err, s, spin);
  if (bn == 128) return launch_tc<0, 128>(ma, mb, m, n, kblocks, alpha, C, mp, np, 0, 0, tm, tn, batch, err, s, spin);
  return launch_tc<0, 256>(ma, mb, m, n, kblocks, alpha, C, mp, np, 0, 0, tm, tn, batch, err, s, spin);
}

}  // namespace tnk
