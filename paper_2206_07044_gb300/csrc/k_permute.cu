// Permute (matricize) kernels: Fig. 3A's grouping of a tensor's indices into
// (left, shared) or (shared, right) order.  Pure data movement, HBM-bound:
// 2 * |T| * 8 bytes per tensor.
//
// Two paths:
//  * the output's innermost axis is the input's innermost axis: a gather whose
//    reads and writes are both contiguous runs along that axis;
//  * otherwise a 32 x 32 shared-memory tile over (input innermost axis,
//    input axis that becomes the output's innermost), so that both the load
//    and the store are coalesced; the other axes index tiles.
#include "tn_kernels.h"

namespace tnk {
namespace {

struct PermParams {
  int nd;
  int64_t n;                      // elements per batch
  int64_t out_dims[kMaxDims];     // output axis sizes
  int64_t in_stride_of_out[kMaxDims];  // input stride of output axis a
};

__global__ void permute_gather(const double* __restrict__ in, int64_t in_bs, double* __restrict__ out,
                               int64_t out_bs, PermParams p) {
  const int b = blockIdx.y;
  const double* src = in + (int64_t)b * in_bs;
  double* dst = out + (int64_t)b * out_bs;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < p.n;
       o += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = o, off = 0;
    for (int a = p.nd - 1; a >= 0; --a) {
      int64_t c = rem % p.out_dims[a];
      rem /= p.out_dims[a];
      off += c * p.in_stride_of_out[a];
    }
    dst[o] = src[off];
  }
}

// Tiled transpose over input axis X (innermost, stride 1) and input axis Y
// (the output's innermost).  "Outer" axes are every other axis.
struct TileParams {
  int64_t nx, ny;                 // sizes of X and Y
  int64_t out_stride_x;           // output stride of axis X
  int64_t in_stride_y;            // input stride of axis Y
  int n_outer;
  int64_t outer_dims[kMaxDims];
  int64_t outer_in_stride[kMaxDims];
  int64_t outer_out_stride[kMaxDims];
  int64_t tiles_x, tiles_y;
};

__global__ void permute_tiled(const double* __restrict__ in, int64_t in_bs, double* __restrict__ out,
                              int64_t out_bs, TileParams p) {
  __shared__ double tile[32][33];
  const int b = blockIdx.z;
  const int64_t t = blockIdx.x;
  const int64_t tx = t % p.tiles_x, ty = t / p.tiles_x;
  // outer coordinates from blockIdx.y (grid-stride for large outer counts)
  int64_t n_outer_total = 1;
  for (int a = 0; a < p.n_outer; ++a) n_outer_total *= p.outer_dims[a];
  for (int64_t ob = blockIdx.y; ob < n_outer_total; ob += gridDim.y) {
    int64_t rem = ob, in_off = 0, out_off = 0;
    for (int a = p.n_outer - 1; a >= 0; --a) {
      int64_t c = rem % p.outer_dims[a];
      rem /= p.outer_dims[a];
      in_off += c * p.outer_in_stride[a];
      out_off += c * p.outer_out_stride[a];
    }
    const double* src = in + (int64_t)b * in_bs + in_off;
    double* dst = out + (int64_t)b * out_bs + out_off;
    const int64_t x0 = tx * 32, y0 = ty * 32;
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      int64_t x = x0 + threadIdx.x, y = y0 + j;
      if (x < p.nx && y < p.ny) tile[j][threadIdx.x] = src[y * p.in_stride_y + x];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      int64_t y = y0 + threadIdx.x, x = x0 + j;
      if (x < p.nx && y < p.ny) dst[x * p.out_stride_x + y] = tile[threadIdx.x][j];
    }
  }
}

}  // namespace

cudaError_t permute_f64(const double* in, int64_t in_bs, double* out, int64_t out_bs, int nd,
                        const int64_t* in_dims, const int* perm, int batch, cudaStream_t s) {
  if (nd > kMaxDims || batch <= 0) return cudaErrorInvalidValue;
  int64_t n = 1;
  int64_t in_stride[kMaxDims];
  for (int a = nd - 1; a >= 0; --a) {
    in_stride[a] = n;
    n *= in_dims[a];
  }
  if (n == 0) return cudaSuccess;
  int64_t out_dims[kMaxDims], out_stride[kMaxDims];
  for (int a = 0; a < nd; ++a) out_dims[a] = in_dims[perm[a]];
  {
    int64_t acc = 1;
    for (int a = nd - 1; a >= 0; --a) {
      out_stride[a] = acc;
      acc *= out_dims[a];
    }
  }
  // drop size-1 axes when deciding the path
  int last_in = -1;
  for (int a = nd - 1; a >= 0; --a)
    if (in_dims[a] > 1) { last_in = a; break; }
  int last_out = -1;
  for (int a = nd - 1; a >= 0; --a)
    if (out_dims[a] > 1) { last_out = a; break; }
  if (last_in < 0 || last_out < 0 || perm[last_out] == last_in || nd == 1) {
    PermParams p{};
    p.nd = nd;
    p.n = n;
    for (int a = 0; a < nd; ++a) {
      p.out_dims[a] = out_dims[a];
      p.in_stride_of_out[a] = in_stride[perm[a]];
    }
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    dim3 grid((unsigned)blocks, (unsigned)batch);
    permute_gather<<<grid, 256, 0, s>>>(in, in_bs, out, out_bs, p);
    return cudaGetLastError();
  }
  // tiled path: X = input axis last_in, Y = input axis perm[last_out]
  const int ax_x = last_in, ax_y = perm[last_out];
  int out_pos_of_in[kMaxDims];
  for (int a = 0; a < nd; ++a) out_pos_of_in[perm[a]] = a;
  TileParams p{};
  p.nx = in_dims[ax_x];
  p.ny = in_dims[ax_y];
  p.out_stride_x = out_stride[out_pos_of_in[ax_x]];
  p.in_stride_y = in_stride[ax_y];
  p.n_outer = 0;
  int64_t n_outer_total = 1;
  for (int a = 0; a < nd; ++a) {
    if (a == ax_x || a == ax_y || in_dims[a] == 1) continue;
    p.outer_dims[p.n_outer] = in_dims[a];
    p.outer_in_stride[p.n_outer] = in_stride[a];
    p.outer_out_stride[p.n_outer] = out_stride[out_pos_of_in[a]];
    p.n_outer++;
    n_outer_total *= in_dims[a];
  }
  p.tiles_x = (p.nx + 31) / 32;
  p.tiles_y = (p.ny + 31) / 32;
  int64_t gy = n_outer_total < 65535 ? n_outer_total : 65535;
  dim3 grid((unsigned)(p.tiles_x * p.tiles_y), (unsigned)gy, (unsigned)batch);
  permute_tiled<<<grid, dim3(32, 8), 0, s>>>(in, in_bs, out, out_bs, p);
  return cudaGetLastError();
}

}  // namespace tnk
