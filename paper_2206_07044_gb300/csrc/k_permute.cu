// Permute (matricize) kernels: Fig. 3A's grouping of a tensor's indices into
// (left, shared) or (shared, right) order.  Pure data movement, HBM-bound:
// 2 * |T| * 8 bytes per tensor.
//
// The permutation is first reduced to canonical form (size-1 axes dropped,
// input axes that stay adjacent and in order merged), then:
//  * a 32 x 32 shared-memory tile over (input innermost axis, input axis that
//    becomes the output's innermost) when both are at least 16 long, so that
//    both the load and the store are coalesced; the other axes index tiles;
//  * otherwise a gather: one thread per output element (coalesced stores,
//    32-bit index arithmetic), the loads in runs along the preserved or short
//    innermost axes.
#include "tn_kernels.h"

namespace tnk {
namespace {

constexpr int kMaxPermAxes = 64;  // axes of a permute before canonicalization

struct PermParams {
  int nd;
  int64_t n;                      // elements per batch
  int64_t out_dims[kMaxDims];     // output axis sizes
  int64_t in_stride_of_out[kMaxDims];  // input stride of output axis a
};

template <typename I>
__global__ void permute_gather(const double* __restrict__ in, int64_t in_bs, double* __restrict__ out,
                               int64_t out_bs, PermParams p) {
  const int b = blockIdx.y;
  const double* src = in + (int64_t)b * in_bs;
  double* dst = out + (int64_t)b * out_bs;
  const I n = (I)p.n;
  for (I o = (I)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (I)gridDim.x * blockDim.x) {
    I rem = o, off = 0;
    for (int a = p.nd - 1; a > 0; --a) {
      const I d = (I)p.out_dims[a];
      const I q = rem / d;
      off += (rem - q * d) * (I)p.in_stride_of_out[a];
      rem = q;
    }
    off += rem * (I)p.in_stride_of_out[0];
    dst[o] = __ldg(src + off);
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

cudaError_t permute_f64(const double* in, int64_t in_bs, double* out, int64_t out_bs, int nd0,
                        const int64_t* in_dims0, const int* perm0, int batch, cudaStream_t s) {
  // intermediates may carry more bonds than an input tensor (kMaxDims); the
  // canonical form below must fit the kernels' kMaxDims axes
  if (nd0 > kMaxPermAxes || batch <= 0) return cudaErrorInvalidValue;
  // Canonical form: drop size-1 axes, then merge input axes a, a+1 that stay
  // adjacent and in order in the output (they move as one axis).  The
  // boundary contraction's permutes shrink to 2-3 axes this way.
  int keep[kMaxPermAxes], nk = 0, new_of[kMaxPermAxes];
  for (int a = 0; a < nd0; ++a) {
    new_of[a] = -1;
    if (in_dims0[a] > 1) {
      new_of[a] = nk;
      keep[nk++] = a;
    }
  }
  int64_t dims1[kMaxPermAxes];
  int perm1[kMaxPermAxes], np1 = 0;
  for (int q = 0; q < nk; ++q) dims1[q] = in_dims0[keep[q]];
  for (int a = 0; a < nd0; ++a)
    if (new_of[perm0[a]] >= 0) perm1[np1++] = new_of[perm0[a]];
  // merge: group output positions into runs of consecutive input axes
  int64_t in_dims[kMaxPermAxes];
  int perm[kMaxPermAxes], nd = 0;
  {
    int64_t gdim[kMaxPermAxes];
    int gfirst[kMaxPermAxes], ng = 0;
    for (int q = 0; q < np1;) {
      int r = q + 1;
      while (r < np1 && perm1[r] == perm1[r - 1] + 1) ++r;
      int64_t d = 1;
      for (int t = q; t < r; ++t) d *= dims1[perm1[t]];
      gdim[ng] = d;
      gfirst[ng] = perm1[q];
      ++ng;
      q = r;
    }
    // input order of the groups: by their first input axis
    int order[kMaxPermAxes];
    for (int g = 0; g < ng; ++g) order[g] = g;
    for (int i = 1; i < ng; ++i)
      for (int j = i; j > 0 && gfirst[order[j - 1]] > gfirst[order[j]]; --j) {
        int t = order[j];
        order[j] = order[j - 1];
        order[j - 1] = t;
      }
    int in_pos[kMaxPermAxes];
    for (int i = 0; i < ng; ++i) {
      in_dims[i] = gdim[order[i]];
      in_pos[order[i]] = i;
    }
    for (int g = 0; g < ng; ++g) perm[g] = in_pos[g];
    nd = ng;
  }
  if (nd > kMaxDims) return cudaErrorInvalidValue;
  int64_t n = 1;
  int64_t in_stride[kMaxDims];
  for (int a = nd - 1; a >= 0; --a) {
    in_stride[a] = n;
    n *= in_dims[a];
  }
  if (n == 0) return cudaSuccess;
  if (nd == 0) {  // a scalar: copy the single element
    nd = 1;
    in_dims[0] = 1;
    in_stride[0] = 1;
    perm[0] = 0;
  }
  int64_t out_dims[kMaxDims], out_stride[kMaxDims];
  for (int a = 0; a < nd; ++a) out_dims[a] = in_dims[perm[a]];
  {
    int64_t acc = 1;
    for (int a = nd - 1; a >= 0; --a) {
      out_stride[a] = acc;
      acc *= out_dims[a];
    }
  }
  const int ax_x = nd - 1, ax_y = perm[nd - 1];
  const bool tiled = ax_y != ax_x && in_dims[ax_x] >= 16 && in_dims[ax_y] >= 16;
  if (!tiled) {
    // gather: each thread writes one output element (coalesced), reads the input
    // at its offset; the innermost run moves contiguously when it is preserved
    PermParams p{};
    p.nd = nd;
    p.n = n;
    for (int a = 0; a < nd; ++a) {
      p.out_dims[a] = out_dims[a];
      p.in_stride_of_out[a] = in_stride[perm[a]];
    }
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    dim3 grid((unsigned)blocks, (unsigned)batch);
    if (n < (int64_t(1) << 31))
      permute_gather<int32_t><<<grid, 256, 0, s>>>(in, in_bs, out, out_bs, p);
    else
      permute_gather<int64_t><<<grid, 256, 0, s>>>(in, in_bs, out, out_bs, p);
    return cudaGetLastError();
  }
  // tiled path: X = the input's innermost axis, Y = the input axis that becomes the output's innermost
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
    if (a == ax_x || a == ax_y) continue;
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
