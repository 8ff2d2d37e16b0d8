// Internal launchers of the CUDA kernels (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace tnk {

constexpr int kMaxDims = 24;

// A batched strided 2-D view: element (r, c) of batch b at p[b*bs + r*rs + c*cs].
struct View {
  const double* p;
  int64_t rs, cs, bs;
};
struct ViewW {
  double* p;
  int64_t rs, cs, bs;
};

// Per-instance bookkeeping on the device.
struct DevState {
  long long* expo;   // [batch] running power-of-two exponent E
  int* status;       // [batch] 0 = ok, else a tn_status-like code set by a kernel
};

// out[b] = in[b] with axes permuted: output axis a is input axis perm[a].
// in_dims are the input's axis sizes (row-major).  Bandwidth-bound.
cudaError_t permute_f64(const double* in, int64_t in_bs, double* out, int64_t out_bs, int nd,
                        const int64_t* in_dims, const int* perm, int batch, cudaStream_t s);

// C[b] = alpha * A[b] (m x k) * B[b] (k x n) + beta * C[b], FP64 on the CUDA cores
// (beta == 0 never reads C).
cudaError_t gemm_f64(int m, int n, int k, double alpha, View A, View B, double beta, ViewW C,
                     int batch, cudaStream_t s);

// Householder QR of A[b] (m x n, any strides): R factor out, reflectors kept.
// work: column-major m x n scratch per batch (stride work_bs >= m*n), followed
// by batch * n doubles of tau; on return it holds the reflectors for
// apply_q_f64.  R: row-major r x n output (r = min(m, n)), zero below the diagonal.
cudaError_t qr_r_f64(int m, int n, View A, double* work, int64_t work_bs, ViewW R, int batch,
                     cudaStream_t s);

// One-sided Jacobi SVD of G[b] (m x n column-major, m >= n, leading dim m):
// on return G holds G V (columns sigma_i u_i) and V (n x n column-major) the
// accumulated rotations (V = I first when init_v), sig the FP64 column norms
// sigma_i (unsorted).  ws: 64 ints per batch of scratch.  Sets st.status[b] = -9
// if the bounded sweep loop ran out.
// sweep_ctr (optional, device): the sweeps run are added to it.  max_sweeps
// caps the sweep loop (0: 60 sweeps).  active (optional): see mark_active_f64.
cudaError_t jacobi_svd_f64(int m, int n, double* G, int64_t g_bs, double* V, int64_t v_bs,
                           double* sig, int64_t sig_bs, int* ws, DevState st, int init_v,
                           int batch, cudaStream_t s, unsigned long long* sweep_ctr = nullptr,
                           double sig_tol = 1e-8, int max_sweeps = 0, const int* active = nullptr,
                           int64_t act_bs = 0);
// Active columns of the FP64 polish (act: n ints per matrix, stride act_bs):
// 1 for the columns of G (m x n column-major) ranked below k + 16 by norm or
// within a factor 2 of the k-th largest norm, 0 for the rest; all 1 when the
// k-th norm is below 1e-4 |G|_F or k + 16 >= n.  The polish rotates every
// pair but judges convergence only on pairs with an active column.
cudaError_t mark_active_f64(int m, int n, int k, const double* G, int64_t g_bs, int* act, int64_t act_bs, int batch,
                            cudaStream_t s);
// The FP32 preconditioning pass (V = I first); never sets a status.
cudaError_t jacobi_svd_f32(int m, int n, float* G, int64_t g_bs, float* V, int64_t v_bs, int* ws,
                           DevState st, int batch, cudaStream_t s, unsigned long long* sweep_ctr = nullptr,
                           int max_sweeps = 0);
// y = (float) x and y1 (= y2 when given) = (double) x, n elements per batch.
cudaError_t convert_f64_to_f32(const double* x, int64_t n, int64_t xbs, float* y, int64_t ybs,
                               int batch, cudaStream_t s);
cudaError_t convert_f32_to_f64(const float* x, int64_t n, int64_t xbs, double* y1, double* y2,
                               int64_t ybs, int batch, cudaStream_t s);

// After Jacobi: pick the k largest sigma and write the truncated factors
// with sigma^1/2 absorbed: L[:, p] = g_i / sqrt(sigma_i) (= u_i sqrt(sigma_i)),
// R[:, p] = V[:, i] sqrt(sigma_i); column-major with leading dims ldl >= m,
// ldr >= n, rows beyond m (n) zero-filled.  With V == nullptr, R's rows
// 0..n-1 are left for a GEMM R = G0^T K3 (G0 the Jacobi input) and K3
// (m x k column-major) receives g_i / sigma_i^3/2, zero for sigma_i <=
// 1e-13 sigma_max (those columns of L are zero too).
cudaError_t select_scale_f64(int m, int n, int k, const double* G, int64_t g_bs, const double* V,
                             int64_t v_bs, const double* sig, int64_t sig_bs, double* L, int64_t l_bs,
                             int ldl, double* R, int64_t r_bs, int ldr, int batch, cudaStream_t s,
                             double* K3 = nullptr, int64_t k3_bs = 0);

// X[b] <- Q[b] X[b], Q the Householder product a qr_r_f64 call left in `work`
// (same m, n, work, work_bs and batch).  X: m x k column-major (ld m).
// trans = 1: X[b] <- Q[b]^T X[b] instead.
cudaError_t apply_q_f64(int m, int n, const double* work, int64_t work_bs, double* X, int64_t x_bs, int k,
                        int batch, cudaStream_t s, int trans = 0);

// X[b] *= 2^-e_b with e_b the binary exponent of max|X[b]|; st.expo[b] += e_b.
// maxbits: [batch] device scratch; e_out (optional, [batch]) receives e_b.
cudaError_t rescale_f64(double* X, int64_t n, int64_t bs, unsigned long long* maxbits, DevState st,
                        int batch, cudaStream_t s, int* e_out = nullptr);

// Final: out_log[b] = ln|x[b]| + expo[b] ln 2 (device arrays), out_sign[b].
cudaError_t finalize_f64(const double* x, int64_t bs, DevState st, double* out_log, int* out_sign,
                         int batch, cudaStream_t s);

// Fill a batch of n x n column-major matrices with the identity.
cudaError_t set_identity_f64(double* V, int n, int64_t bs, int batch, cudaStream_t s);

// Mixed-precision GEMM on tcgen05 tensor cores (TF32 or BF16 inputs, FP32
// accumulation in TMEM, TMA-fed): C = alpha * A * B written as FP64.
// workspace: device scratch of gemm_tc_workspace_bytes(...) bytes (16-byte
// aligned) for the K-major staged operands; err: device int set to 1 if a
// bounded wait inside the kernel ran out.
// mode: 0 = TF32, 1 = BF16, 2 = split TF32 (3 products, about FP32 accuracy).
size_t gemm_tc_workspace_bytes(int m, int n, int k, int mode, int batch);
// give_up_at_once (tests of the bounded waits): the pipeline waits give up
// without polling, so the kernel sets *err and returns after draining its copies.
cudaError_t gemm_tc(int m, int n, int k, double alpha, View A, View B, ViewW C, int batch, int mode,
                    void* workspace, size_t ws_bytes, int* err, cudaStream_t s, bool give_up_at_once = false);

// ---- reverse pass (d log|Z| / d inputs)

// X[b] *= 2^-e[b] (the adjoint of a rescale that divided by 2^e[b]).
cudaError_t scale_pow2_f64(double* X, int64_t n, int64_t bs, const int* e, int batch, cudaStream_t s);

// g[b] = 1 / x[b]: the adjoint of ln|x| for the final scalar.
cudaError_t final_grad_f64(const double* x, int64_t xbs, double* g, int64_t gbs, int batch, cudaStream_t s);

// From a Jacobi SVD of J (m x n column-major, m >= n: G = J V holds sigma_i u_i,
// V the right vectors, sig unsorted) build, in descending order of sigma
// (ties by index, as select_scale_f64 ranks them), the factors of M = J when
// tall, else M = J^T:  U (rows_u x n, ld rows_u), W (rows_w x n, ld rows_w)
// with M = U diag(s) W^T, s (n), and the first k columns scaled by s^-1/2:
// Us (rows_u x k), Ws (rows_w x k).  Columns with sigma <= 1e-13 sigma_max get
// u_i = 0 (when u comes from G) and s^-1/2 = 0.
cudaError_t svd_factors_f64(int m, int n, int k, int tall, const double* G, int64_t g_bs, const double* V,
                            int64_t v_bs, const double* sig, int64_t sig_bs, double* U, int64_t u_bs, double* W,
                            int64_t w_bs, double* s_out, int64_t s_bs, double* Us, int64_t us_bs, double* Ws,
                            int64_t ws_bs, int batch, cudaStream_t s);

// Core matrix of the truncated-SVD adjoint (q x q column-major):
//   C_ij = F_ij (a_ij - a_ji) s_j + s_i F_ij (b_ij - b_ji) + [i == j < k] (P_ii + Q_ii) / (2 s_i^1/2)
// with a_ij = P_ij s_j^1/2, b_ij = Q_ij s_j^1/2 for j < k (0 otherwise),
// F_ij = d / (d^2 + 1e-12 s_0^2), d = s_j^2 - s_i^2 (F_ii = 0), s descending;
// P, Q: q x k column-major.
cudaError_t svd_adjoint_core_f64(int q, int k, const double* P, int64_t p_bs, const double* Q, int64_t q_bs,
                                 const double* s, int64_t s_bs, double* C, int64_t c_bs, int batch, cudaStream_t st);

// Y[b] (m x n) <- X[b] (m x n), both strided views.
cudaError_t copy2d_f64(int m, int n, View X, ViewW Y, int batch, cudaStream_t s);

}  // namespace tnk
