// Host-side schedule: a frozen tree + a network structure + chi expanded into
// a static list of kernel steps with fixed shapes and a static device memory
// plan (the tree is independent of the tensor entries, so one plan serves
// every instance of a batch and every call at that chi).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace tnp {

// Which device buffer a view points into.
enum BufKind : int { BUF_ARENA = 0, BUF_INPUT = 1, BUF_GIN = 2 };  // GIN: adjoints of the inputs,
                                                                    // laid out like the input block

// A 2-D strided view of one instance's matrix: element (r, c) at
// base + r*rs + c*cs; per-instance stride bs.  For the arena, base is
// off * batch (buffers are laid out buffer-major, instance-minor).
struct PView {
  int buf = BUF_ARENA;
  int64_t off = 0;  // arena: per-instance-unit offset; input: element offset
  int64_t rs = 0, cs = 0;
  int64_t bs = 0;   // per-instance stride (arena: the buffer's per-instance size)
  int64_t eo = 0;   // element offset inside each instance's block (sub-matrix views)
};

enum StepKind : int {
  ST_PERMUTE = 0,
  ST_GEMM = 1,
  ST_QR = 2,
  ST_JACOBI = 3,
  ST_SELECT = 4,
  ST_RESCALE = 5,
  ST_FINAL = 6,
  ST_TO_F32 = 7,      // src (FP64) -> dst (FP32), count elements
  ST_JACOBI32 = 8,    // FP32 preconditioning Jacobi on C (float), V = aux1 (float)
  ST_TO_F64 = 9,      // src (FP32) -> dst and out1 (FP64), count elements
  ST_COPY = 10,       // dst <- src, count elements per instance (same per-instance stride)
  ST_APPLYQ = 11,     // C (m x k col-major) <- Q C, Q the reflectors in `work` (m x n QR)
  ST_GEMM_TC = 12,    // C = alpha A B on tcgen05 tensor cores (tc_mode), FP64 in and out, `work` scratch
  // reverse pass
  ST_SCALE_POW2 = 13,   // C (count elements) *= 2^-e, e from rescale tape slot `slot`
  ST_FINAL_GRAD = 14,   // out1 = 1 / C (the root scalar)
  ST_SVD_FACTORS = 15,  // sorted factors of a Jacobi SVD (C = G, aux1 = V, aux2 = sigma; flag = tall)
                        //   -> out1 = U, out2 = W, work = s, A = Us, B = Ws
  ST_SVD_ADJ_CORE = 16, // C (n x n) from A = P, B = Q (n x k), work = s
  ST_COPY2D = 17,       // C view <- A view (m x n)
  ST_MARK_ACTIVE = 18,  // active columns of the FP64 polish: C = G (m x n), k kept -> out1 (n ints per instance)
};
constexpr int kNumStepKinds = 19;

struct Step {
  int kind = 0;
  int op_index = -1;       // tree op this step belongs to
  // permute
  PView src, dst;          // src/dst: rs/cs unused, bs used
  std::vector<int64_t> in_dims;
  std::vector<int> perm;
  // gemm: C = A * B (m x k) (k x n); qr: A view (m x n) -> R view, work buffer
  int m = 0, n = 0, k = 0;
  PView A, B, C;
  PView work;              // qr work (bs = m*n), jacobi V, select outputs ...
  PView aux1, aux2;        // jacobi: V, sigma; select: V, sigma
  PView out1, out2;        // select: X, Y
  int64_t count = 0;       // rescale / convert: elements
  double alpha = 1.0, beta = 0.0;  // gemm: C = alpha A B + beta C
  int init_v = 1;          // jacobi: start from V = I
  int64_t fbs_src = 0, fbs_dst = 0;  // per-instance strides in floats for FP32 buffers
  int tc_mode = 0;         // tensor-core GEMM: 0 TF32, 1 BF16, 2 split TF32
  int64_t work_bytes = 0;  // tensor-core GEMM: scratch bytes for the whole batch (per instance x batch)
  double jac_tol = 1e-9;   // FP64 Jacobi: relative off-diagonal below which a pair counts as converged
  int no_v = 0;            // FP64 Jacobi / select: V not accumulated; select writes K3 into `work`
  int flag = 0;            // apply_q: 1 = apply Q^T; svd factors: 1 = the Jacobi matrix is M (else M^T)
  int slot = -1;           // rescale: tape slot receiving the exponents (reverse-pass plans)
  int lane = 0;            // 1: may run on the side stream, concurrently with the main stream
  int join = 0;            // 1: the main stream waits for the side stream before this step
  // accounting
  double flops = 0.0;      // algorithmic FP64-or-GEMM flops
  double bytes = 0.0;      // algorithmic bytes
};

// Where a tensor version lives after tree op `op_index` (-1: network input).
struct TensorRec {
  int op_index = -1;
  int tensor_id = -1;
  PView view;
  std::vector<int> bonds;       // storage order; ids >= n_bonds are bonds made by compressions
  std::vector<int64_t> dims;
};

struct Plan {
  std::vector<TensorRec> records;
  std::vector<std::pair<int, int>> consumed;  // (op_index, tensor id) of each C op's inputs
  int chi = 0;
  int prec = 0;
  std::vector<Step> steps;
  int64_t arena_units = 0;   // per-instance arena size in doubles
  int64_t n_contractions = 0, n_compressions = 0;
  double gemm_flops = 0, qr_flops = 0, svd_flops = 0, permute_bytes = 0;
  int64_t max_jacobi_n = 0;
  PView final_scalar;
  // reverse-pass plans: the forward keeps every operand, then the steps of the
  // reverse pass follow ST_FINAL; the adjoints of the inputs land in BUF_GIN
  bool grad = false;
  int n_slots = 0;           // rescale tape slots (ints per instance)
  int segments = 1;          // checkpointed segments of the reverse pass (1: one tape of the whole pass)
  int gauge_r = -1;          // tree-gauge distance of the compressions (-1: plain Q-form)
  int64_t in_total = 0;      // elements of the input block per instance
  double bwd_flops = 0;      // GEMM flops of the reverse pass
  uint64_t serial = 0;       // set by the owner; distinct per plan built (keys captured graphs)
};

// Network structure (no data).
struct Structure {
  std::vector<int64_t> bond_dims;
  std::vector<std::vector<int>> bonds;   // per tensor, storage order
  std::vector<int64_t> in_off;           // element offset of each tensor in the input block
  int64_t in_total = 0;
};

// ops: rows {kind, i, j, k}.  Returns "" on success, else an error message.
// grad: also emit the reverse pass (d log|Z| / d inputs); segments > 1 (with
// grad): checkpoint the live tensors at that many segment starts and
// recompute each segment's operands just before its reverse steps.
// gauge_r >= 0: compressions in the tree gauge of distance gauge_r, projector
// form (forward only); -1: the plain Q-form.
std::string build_plan(const Structure& s, const std::vector<int32_t>& ops, int n_inputs, int chi,
                       int prec, Plan* out, bool grad = false, int segments = 1, int gauge_r = -1);

// Validate a tree against a structure without chi (ids, order, final scalar).
std::string validate_tree(const Structure& s, const std::vector<int32_t>& ops, int n_inputs);

}  // namespace tnp
