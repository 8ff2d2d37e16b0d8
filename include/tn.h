/*
 * tn.h -- C ABI of the GB300 approximate tensor-network contraction library.
 *
 * The library executes a frozen, ordered approximate contraction tree
 * (Algorithm 1 of Gray & Chan, "Hyper-optimized approximate contraction of
 * tensor networks with arbitrary geometry", arXiv:2206.07044) on one GPU:
 *
 *   C i j k : pairwise contraction of tensors i and j over all their shared
 *             bonds (Eq. 1 for one pair; Fig. 3B), producing tensor k;
 *   S i j   : compression of the bonds shared by i and j when the product of
 *             their sizes D_AB exceeds chi (Sec. "Bond compression strategies"):
 *             QR of A, LQ of B, truncated SVD of R_A R_B to
 *             k = min(chi, D_A, D_B) singular values, sqrt(sigma) absorbed on
 *             both sides (Eq. "svd"): A_bar = Q_A U_k sigma^1/2 and
 *             B_bar = sigma^1/2 V_k^T Q_B, with the Householder products of the
 *             two QRs applied to the zero-padded factors (the Q-form; Q is
 *             never formed).  The equivalent projector form A P_L, P_R B of the
 *             SI section "Explicit projector form" is used only for
 *             compressions in the tree gauge (tn_set_tree_gauge).
 *
 * A power-of-two running log-norm keeps every intermediate in range, so log|Z|
 * never overflows.  All arithmetic runs in CUDA kernels on the GPU; there is
 * no CPU fallback.
 *
 * Conventions
 *   - Every function returns a tn_status (0 = TN_OK).  No exception crosses
 *     the ABI.  On error, tn_last_error() describes the failure.
 *   - Pointers are host pointers unless stated otherwise.  The library copies
 *     what it keeps; the caller keeps ownership of everything it passes in.
 *   - A context lives on one CUDA device and owns the device memory it
 *     allocates.  Calls are not thread-safe on one context.
 *   - Work is issued on the context's stream (tn_set_stream; default: the
 *     legacy default stream) and calls that return results synchronise it.
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tn_ctx tn_ctx;

typedef enum {
  TN_OK = 0,
  TN_EINVAL = -1,      /* bad argument (null pointer, chi < 1, unknown id, ...) */
  TN_EFORMAT = -2,     /* malformed network or tree (file or descriptor)        */
  TN_ESHAPE = -3,      /* shapes disagree (bond listed != twice, data size, ...) */
  TN_ENOMEM = -4,      /* device or host allocation failed                      */
  TN_ECUDA = -5,       /* a CUDA runtime call or kernel launch failed           */
  TN_ETIMEOUT = -6,    /* a bounded device-side wait ran out                    */
  TN_ENONFINITE = -7,  /* NaN or Inf in input tensor data                       */
  TN_ESTATE = -8,      /* call out of order (e.g. no tree loaded)               */
  TN_ENOCONV = -9      /* an iterative kernel (Jacobi SVD) did not converge     */
} tn_status;

/* Arithmetic form of the contraction and absorb GEMMs.  QR/LQ and the SVD of
 * the R_A L_B core are FP64 in every form. */
typedef enum {
  TN_F64 = 0,    /* every step in FP64 (the plain form)                          */
  TN_TF32 = 1,   /* GEMMs on tcgen05 tensor cores, TF32 inputs, FP32 accumulate  */
  TN_BF16 = 2,   /* GEMMs on tcgen05 tensor cores, BF16 inputs, FP32 accumulate  */
  TN_TF32X3 = 3  /* split-TF32 GEMMs (3 tcgen05 products), near-FP32 accuracy    */
} tn_prec;

/* A closed tensor network (Eq. 1 with no open indices).
 *   n_bonds      number of bonds; bond b has size bond_dims[b] >= 1
 *   n_tensors    number of tensors
 *   ndims[t]     number of bonds of tensor t (0 allowed: a scalar tensor)
 *   bond_ids     concatenation over t of tensor t's bond ids, in storage order;
 *                every bond id must appear in exactly two different tensors
 *   data[t]      host pointer to tensor t's FP64 entries, row-major over its
 *                listed bond order (prod of its bond sizes elements)        */
typedef struct {
  int32_t n_bonds;
  const int64_t* bond_dims;
  int32_t n_tensors;
  const int32_t* ndims;
  const int32_t* bond_ids;
  const double* const* data;
} tn_network_desc;

/* An ordered approximate contraction tree (Fig. 2B/C).
 *   n_inputs     must equal the network's n_tensors
 *   ops          n_ops rows of 4 int32: {0, i, j, k} = C i j k, {1, i, j, -1} = S i j
 *                Ids 0..n_inputs-1 are the network tensors; the m-th C op must
 *                create id n_inputs + m.  The ops must reduce the network to
 *                scalars (every tensor contracted, last op a C).             */
typedef struct {
  int32_t n_inputs;
  int32_t n_ops;
  const int32_t* ops;
} tn_tree_desc;

/* Algorithmic work of one instance at one chi (the SI's cost-tracer units,
 * counted on the schedule the library executes).                            */
typedef struct {
  int64_t n_contractions;     /* C ops                                         */
  int64_t n_compressions;     /* S ops that run at this chi                    */
  double gemm_flops;          /* 2 m n k over contraction, core and absorb GEMMs */
  double qr_flops;            /* Householder 2 m n^2 - 2/3 n^3 per factored side */
  double svd_flops;           /* 4 m n^2 - 4/3 n^3 per core SVD (the SI's count) */
  double permute_bytes;       /* bytes read + written by permutes              */
  double peak_bytes;          /* device arena bytes for one instance           */
  int64_t kernel_launches;    /* kernels per evaluation of this instance       */
} tn_plan_stats;

/* Options of a context (tn_create).  Fill with tn_options_default, then
 * change fields; struct_size lets later versions add fields at the end.
 *   graph_mode         initial tn_set_graph_mode value (default 1)
 *   grad_segments      initial tn_set_grad_segments value (default 0)
 *   tape_budget_bytes  tn_grad with grad_segments 0: the device bytes the
 *                      tape of one batch may take before the pass is
 *                      checkpointed in ceil(sqrt(ops)) segments
 *                      (default 0: half the free device memory)
 *   debug_max_sweeps   > 0: cap the FP64 Jacobi sweep loop of every core
 *                      SVD at this many sweeps (a matrix that needs more
 *                      makes the call return TN_ENOCONV); 0: 60 sweeps.
 *                      For tests of the bounded loop; leave 0 otherwise.
 *   debug_tc_give_up   1: the pipeline waits of the tensor-core GEMM (mixed
 *                      forms) give up without polling, as if their poll
 *                      budget had run out: each such GEMM drains its copies
 *                      in flight, releases its TMEM and flags the call,
 *                      which returns TN_ETIMEOUT.  For tests of the bounded
 *                      waits; leave 0 otherwise.
 *   tuner_cache        path of the autotuner's cache file (NULL: none).  On
 *                      tn_create its choices are loaded if the file exists
 *                      and was written on the same GPU model (a file from
 *                      another model is ignored; an unreadable one gives
 *                      TN_EFORMAT); tn_autotune rewrites it.
 *   sequential_groups  1: a tn_contract_approx call whose instances fall into
 *                      several groups (different structures or trees) runs
 *                      the groups one after the other; 0 (default): as
 *                      concurrent branches of one pass (see
 *                      tn_contract_approx).  Results are identical.
 *   split_batches      k >= 2: each batch of instances sharing a tree runs
 *                      as k concurrent sub-batches (branches of one pass, as
 *                      for several groups), so that one sub-batch's kernels
 *                      fill the SMs another leaves idle; 0 or 1 (default):
 *                      one batch.  Results may differ in the last bits from
 *                      the unsplit batch (launch shapes depend on the batch
 *                      size).  Requires sequential_groups = 0.  On the
 *                      8-instance 32x32 D=4 chi=64 batch it ran slower at
 *                      k = 2 and 4 (the sub-batches' cluster launches
 *                      compete for the same GPCs). */
typedef struct {
  int32_t struct_size;
  int32_t graph_mode;
  int32_t grad_segments;
  int32_t debug_max_sweeps;
  double tape_budget_bytes;
  int32_t debug_tc_give_up;
  int32_t reserved;
  const char* tuner_cache;
  int32_t sequential_groups;
  int32_t split_batches;
} tn_options;

/* Default options (struct_size = sizeof(tn_options)). */
void tn_options_default(tn_options* opt);

/* Create a context on CUDA device `device` with options `opt` (NULL: the
 * defaults).  *out receives the context.  Errors: TN_EINVAL (NULL out, a
 * struct_size smaller than this version's, fields out of range), TN_ECUDA
 * (no such device). */
int tn_create(tn_ctx** out, int device, const tn_options* opt);

/* Autotuner of the launch shapes (tile and cluster sizes): for the plan
 * of the instances' groups at this chi and form, every distinct launch shape
 * of the QR, the FP32 and FP64 Jacobi passes (cluster size P of the
 * one-matrix-per-cluster kernels) and the GEMMs that carry 98% of the plan's
 * GEMM flops (FP64 tile variant; tensor-core N tile) is timed with each
 * candidate on random scratch data of that shape and the plan's batch size
 * (CUDA events, fastest of two launches; the Jacobi passes capped at two
 * sweeps), and the fastest is recorded in the device's table, which the
 * launchers consult before their built-in rules.  Results of later calls may
 * differ in rounding from untuned ones (a different cluster size changes the
 * order of reductions).  Writes the table to options.tuner_cache when set.
 * *n_tuned (may be NULL) receives the number of shapes tuned.  Allocates its
 * own scratch and frees it.  Errors: TN_EINVAL, TN_ENOMEM, TN_ECUDA. */
int tn_autotune(tn_ctx* ctx, int n_inst, const int* inst_ids, int chi, int prec, int* n_tuned);

/* The device's tuned choices as rows of 6 int32 (kernel family, m, n, k,
 * batch, choice): families 1 QR cluster size, 2 FP64 Jacobi cluster size,
 * 3 FP32 Jacobi cluster size, 4 FP64 GEMM tile variant (1 64x64, 2 32x32,
 * 3 128x32, 4 128x16), 5 tensor-core N tile.  Copies up to `cap` rows and
 * returns the number of entries (rows may be NULL when cap is 0). */
int tn_tuned_choices(tn_ctx* ctx, int cap, int32_t* rows);

/* Destroy a context and free its device memory.  NULL is ignored. */
void tn_destroy(tn_ctx* ctx);

/* Issue all later work on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream).  The stream must belong to the context's device. */
int tn_set_stream(tn_ctx* ctx, void* cuda_stream);

/* CUDA-graph replay of whole schedules (batching across instances, Algorithm 1
 * run as one pre-built launch sequence).  mode 1 (default): the first
 * tn_contract_approx on a given (plan, ordered instance list) runs eagerly, the
 * second captures the whole pass (input gather, every kernel and copy of the
 * schedule, both streams) into a graph and launches it, later calls replay it.
 * Results are bitwise identical to eager launches.  A capture the runtime
 * refuses leaves that key on eager launches (counted in `refused`).  Graphs
 * are dropped when the context's device buffers grow.  mode 0: always eager.
 * Profiling (tn_profile_enable) and tn_debug_tensor always run eagerly.
 * Errors: TN_EINVAL for another mode. */
int tn_set_graph_mode(tn_ctx* ctx, int mode);

/* Counters of the graph path since tn_create: graphs captured, replays
 * launched, captures refused.  Any pointer may be NULL. */
int tn_graph_info(const tn_ctx* ctx, int64_t* captured, int64_t* replays, int64_t* refused);

/* Copy a network into the context (host data -> device).  Validates that each
 * bond appears in exactly two tensors and that entries are finite
 * (TN_ENONFINITE otherwise).  *net_id receives the network's id. */
int tn_load_network(tn_ctx* ctx, const tn_network_desc* desc, int* net_id);

/* Same, from a TNNET1 file (format documented in tn_inputs/formats.py). */
int tn_load_network_file(tn_ctx* ctx, const char* path, int* net_id);

/* Replace the entries of a loaded network with new values of the same shapes
 * (e.g. the next beta of a sweep).  data[t] are host pointers when
 * on_device == 0, device pointers on the context's device otherwise.
 * Host data is copied with cudaMemcpyAsync on the context's stream and the
 * call returns once the copy has been issued (host buffers must stay valid
 * until the next synchronising call). */
int tn_set_network_data(tn_ctx* ctx, int net_id, const double* const* data, int on_device);

/* Attach an ordered tree to a loaded network, creating an instance (a
 * network + tree pair).  The tree is validated against the network's shapes
 * (TN_EFORMAT on a malformed op sequence).  *inst_id receives the instance. */
int tn_load_tree(tn_ctx* ctx, int net_id, const tn_tree_desc* desc, int* inst_id);

/* Same, from a "tntree 1" text file. */
int tn_load_tree_file(tn_ctx* ctx, int net_id, const char* path, int* inst_id);

/* Approximately contract n_inst instances at bond dimension chi (>= 1) in the
 * given arithmetic form.  Instances with identical network structure and tree
 * run as one batch (a group: every launch covers the whole group).  Several
 * groups -- instances of uneven trees, such as different random graphs --
 * run as concurrent branches of one pass: each group has its own slice of
 * the device buffers and its own stream pair, forked from and joined back to
 * the context's stream; with graph mode the multi-group pass is captured as
 * one CUDA graph on its second call and replayed after (batching across
 * instances of different shapes, Sec. on beta sweeps and instances).  logabsz_out[n] = ln|Z_n| (-inf when Z_n == 0) and
 * sign_out[n] in {-1, 0, +1} are caller-allocated host arrays of n_inst.
 * Synchronises the context's stream before returning. */
int tn_contract_approx(tn_ctx* ctx, int n_inst, const int* inst_ids, int chi, int prec,
                       double* logabsz_out, int* sign_out);

/* Gradient of the approximate log|Z| with respect to every input tensor
 * (reverse-mode differentiation of Algorithm 1 as executed; the paper gives no
 * adjoint).  Runs the same schedule as tn_contract_approx with every operand
 * kept on the device, then its reverse pass on the GPU:
 *   - a contraction C = A B returns A' = C' B^T and B' = A^T C';
 *   - a rescale by 2^-e (exact, piecewise constant) returns 2^-e times;
 *   - the root scalar x of ln|x| gets 1 / x;
 *   - a compression returns the adjoint of the truncated SVD of X = A B
 *     (A_bar = U_k s^1/2, B_bar = s^1/2 V_k^T up to a gauge the result does not
 *     see), with F_ij = d / (d^2 + 1e-12 s_1^2), d = s_j^2 - s_i^2, and no
 *     inverse for kept singular values at or below 1e-13 s_1; then A' = X' B^T,
 *     B' = A^T X'.  All of it is evaluated in the bases of the forward QRs.
 * The compressions' FP64 Jacobi keeps its rotations in this mode, so log|Z|
 * may differ from tn_contract_approx's in the last bits.  In the mixed forms
 * the contraction GEMMs of both passes run on the tensor cores; everything
 * else stays FP64.
 * grad_out[n] (n < n_inst) points to sum_t |T_t| doubles for instance n: the
 * gradients of the input tensors packed in network order, each row-major over
 * its listed bonds (the layout the network was loaded in); host pointers when
 * on_device == 0, device pointers on the context's device otherwise.
 * logabsz_out / sign_out as for tn_contract_approx.  Device memory: by
 * default every intermediate of the forward pass stays allocated until the
 * call returns; when that tape would exceed half the free device memory the
 * pass is checkpointed instead (see tn_set_grad_segments).
 * Errors: TN_EINVAL (bad ids, NULL pointers), TN_ENONFINITE when some Z == 0
 * (log|Z| has no gradient there; the other instances' outputs are written),
 * TN_ENOMEM, TN_ENOCONV, TN_ETIMEOUT, TN_ECUDA as for tn_contract_approx.
 * Synchronises the context's stream before returning. */
int tn_grad(tn_ctx* ctx, int n_inst, const int* inst_ids, int chi, int prec, double* logabsz_out,
            int* sign_out, double* const* grad_out, int on_device);

/* Compressions in the tree gauge of distance r (Sec. "Bond compression
 * strategies", tree gauge; SI: r-local spanning tree, Algorithm 2; explicit
 * projector form).  r >= 0: before each compression of the bond between A
 * and B, the environment within graph distance r -- a spanning tree grown
 * from {A, B} over tensors made by contractions, closest first, then by the
 * largest product of shared bond sizes, then by the smallest ids -- is put in
 * the tree gauge on virtual copies (QR of each outer tensor over its bonds to
 * its parent, R absorbed into the parent); R_A and L_B of the gauged A and B
 * give the core SVD R_A L_B = U s V^T, and the projectors P_L = L_B V_k s^-1/2,
 * P_R = s^-1/2 U_k^T R_A are applied to the original tensors (A <- A P_L,
 * B <- P_R B; s^-1/2 = 0 for s <= 1e-13 s_1).  No other tensor changes.
 * r = 0 is the projector form of the plain compression.  r = -1 (default):
 * the plain Q-form.  Applies to later tn_contract_approx calls (tn_grad
 * refuses it with TN_EINVAL).  Errors: TN_EINVAL for r < -1. */
int tn_set_tree_gauge(tn_ctx* ctx, int r);

/* Checkpointing of tn_grad's tape.  segments = k >= 2: the forward pass
 * copies the live tensors at the start of each of k segments of the tree's
 * ops (equal op counts) and keeps nothing else; the reverse pass then, for
 * each segment from the last, recomputes that segment from its checkpoint
 * with every operand kept, runs its reverse steps and frees its tape, so the
 * device holds the checkpoints plus one segment's tape (about 1/k of the
 * whole, at the price of one more forward pass).  Results equal the
 * one-tape pass (the recomputation repeats the same kernels on the same
 * data).  segments = 1: one tape of the whole pass.  segments = 0 (default):
 * one tape if it fits in half the free device memory, else ceil(sqrt(ops))
 * segments.  Errors: TN_EINVAL for segments < 0. */
int tn_set_grad_segments(tn_ctx* ctx, int segments);

/* Diagnostic, needs no context and no GPU: the static schedule that
 * tn_contract_approx (grad = 0) or tn_grad (grad = 1; grad = k >= 2: with k
 * checkpointed segments) would run for this, with compressions in the
 * tree gauge of distance gauge_r (-1: the plain form; see tn_set_tree_gauge), for this
 * network structure (the data pointers are not read), tree, chi and form
 * (schedule expansion, Algorithm 1 with explicit ops), written as one JSON
 * object: {"arena_units", "n_slots", "in_total", "grad", "segments", "in_off": [...],
 * "steps": [{"kind", "op", "m", "n", "k", "flag", "slot", "no_v", "init_v",
 * "count", "fbs_src", "fbs_dst", "alpha", "beta", "tc_mode", "A", "B", "C",
 * "src", "dst", "work", "aux1", "aux2", "out1", "out2", "in_dims", "perm"}]},
 * each view as [buffer (0 arena, 1 inputs, 2 input adjoints), offset,
 * row stride, column stride, per-instance stride, element offset]; the step
 * kinds and buffer layouts are those of the library's executor (arena
 * buffers at offset * batch + instance * stride).  *need receives the size
 * including the terminating NUL; buf == NULL queries it.  Errors: TN_EINVAL
 * (bad arguments, cap too small), TN_ESHAPE / TN_EFORMAT (bad network or tree). */
int tn_plan_describe(const tn_network_desc* net, const tn_tree_desc* tree, int chi, int prec, int grad, int gauge_r,
                     char* buf, size_t cap, size_t* need);

/* Schedule statistics of one instance at chi (no GPU work). */
int tn_plan_stats_get(tn_ctx* ctx, int inst_id, int chi, int prec, tn_plan_stats* out);

/* Diagnostic: run the batch inst_ids[0..n_inst) exactly as tn_contract_approx
 * would (same plan, same launches) but stop after the steps of tree op
 * `stop_op` (0-based op index; -1 = before any op), then copy tensor
 * `tensor_id` of instance inst_ids[which] to host `out` (cap doubles),
 * row-major over its storage order.  *ndim_out receives its number of bonds,
 * bond_ids_out / dims_out (24 entries each, may be NULL) the bond ids and
 * sizes in storage order; bond ids >= the network's n_bonds are bonds created
 * by compressions, numbered in execution order.  out == NULL queries the
 * shape only and runs nothing.  TN_EINVAL if the tensor does not exist after
 * that op.  Intermediates carry the running power-of-two scale, so values
 * equal the exact ones up to a factor 2^e.  Consecutive calls on the same
 * batch and plan with non-decreasing stop_op (and no other work on the
 * context in between) continue from where the previous call stopped instead
 * of re-running the schedule from the start; the pass is deterministic, so
 * the tensors are the same as from a fresh run. */
int tn_debug_tensor(tn_ctx* ctx, int n_inst, const int* inst_ids, int which, int chi, int prec,
                    int stop_op, int tensor_id, double* out, int64_t cap, int32_t* ndim_out,
                    int32_t* bond_ids_out, int64_t* dims_out);

/* Time every kernel of the next tn_contract_approx with CUDA events, grouped
 * by kernel family, when enable != 0 (off by default; adds one event pair per
 * launch).  tn_kernel_times copies up to `cap` entries of (family name,
 * launches, total milliseconds) and returns the number of families. */
int tn_profile_enable(tn_ctx* ctx, int enable);
int tn_kernel_times(tn_ctx* ctx, int cap, const char** names, int64_t* launches, double* total_ms);

/* Approximate contraction of ONE instance without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- a plug-in inside a host application whose own
 * allocator has already reserved the device memory, or code on a
 * latency-critical path where cudaMalloc / cudaFree would synchronise the
 * whole device.  Every device buffer (the copied inputs, the schedule's arena,
 * the QR / Jacobi / log-norm scratch, the result words) is carved from one
 * file-scope __device__ array of 8 MiB that every GPU loading the library
 * holds until the process exits; an instance needing more is rejected with
 * TN_ENOMEM and a message giving both sizes, before any GPU work.
 *   net, tree   as for tn_load_network / tn_load_tree (host data, copied)
 *   chi         >= 1; the FP64 form is used
 *   cuda_stream the stream to run on (NULL = legacy default), on the current
 *               device; the call synchronises it before returning
 *   outputs     *logabsz_out = ln|Z|, *sign_out in {-1, 0, +1} (host)
 *   err_msg     optional host buffer (err_cap bytes) for a message
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  All calls
 * on a device share the one array (what must start at zero is cleared on
 * each call), so calls that overlap on the GPU -- on two streams or from two
 * threads -- race; serialise them.  Results equal those of tn_contract_approx
 * for a batch of one in the FP64 form with the plain Q-form compressions (no
 * tree gauge): the same schedule and the same kernels. */
int tn_contract_approx_noalloc(const tn_network_desc* net, const tn_tree_desc* tree, int chi,
                               void* cuda_stream, double* logabsz_out, int* sign_out, char* err_msg,
                               size_t err_cap);

/* Message for the last non-OK status returned on this context (never NULL). */
const char* tn_last_error(const tn_ctx* ctx);

/* Library version string. */
const char* tn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
