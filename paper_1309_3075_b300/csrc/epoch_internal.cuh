// epoch_internal.cuh -- context layout and kernel-launch interfaces shared by
// the translation units of libepoch.  Not installed; the public interface is
// include/epoch.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "epoch.h"

namespace epoch {

// Device status word bits (read back at synchronising calls).
enum : int {
  ST_NONFINITE = 1,      // a partial likelihood or scale became NaN/Inf
  ST_EIG_NOCONV = 2,     // Jacobi sweeps hit their limit
  ST_TIMEOUT = 4,        // a bounded wait ran out
  ST_SEGMENTS = 8,       // a branch produced more segments than its slots
  ST_HEIGHTS = 16,       // heights set from device memory failed the tree check
};

constexpr int kTile = 256;       // patterns per CTA in the streaming kernels

// What has been set on the context (for EPOCH_ERR_ORDER).
enum : unsigned {
  HAVE_RATES = 1u, HAVE_CATS = 2u, HAVE_TREE = 4u, HAVE_TIPS = 8u,
  HAVE_BRANCH = 16u, HAVE_PARTIALS = 32u,
  HAVE_GRADIENT = 64u  // G of the current inputs (expected counts need it)
};

// Regions of the per-step input block (epoch_ctx::d_in).
enum : int { IN_Q = 0, IN_PI, IN_BOUND, IN_CATR, IN_CATW, IN_HEIGHTS, IN_END };

// Device views handed to kernels (plain pointers and sizes).
struct Dims {
  int K;      // states
  int Kp;     // padded row length of a partial vector (multiple of 4)
  int KK;     // K*K
  int NR;     // rows of the transposed branch-matrix table: K + 1 + n_masks
  int E;      // epochs
  int S;      // rate matrices
  int C;      // categories
  int P;      // patterns
  int Pp;     // row stride of the per-pattern byte/short/float arrays (P rounded
              // up to 16: every row starts on a 16-byte boundary for bulk copies)
  int N;      // taxa of the current tree
  int nn;     // 2N-1
  int np;     // model parameters
  int reversible;
  int n_masks;
};

struct epoch_state;  // forward

}  // namespace epoch

struct epoch_ctx {
  epoch::Dims d{};
  int max_taxa = 0;
  int precision = 0;            // the path in use (EPOCH_FP32_AUTO resolved)
  int requested_precision = 0;  // as passed to epoch_create
  double probe_ms_simt = -1.0, probe_ms_tc = -1.0, probe_ms_bf = -1.0;  // EPOCH_FP32_AUTO's timings
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // side branches: work no later kernel of the pass needs runs off the main
  // stream (captured as parallel graph branches); 0: parameter transform,
  // 1: per-pattern log-sum
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork_ev[2] = {nullptr, nullptr}, join_ev[2] = {nullptr, nullptr};
  bool side_pending[2] = {false, false};
  std::string err;
  unsigned have = 0;
  int normalise = 1;

  // host copies of inputs
  std::vector<int> h_phi;             // [E]
  std::vector<int> h_parent;          // [nn]
  std::vector<int> h_child;           // [NI][2]
  std::vector<int> h_level_nodes;     // internal nodes, level-ascending
  std::vector<int> h_level_off;       // [L+1]
  std::vector<unsigned long long> h_masks;
  // host copies of the other inputs: device copies are made from these
  // (owned by the context), so a caller's array -- pinned or not -- is free
  // again when the call returns
  std::vector<double> h_brate, h_pw;
  int topo_version = 0;

  // ---- device buffers (owned) ----
  // The per-step inputs (Q, pi, boundaries, category rates and weights,
  // heights) are regions of one device block d_in with a pinned host mirror
  // h_in: a setter writes its region of the mirror and copies it up, and
  // epoch_evaluate_step copies all the regions it was given with one copy.
  // in_ev marks the last copy out of the mirror, which is written only after
  // it; the mirror equals the device block in every region except the
  // heights after epoch_set_heights_device (the last region, so a copy
  // spanning it is one that was given heights).
  double *d_in = nullptr, *h_in = nullptr;
  size_t in_off[7] = {0, 0, 0, 0, 0, 0, 0};  // region starts (IN_Q ... IN_HEIGHTS), end
  cudaEvent_t in_ev = nullptr;
  double *h_dq = nullptr;             // pinned mirror of dQ [np][S][K][K]
  // device addresses of the pinned mirrors (k_stage.cu reads and writes them)
  double *h_in_dev = nullptr, *h_dq_dev = nullptr, *h_out_dev = nullptr;
  double *d_boundaries = nullptr;     // [E-1] (at least 1), in d_in
  int *d_phi = nullptr;               // [E]
  double *d_Qraw = nullptr;           // [S][K][K], in d_in
  double *d_pi = nullptr;             // [K], in d_in
  double *d_Q = nullptr;              // [S][K][K] normalised
  double *d_cnorm = nullptr;          // [S]
  double *d_lam = nullptr;            // [S][K]
  double *d_V = nullptr;              // [S][K][K]
  double *d_Vinv = nullptr;           // [S][K][K]
  double *d_eig = nullptr;            // K > 8: eigenvector refinement scratch (k_model.cu)
  float2 *d_dfU = nullptr;            // [S][K K + 2 K] float pairs of U, sqrt(pi), 1/sqrt(pi)
  float *d_eig32 = nullptr;           // V [S][K][K], V^-1 [S][K][K], lambda [S][K] in FP32
  double *d_dQraw = nullptr;          // [np][S][K][K]
  double *d_Dth = nullptr;            // [np][S][K][K]  V^-1 dQ_eff V (FP64)
  float *d_Dth32 = nullptr;           // same in FP32
  int *d_Dnz = nullptr;               // [np][S] nonzero flags
  double *d_catr = nullptr, *d_catw = nullptr;  // [C]
  unsigned long long *d_masks = nullptr;        // [n_masks]
  double *d_heights = nullptr;        // [nn]
  int *d_parent = nullptr;            // [nn]
  double *d_brate = nullptr;          // [nn]
  int *d_child = nullptr;             // [NI][2]
  int *d_level_nodes = nullptr;       // [NI]
  // segments, fixed stride E per branch (indexed by child node)
  int *d_nseg = nullptr;              // [nn]
  int *d_seg_mat = nullptr;           // [nn][E]
  double *d_seg_dt = nullptr;         // [nn][E]
  int *d_seg_hi = nullptr;            // [nn][E]
  int *d_seg_lo = nullptr;            // [nn][E]
  // branch matrices
  double *d_P64 = nullptr;            // [nn][C][K][K]
  float *d_PT32 = nullptr;            // [nn][C][NR][Kp]  transposed + tip rows
  // partials
  void *d_part = nullptr;             // [NI][C][P][Kp]  (float or double)
  void *d_pre = nullptr;              // [NI][C][P][Kp]  pre-order partials
  void *d_xbuf = nullptr;             // generic adjoint scratch [2*maxw][C][P][Kp]
  int16_t *d_scale = nullptr;         // [NI][P] power-of-two exponents
  uint8_t *d_tips = nullptr;          // [N][P]
  double *d_pw = nullptr;             // [P]
  float *d_pwf = nullptr;             // [Pp] pattern weights as FP32 (0 in the padding)
  double *d_site_lnl = nullptr;       // [P]
  double *d_site_inv = nullptr;       // [P]  1 / scaled site value
  double *d_lnl_part = nullptr;       // [ceil(P/kTile)]
  // lnL, the status word and the gradient are one block d_out (pinned
  // mirror h_out), read back with one copy: [lnL | status | gradient]
  double *d_out = nullptr, *h_out = nullptr;
  double *d_lnl = nullptr;            // [1], d_out[0]
  void *d_Gpart = nullptr;            // [NI*nblk*2][C][K][K] (T)
  double *d_G = nullptr;              // [nn][C][K][K]
  void *d_gseg = nullptr;             // [nn][E][C][1+np]  (T)
  double *d_grad = nullptr;           // [nn (heights) + (E-1) + np + nn (rates)], d_out + 2
  double *d_jumps = nullptr;          // [nn][E][C][K][K] expected counts per segment
  double *d_jump_out = nullptr;       // [nn + E][K][K] per-branch | per-epoch sums
  double *d_anc = nullptr;            // [N-1][P][K] ancestral-state posteriors
  int *d_status = nullptr;            // [1], in d_out[1]
  int *d_ctl = nullptr;               // [8] block counters of last-block reductions
  double *d_site_log = nullptr;       // [P] log of the scaled root sum
  int *d_level_off = nullptr;         // [L+1] level offsets into d_level_nodes
  // FP32 K = 4 schedule (k_k4.cu): level 0 holds the cherries, which the
  // post-order pass recomputes instead of storing (unless level 0 is the
  // root's level); k4_first_level is the first stored post-order level
  int root = -1;
  int k4_first_level = 1;
  // walks over the narrow top levels [k4_top, L) and the adjoint launches
  // below them (k4_schedule in k_k4.cu)
  int k4_top = 0;
  int k4_top_begin = 0;               // level-order index of the first walk node
  int k4_walk_post = 0, k4_walk_pre = 0;    // steps of each walk
  int k4_slots_post = 0, k4_slots_pre = 0;  // value slots per walk thread
  std::vector<int4> h_k4_walk;        // post-order steps, then pre-order steps (4 int4 each),
                                      // then the level kernels' node descriptors (3 int4 each)
  int k4_desc_off = 0;                // int4 offset of the node descriptors in h_k4_walk
  std::vector<int> h_k4_launch;       // adjoint launches: (first node, nodes, tiles per CTA)
  std::vector<int> h_k4_nt;           // [nn] G tiles of each branch
  int4 *d_k4_walk = nullptr;
  size_t k4_walk_cap = 0;             // int4 capacity of d_k4_walk
  int *d_k4_nt = nullptr;             // [nn]
  int *d_k4_esum = nullptr;           // [P] per-pattern exponent sum of the level kernels
  float *d_tcB = nullptr;             // [nn][C][4][64*64] tensor-core operands (k_tc.cu)
  float *d_pairS = nullptr;           // [nn][C][NR*NR][4] S of each cherry per code pair
  float *d_pairL = nullptr;           // [nn][C][NR*NR][4] L of each cherry per code pair
  size_t gpart_bytes = 0;
  size_t part_elem = 0;               // sizeof(T) of partials
  int max_level_width = 0;

  // pinned host staging (views of h_out)
  double *h_grad_pinned = nullptr;
  double *h_lnl_pinned = nullptr;
  int *h_status_pinned = nullptr;
  uint8_t *h_tips_staging = nullptr;  // two halves, used in turn (see set_tip_data)
  size_t tips_staging_half = 0;        // bytes per half
  int tips_staging_cur = 0;
  cudaEvent_t tips_staging_ev[2] = {nullptr, nullptr};  // copy out of each half done

  // graph replay
  // slots: lnL, lnL + gradient (epoch_evaluate_async), partials only
  // (epoch_update_partials), gradient only (epoch_gradient)
  static constexpr int kGraphSlots = 4;
  cudaGraphExec_t graph_exec[kGraphSlots] = {nullptr, nullptr, nullptr, nullptr};
  int graph_topo[kGraphSlots] = {-1, -1, -1, -1};
  long long graph_kernels[kGraphSlots] = {0, 0, 0, 0};
  long long launches = 0;
  long long captures = 0;
  bool capturing = false;
};

namespace epoch {

// ---- kernel launch wrappers (each returns cudaGetLastError()) ----
// k_model.cu
// k_stage.cu: n0 doubles src0 -> dst0 and n1 doubles src1 -> dst1 (n1 may
// be 0) by a kernel on the stream; pinned host memory by its device address
cudaError_t launch_stage(const double *src0, double *dst0, size_t n0, const double *src1,
                         double *dst1, size_t n1, cudaStream_t stream);
cudaError_t launch_segments(epoch_ctx *c);
cudaError_t launch_model_setup(epoch_ctx *c);
size_t eig_scratch_doubles(int K, int S);  // eigenvector refinement scratch (K > 8)
cudaError_t launch_param_transform(epoch_ctx *c);
cudaError_t launch_branch_matrices(epoch_ctx *c);
cudaError_t launch_check_heights(epoch_ctx *c);  // device-side check of d_heights
// k_partials.cu
cudaError_t launch_partials(epoch_ctx *c);
cudaError_t launch_root(epoch_ctx *c);
// k_adjoint.cu
cudaError_t launch_adjoint(epoch_ctx *c);
cudaError_t launch_chain_rule(epoch_ctx *c);
cudaError_t launch_expected_counts(epoch_ctx *c, double *d_per_branch, double *d_per_epoch);
// k_ancestral.cu
cudaError_t launch_ancestral(epoch_ctx *c, double *d_out);  // [N-1][P][K]
// k_k4.cu (FP32, K = 4)
int k4_tiles(int P);                            // pattern tiles of the K = 4 kernels
int resolve_auto(int K, int E, int C, int P, int max_taxa, cudaStream_t stream, double *ms_simt,
                 double *ms_tc, double *ms_bf);  // EPOCH_FP32_AUTO (autotune.cu)
cudaError_t launch_pair_tables_k4(epoch_ctx *c); // cherries' code-pair tables
cudaError_t launch_partials_k4(epoch_ctx *c);   // pruning, rescaling, root log-sum
cudaError_t launch_preorder_k4(epoch_ctx *c);   // adjoint pass and G
void k4_schedule(epoch_ctx *c);                 // host: walks, launches, tile counts
// k_k4small.cu (FP32, K = 4, reversible): per-(branch, category) threads
cudaError_t launch_branch_k4(epoch_ctx *c);     // segments + branch matrices + tables
cudaError_t launch_chain_k4(epoch_ctx *c);      // chain rule through the products
size_t k4_chain_smem(const Dims &d);            // its shared memory (model tables)

// k_tc.cu (FP32_TC, 4 < K <= 64): tcgen05 tile products
bool tc_path(const epoch_ctx *c);
// the tensor-core precisions (TF32 x 3 or BF16 x 3 tile products)
inline bool is_tc_precision(int p) { return p == EPOCH_FP32_TC || p == EPOCH_FP32_TC_BF16; }
cudaError_t launch_tc_prep(epoch_ctx *c);          // P and P^T as TF32 hi/lo operands
cudaError_t launch_tc_pre_u(epoch_ctx *c, int level);  // U = P^T X of one level
cudaError_t launch_tc_post(epoch_ctx *c, int level);   // pruning + rescaling of one level
cudaError_t launch_tc_pre_x(epoch_ctx *c, int level, int root);  // X of one level
size_t tc_operand_floats(const epoch_ctx *c);

// FP32, K = 4, at most 8 categories and 3 ambiguity masks (NR <= 8)
inline bool fast_k4(const epoch_ctx *c) {
  return c->precision != EPOCH_FP64 && c->d.K == 4 && c->d.C <= 8 && c->d.NR <= 8;
}

// Few patterns (discrete traits): one CTA per pattern walks the whole tree
// in one launch per pass (k_small.cu) instead of one launch per level.  A
// node's values over (category, state) must fit one warp.
// The kernels keep the pattern's tree in shared memory: topology, tip codes,
// exponents, and the partials (post-order, plus outside partials in the
// adjoint kernel) of every internal node, elements of es bytes.
constexpr int kSmallMaxPatterns = 64;
constexpr size_t kSmallMaxSmem = 200 * 1024;
inline size_t small_smem_bytes(const Dims &d, int N, size_t es, bool with_pre,
                               bool tables = false) {
  const size_t nv = (size_t)(N - 1) * d.C * d.Kp;
  const size_t nt = tables ? (size_t)(N - 1) * d.C * d.KK + (size_t)N * d.C * d.K : 0;
  return es * (nv * (with_pre ? 2 : 1) + nt) + sizeof(int) * 5 * N + N;
}
inline bool small_path(const epoch_ctx *c) {
  const size_t es = c->precision == EPOCH_FP64 ? sizeof(double) : sizeof(float);
  return !fast_k4(c) && c->d.P <= kSmallMaxPatterns && c->d.C * c->d.Kp <= 32 &&
         small_smem_bytes(c->d, c->max_taxa, es, true) <= kSmallMaxSmem;
}
// k_small.cu
cudaError_t launch_small_post(epoch_ctx *c);  // pruning, rescaling, root, lnL
cudaError_t launch_small_pre(epoch_ctx *c);   // adjoint pass; G terms per pattern

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// A sum of floats carried as a float and its running rounding error (each
// addition by Knuth's two-sum, exact): about as accurate as adding in FP64,
// on the FP32 pipes (FP64 instructions run at a small fraction of their
// rate on this part).  value() is the sum in FP64.
struct CSum {
  float s = 0.f, e = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
    s = t;
  }
  __device__ __forceinline__ void merge(const CSum &o) {
    add(o.s);
    e = __fadd_rn(e, o.e);
  }
  __device__ __forceinline__ CSum shfl_xor(int lane_mask) const {
    CSum o;
    o.s = __shfl_xor_sync(0xffffffffu, s, lane_mask);
    o.e = __shfl_xor_sync(0xffffffffu, e, lane_mask);
    return o;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};

// Programmatic dependent launch: a level kernel is launched while its
// predecessor finishes; it reads only data of launches before the predecessor
// (tables, topology) until pdl_wait() returns, which is when the predecessor
// has completed and its writes are visible.  pdl_trigger() lets the next
// level be scheduled as soon as every CTA of this one has passed its wait.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }

// Launch with programmatic stream serialisation (see pdl_wait).
template <typename Kern, typename... Args>
cudaError_t launch_pdl(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Enqueue `launch` (which launches on c->stream) on side stream s after all
// work queued so far on the main stream; join_side makes the main stream wait
// for it.  Every fork is joined before a capture ends or a call returns.
template <class F>
cudaError_t fork_side(epoch_ctx *c, int s, F launch) {
  if (!c->side[s]) return launch();
  cudaError_t e = cudaEventRecord(c->fork_ev[s], c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side[s], c->fork_ev[s], 0);
  if (e != cudaSuccess) return e;
  cudaStream_t keep = c->stream;
  c->stream = c->side[s];
  e = launch();
  c->stream = keep;
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(c->join_ev[s], c->side[s]);
  c->side_pending[s] = (e == cudaSuccess);
  return e;
}
inline cudaError_t join_side(epoch_ctx *c, int s) {
  if (!c->side_pending[s]) return cudaSuccess;
  c->side_pending[s] = false;
  return cudaStreamWaitEvent(c->stream, c->join_ev[s], 0);
}
inline cudaError_t join_sides(epoch_ctx *c) {
  cudaError_t e = join_side(c, 0);
  cudaError_t e2 = join_side(c, 1);
  return e != cudaSuccess ? e : e2;
}

}  // namespace epoch
