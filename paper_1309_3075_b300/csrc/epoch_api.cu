// epoch_api.cu -- the C ABI of include/epoch.h: argument validation, the
// post-order level schedule, device allocation, call ordering, and the
// replay of the whole path from a captured CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "epoch_internal.cuh"

using namespace epoch;

namespace {

epoch_status fail(epoch_ctx *c, epoch_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

epoch_status cuda_fail(epoch_ctx *c, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, EPOCH_ERR_CUDA, m);
}

#define CK(call, what)                        \
  do {                                        \
    cudaError_t _e = (call);                  \
    if (_e != cudaSuccess) return cuda_fail(c, _e, what); \
  } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void **)p, n * sizeof(T));
}

void dfree(void *p) {
  if (p) cudaFree(p);
}

bool fin(double x) { return std::isfinite(x); }

// Check that every kernel of the path is available on this device (a build
// for another architecture would otherwise fail at the first launch).
epoch_status check_device(epoch_ctx *c) {
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
  (void)prop;
  return EPOCH_OK;
}

size_t elem_size(int precision) { return precision == EPOCH_FP64 ? sizeof(double) : sizeof(float); }

bool generic_path(const epoch_ctx *c) { return !fast_k4(c); }

epoch_status ensure_pt32(epoch_ctx *c) {
  const Dims &d = c->d;
  dfree(c->d_PT32);
  c->d_PT32 = nullptr;
  if (c->precision == EPOCH_FP64) return EPOCH_OK;
  size_t n = (size_t)(2 * c->max_taxa - 1) * d.C * d.NR * d.Kp;
  CK(dalloc(&c->d_PT32, n), "cudaMalloc(branch tables)");
  CK(cudaMemsetAsync(c->d_PT32, 0, n * sizeof(float), c->stream), "cudaMemset");
  dfree(c->d_pairS);
  dfree(c->d_pairL);
  c->d_pairS = c->d_pairL = nullptr;
  dfree(c->d_tcB);
  c->d_tcB = nullptr;
  if (tc_path(c)) CK(dalloc(&c->d_tcB, tc_operand_floats(c)), "cudaMalloc(tensor-core operands)");
  if (fast_k4(c)) {  // code-pair tables of the cherries
    const size_t np = (size_t)(2 * c->max_taxa - 1) * d.C * d.NR * d.NR * 4;
    CK(dalloc(&c->d_pairS, np), "cudaMalloc(pair tables)");
    CK(dalloc(&c->d_pairL, np), "cudaMalloc(pair tables)");
  }
  return EPOCH_OK;
}

epoch_status ensure_param_buffers(epoch_ctx *c) {
  const Dims &d = c->d;
  const int nn_max = 2 * c->max_taxa - 1;
  dfree(c->d_gseg);
  c->d_gseg = nullptr;
  size_t ng = (size_t)nn_max * d.E * d.C * (1 + d.np);
  if (c->precision == EPOCH_FP64)
    CK(dalloc((double **)&c->d_gseg, ng), "cudaMalloc(gseg)");
  else
    CK(dalloc((float **)&c->d_gseg, ng), "cudaMalloc(gseg)");
  // [lnL | status word | gradient]; the lnL and a pending status word carry
  // over when the block grows
  const size_t nout = 2 + (size_t)2 * nn_max + (d.E - 1) + d.np;
  double *out = nullptr, *h = nullptr;
  CK(dalloc(&out, nout), "cudaMalloc(results)");
  if (cudaMallocHost((void **)&h, nout * sizeof(double)) != cudaSuccess) {
    dfree(out);
    return fail(c, EPOCH_ERR_CUDA, "cudaMallocHost(results)");
  }
  if (c->d_out) {
    CK(cudaMemcpyAsync(out, c->d_out, 2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream),
       "cudaMemcpyAsync(results)");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    dfree(c->d_out);
    cudaFreeHost(c->h_out);
  } else {
    CK(cudaMemsetAsync(out, 0, 2 * sizeof(double), c->stream), "cudaMemset(results)");
  }
  CK(cudaHostGetDevicePointer((void **)&c->h_out_dev, h, 0), "cudaHostGetDevicePointer(results)");
  c->d_out = out;
  c->h_out = h;
  c->d_lnl = out;
  c->d_status = reinterpret_cast<int *>(out + 1);
  c->d_grad = out + 2;
  c->h_lnl_pinned = h;
  c->h_status_pinned = reinterpret_cast<int *>(h + 1);
  c->h_grad_pinned = h + 2;
  return EPOCH_OK;
}

void invalidate_graphs(epoch_ctx *c) {
  for (int g = 0; g < epoch_ctx::kGraphSlots; g++) {
    if (c->graph_exec[g]) cudaGraphExecDestroy(c->graph_exec[g]);
    c->graph_exec[g] = nullptr;
    c->graph_topo[g] = -1;
  }
}

// Copies the first n doubles of the result block (lnL, the status word, then
// the gradient) to its pinned mirror, waits, and turns the status word into
// the call's status.
static epoch_status read_results_head(epoch_ctx *c, size_t n) {
  CK(launch_stage(c->d_out, c->h_out_dev, n, nullptr, nullptr, 0, c->stream), "k_stage(results)");
  c->launches++;
  CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  int st = *c->h_status_pinned;
  if (st == 0) return EPOCH_OK;
  CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "cudaMemset(status)");
  if (st & ST_TIMEOUT) return fail(c, EPOCH_ERR_TIMEOUT, "a bounded device wait ran out");
  if (st & ST_HEIGHTS)  // first: bad heights also make everything after them non-finite
    return fail(c, EPOCH_ERR_ARG, "heights set from device memory: non-finite or a parent "
                                  "below its child");
  if (st & ST_EIG_NOCONV)
    return fail(c, EPOCH_ERR_NUMERIC, "Jacobi eigensolver did not converge");
  if (st & ST_NONFINITE)
    return fail(c, EPOCH_ERR_NUMERIC, "non-finite partial likelihood (check rates and heights)");
  if (st & ST_SEGMENTS) return fail(c, EPOCH_ERR_NUMERIC, "segment overflow");
  return fail(c, EPOCH_ERR_NUMERIC, "device status word set");
}

epoch_status read_status(epoch_ctx *c) { return read_results_head(c, 2); }

// ---- the enqueued sequences ---------------------------------------------

epoch_status enqueue_branch(epoch_ctx *c) {
  if (fast_k4(c) && c->d.reversible) {
    CK(launch_model_setup(c), "model setup kernel");
    CK(fork_side(c, 0, [&] { return launch_param_transform(c); }), "parameter transform kernel");
    CK(launch_branch_k4(c), "branch matrix kernel");
  } else {
    CK(launch_segments(c), "segments kernel");
    CK(launch_model_setup(c), "model setup kernel");
    CK(fork_side(c, 0, [&] { return launch_param_transform(c); }), "parameter transform kernel");
    CK(launch_branch_matrices(c), "branch matrix kernel");
  }
  if (fast_k4(c)) CK(launch_pair_tables_k4(c), "pair table kernel");
  if (tc_path(c)) CK(launch_tc_prep(c), "tensor-core operand kernel");
  return EPOCH_OK;
}

epoch_status enqueue_partials(epoch_ctx *c) {
  CK(launch_partials(c), "partials kernels");
  CK(launch_root(c), "root kernel");
  return EPOCH_OK;
}

epoch_status enqueue_gradient(epoch_ctx *c) {
  CK(launch_adjoint(c), "adjoint kernels");
  CK(launch_chain_rule(c), "chain-rule kernels");
  return EPOCH_OK;
}

epoch_status need(epoch_ctx *c, unsigned bits, const char *what) {
  if ((c->have & bits) != bits)
    return fail(c, EPOCH_ERR_ORDER, std::string(what) + ": required inputs not set yet");
  return EPOCH_OK;
}

// Replays the captured graph of slot g (0: branch matrices + partials,
// 1: the same + gradient, 2: partials only, 3: gradient only), capturing it
// first when there is none for the current topology.  enqueue() puts the slot's work on the
// stream; every side branch rejoins before the capture ends.
template <class F>
epoch_status replay(epoch_ctx *c, int g, F enqueue) {
  if (!c->graph_exec[g] || c->graph_topo[g] != c->topo_version) {
    if (c->graph_exec[g]) cudaGraphExecDestroy(c->graph_exec[g]);
    c->graph_exec[g] = nullptr;
    cudaGraph_t graph;
    const long long before = c->launches;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
    c->capturing = true;
    epoch_status es = enqueue();
    cudaError_t je = join_sides(c);
    if (es == EPOCH_OK && je != cudaSuccess) es = cuda_fail(c, je, "join");
    cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
    c->capturing = false;
    if (es != EPOCH_OK) {
      if (ee == cudaSuccess) cudaGraphDestroy(graph);
      return es;
    }
    CK(ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&c->graph_exec[g], graph, 0);
    cudaGraphDestroy(graph);
    CK(ie, "cudaGraphInstantiate");
    c->graph_kernels[g] = c->launches - before;
    c->launches = before;
    c->graph_topo[g] = c->topo_version;
    c->captures++;
  }
  CK(cudaGraphLaunch(c->graph_exec[g], c->stream), "cudaGraphLaunch");
  c->launches += c->graph_kernels[g];
  return EPOCH_OK;
}


epoch_status copy_grad_out(epoch_ctx *c, double *d_heights, double *d_boundaries,
                           double *d_params, double *d_branch_rates) {
  const Dims &d = c->d;
  const size_t nout = (size_t)2 * d.nn + (d.E - 1) + d.np;
  // the gradient's layout is [heights nn | boundaries E-1 | params np | rates nn]
  epoch_status s = read_results_head(c, 2 + nout);
  if (s != EPOCH_OK) return s;
  const double *g = c->h_grad_pinned;
  if (d_heights) memcpy(d_heights, g, sizeof(double) * d.nn);
  if (d_boundaries && d.E > 1) memcpy(d_boundaries, g + d.nn, sizeof(double) * (d.E - 1));
  if (d_params && d.np > 0) memcpy(d_params, g + d.nn + d.E - 1, sizeof(double) * d.np);
  if (d_branch_rates) memcpy(d_branch_rates, g + d.nn + d.E - 1 + d.np, sizeof(double) * d.nn);
  return EPOCH_OK;
}

// Topology and height checks for a binary tree with tips 0..N-1.  Fills the
// root, the child pairs of internal nodes [N-1][2] and, when asked, the
// post-order level of every node (tips 0, internal 1 + max of children).
epoch_status check_tree(int N, const double *heights, const int *parent, const double *rates,
                        int *root_out, std::vector<int> *child_out, std::vector<int> *level_out,
                        std::string *msg) {
  if (N < 2) {
    *msg = "need at least 2 taxa";
    return EPOCH_ERR_ARG;
  }
  const int nn = 2 * N - 1;
  std::vector<int> nchild(nn, 0), child(2 * (N - 1), -1);
  int root = -1;
  for (int v = 0; v < nn; v++) {
    const int u = parent[v];
    if (u == -1) {
      if (root >= 0) {
        *msg = "more than one root";
        return EPOCH_ERR_ARG;
      }
      root = v;
      continue;
    }
    if (u < N || u >= nn) {
      *msg = "parent index out of range (tips are 0..N-1, internal N..2N-2)";
      return EPOCH_ERR_ARG;
    }
    if (nchild[u] >= 2) {
      *msg = "tree is not binary";
      return EPOCH_ERR_ARG;
    }
    child[2 * (u - N) + nchild[u]] = v;
    nchild[u]++;
  }
  if (root < N) {
    *msg = "no root, or the root is a tip";
    return EPOCH_ERR_ARG;
  }
  for (int u = N; u < nn; u++)
    if (nchild[u] != 2) {
      *msg = "an internal node without two children";
      return EPOCH_ERR_ARG;
    }
  // post-order from the root; a cycle leaves nodes unvisited
  std::vector<int> level(nn, 0), stack{root};
  std::vector<char> state(nn, 0);
  int visited = 0;
  while (!stack.empty()) {
    const int u = stack.back();
    if (u < N) {
      stack.pop_back();
      if (state[u]) break;
      state[u] = 2;
      visited++;
      continue;
    }
    if (state[u] == 0) {
      state[u] = 1;
      stack.push_back(child[2 * (u - N)]);
      stack.push_back(child[2 * (u - N) + 1]);
      if ((int)stack.size() > 2 * nn) break;
    } else {
      stack.pop_back();
      if (state[u] == 2) break;
      state[u] = 2;
      visited++;
      level[u] = 1 + std::max(level[child[2 * (u - N)]], level[child[2 * (u - N) + 1]]);
    }
  }
  if (visited != nn) {
    *msg = "parent array does not describe one tree";
    return EPOCH_ERR_ARG;
  }
  for (int v = 0; v < nn; v++) {
    if (!fin(heights[v])) {
      *msg = "non-finite height";
      return EPOCH_ERR_ARG;
    }
    const int u = parent[v];
    if (u >= 0 && !(heights[u] >= heights[v])) {
      *msg = "a parent is younger than its child";
      return EPOCH_ERR_ARG;
    }
    if (rates && (!fin(rates[v]) || rates[v] < 0.0)) {
      *msg = "bad branch rate";
      return EPOCH_ERR_ARG;
    }
  }
  if (root_out) *root_out = root;
  if (child_out) *child_out = child;
  if (level_out) *level_out = level;
  return EPOCH_OK;
}

// FP32 K = 4 schedule (see k_k4.cu): level 0 holds the cherries (both
// children tips); the post-order pass recomputes them from code-pair tables
// instead of storing them, unless level 0 is the root's own level (two
// taxa).  G tile sums are [nn][tiles][C][16]; code-pair tables are
// [nn][C][NR^2] float4 each.
epoch_status plan_k4(epoch_ctx *c) {
  const Dims &d = c->d;
  const int L = (int)c->h_level_off.size() - 1;
  c->k4_first_level = (L == 1) ? 0 : 1;
  const size_t nn_max = (size_t)(2 * c->max_taxa - 1);
  const size_t need = nn_max * k4_tiles(d.P) * d.C * 16 * sizeof(float);
  if (c->gpart_bytes < need) {
    dfree(c->d_Gpart);
    c->d_Gpart = nullptr;
    c->gpart_bytes = need;
    CK(cudaMalloc(&c->d_Gpart, c->gpart_bytes), "cudaMalloc(G tile sums)");
  }
  // exponents of cherries are never written: they stay zero
  CK(cudaMemsetAsync(c->d_scale, 0, (size_t)(d.N - 1) * d.Pp * sizeof(int16_t), c->stream),
     "cudaMemset(scale)");
  k4_schedule(c);
  if (c->k4_walk_cap < c->h_k4_walk.size()) {
    dfree(c->d_k4_walk);
    c->d_k4_walk = nullptr;
    c->k4_walk_cap = c->h_k4_walk.size();
    CK(cudaMalloc(&c->d_k4_walk, sizeof(int4) * c->k4_walk_cap), "cudaMalloc(walk steps)");
  }
  if (!c->d_k4_nt) CK(dalloc(&c->d_k4_nt, nn_max), "cudaMalloc(G tile counts)");
  if (!c->d_k4_esum) CK(dalloc(&c->d_k4_esum, d.P), "cudaMalloc(exponent sums)");
  // the partials pass leaves both zero for the next one
  CK(cudaMemsetAsync(c->d_k4_esum, 0, sizeof(int) * d.P, c->stream), "cudaMemset(exponent sums)");
  CK(cudaMemsetAsync(c->d_ctl, 0, sizeof(int), c->stream), "cudaMemset(counter)");
  if (!c->h_k4_walk.empty())
    CK(cudaMemcpyAsync(c->d_k4_walk, c->h_k4_walk.data(), sizeof(int4) * c->h_k4_walk.size(),
                       cudaMemcpyHostToDevice, c->stream),
       "cudaMemcpyAsync(walk steps)");
  CK(cudaMemcpyAsync(c->d_k4_nt, c->h_k4_nt.data(), sizeof(int) * d.nn, cudaMemcpyHostToDevice,
                     c->stream),
     "cudaMemcpyAsync(G tile counts)");
  return EPOCH_OK;
}

}  // namespace

// =========================================================================
extern "C" {

epoch_status epoch_check_tree(int n_taxa, const double *heights, const int *parent,
                              const double *branch_rates, int *n_levels) {
  if (!heights || !parent) return EPOCH_ERR_ARG;
  std::vector<int> level;
  int root = -1;
  std::string msg;
  epoch_status s = check_tree(n_taxa, heights, parent, branch_rates, &root, nullptr, &level, &msg);
  if (s == EPOCH_OK && n_levels) *n_levels = level[root];
  return s;
}

const char *epoch_status_string(epoch_status s) {
  switch (s) {
    case EPOCH_OK: return "ok";
    case EPOCH_ERR_ARG: return "invalid argument";
    case EPOCH_ERR_ORDER: return "call out of order";
    case EPOCH_ERR_CAPACITY: return "capacity exceeded";
    case EPOCH_ERR_NUMERIC: return "numerical error";
    case EPOCH_ERR_CUDA: return "CUDA error";
    case EPOCH_ERR_TIMEOUT: return "device wait timed out";
    case EPOCH_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *epoch_last_error(const epoch_ctx *c) { return c ? c->err.c_str() : "null context"; }

epoch_status epoch_path_info(const epoch_ctx *c, int *precision_in_use, double *probe_ms_simt,
                             double *probe_ms_tc, double *probe_ms_tc_bf16) {
  if (!c) return EPOCH_ERR_ARG;
  if (precision_in_use) *precision_in_use = c->precision;
  if (probe_ms_simt) *probe_ms_simt = c->probe_ms_simt;
  if (probe_ms_tc) *probe_ms_tc = c->probe_ms_tc;
  if (probe_ms_tc_bf16) *probe_ms_tc_bf16 = c->probe_ms_bf;
  return EPOCH_OK;
}

epoch_status epoch_counters(const epoch_ctx *c, long long *kernel_launches,
                            long long *graph_captures) {
  if (!c) return EPOCH_ERR_ARG;
  if (kernel_launches) *kernel_launches = c->launches;
  if (graph_captures) *graph_captures = c->captures;
  return EPOCH_OK;
}

void epoch_destroy(epoch_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  invalidate_graphs(c);
  void *bufs[] = {c->d_in,         c->d_phi,     c->d_Q,
                  c->d_cnorm,      c->d_lam,     c->d_V,        c->d_Vinv,       c->d_dQraw,
                  c->d_Dth,        c->d_Dth32,   c->d_Dnz,
                  c->d_masks,      c->d_parent,   c->d_brate,      c->d_child,
                  c->d_level_nodes, c->d_nseg,   c->d_seg_mat,  c->d_seg_dt,     c->d_seg_hi,
                  c->d_seg_lo,     c->d_P64,     c->d_PT32,     c->d_part,       c->d_pre,
                  c->d_xbuf,       c->d_scale,   c->d_tips,     c->d_pw,         c->d_pwf,
                  c->d_site_lnl,
                  c->d_site_inv,   c->d_lnl_part, c->d_out,     c->d_Gpart,      c->d_G,
                  c->d_gseg,       c->d_ctl,        c->d_site_log,
                  c->d_level_off,  c->d_pairS,   c->d_pairL,    c->d_k4_walk,    c->d_k4_nt,
                  c->d_k4_esum,    c->d_tcB,     c->d_jumps,    c->d_jump_out,   c->d_anc,
                  c->d_eig,        c->d_dfU,     c->d_eig32};
  for (void *p : bufs) dfree(p);
  if (c->h_out) cudaFreeHost(c->h_out);
  if (c->h_in) cudaFreeHost(c->h_in);
  if (c->h_dq) cudaFreeHost(c->h_dq);
  if (c->in_ev) cudaEventDestroy(c->in_ev);
  if (c->h_tips_staging) cudaFreeHost(c->h_tips_staging);
  for (cudaEvent_t e : c->tips_staging_ev)
    if (e) cudaEventDestroy(e);
  for (int k = 0; k < 2; k++) {
    if (c->side[k]) cudaStreamSynchronize(c->side[k]);
    if (c->side[k]) cudaStreamDestroy(c->side[k]);
    if (c->fork_ev[k]) cudaEventDestroy(c->fork_ev[k]);
    if (c->join_ev[k]) cudaEventDestroy(c->join_ev[k]);
  }
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

epoch_status epoch_create(epoch_ctx **out, int states, int n_epochs, const double *boundaries,
                          const int *epoch_to_matrix, int n_matrices, int max_taxa,
                          int n_patterns, int n_categories, int precision, void *cuda_stream) {
  if (!out) return EPOCH_ERR_ARG;
  *out = nullptr;
  if (states < 2 || states > EPOCH_MAX_STATES) return EPOCH_ERR_ARG;
  if (n_epochs < 1 || n_epochs > EPOCH_MAX_EPOCHS) return EPOCH_ERR_ARG;
  if (n_matrices < 1) return EPOCH_ERR_ARG;
  if (max_taxa < 2 || max_taxa > 65535) return EPOCH_ERR_ARG;
  if (n_patterns < 1) return EPOCH_ERR_ARG;
  if (n_categories < 1 || n_categories > EPOCH_MAX_CATEGORIES) return EPOCH_ERR_ARG;
  if (precision < EPOCH_FP64 || precision > EPOCH_FP32_TC_BF16) return EPOCH_ERR_ARG;
  if (n_epochs > 1) {
    if (!boundaries) return EPOCH_ERR_ARG;
    for (int j = 0; j < n_epochs - 1; j++) {
      if (!fin(boundaries[j])) return EPOCH_ERR_ARG;
      if (j > 0 && !(boundaries[j] > boundaries[j - 1])) return EPOCH_ERR_ARG;
    }
  }
  std::vector<int> phi(n_epochs);
  for (int e = 0; e < n_epochs; e++) {
    phi[e] = epoch_to_matrix ? epoch_to_matrix[e] : e;
    if (phi[e] < 0 || phi[e] >= n_matrices) return EPOCH_ERR_ARG;
  }
  if (!epoch_to_matrix && n_matrices != n_epochs) return EPOCH_ERR_ARG;

  // EPOCH_FP32_AUTO: the faster FP32 path for this shape, timed once per
  // process (autotune.cu)
  double probe_simt = -1.0, probe_tc = -1.0, probe_bf = -1.0;
  const int requested = precision;
  if (precision == EPOCH_FP32_AUTO)
    precision = resolve_auto(states, n_epochs, n_categories, n_patterns, max_taxa,
                             (cudaStream_t)cuda_stream, &probe_simt, &probe_tc, &probe_bf);

  epoch_ctx *c = new (std::nothrow) epoch_ctx();
  if (!c) return EPOCH_ERR_CAPACITY;
  c->requested_precision = requested;
  c->probe_ms_simt = probe_simt;
  c->probe_ms_tc = probe_tc;
  c->probe_ms_bf = probe_bf;
  Dims &d = c->d;
  d.K = states;
  d.Kp = (states + 3) / 4 * 4;
  // the tensor-core tiles are 64, 32 or 16 states wide: pad to the tile width
  if (is_tc_precision(precision) && states > 32) d.Kp = 64;
  if (is_tc_precision(precision) && states > 16 && states <= 32) d.Kp = 32;
  if (is_tc_precision(precision) && states > 8 && states <= 16) d.Kp = 16;
  d.KK = states * states;
  d.n_masks = 0;
  d.NR = states + 1;
  d.E = n_epochs;
  d.S = n_matrices;
  d.C = n_categories;
  d.P = n_patterns;
  d.Pp = (n_patterns + 15) / 16 * 16;
  d.N = 0;
  d.nn = 0;
  d.np = 0;
  d.reversible = 1;
  c->max_taxa = max_taxa;
  c->precision = precision;
  c->h_phi = phi;

  epoch_status st = check_device(c);
  if (st != EPOCH_OK) {
    epoch_destroy(c);
    return st;
  }
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      epoch_destroy(c);
      return EPOCH_ERR_CUDA;
    }
    c->own_stream = true;
  }
  for (int k = 0; k < 2; k++) {
    if (cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev[k], cudaEventDisableTiming) != cudaSuccess) {
      epoch_destroy(c);
      return EPOCH_ERR_CUDA;
    }
  }

  const int nn_max = 2 * max_taxa - 1, ni_max = max_taxa - 1;
  const size_t es = elem_size(precision);
  const size_t P = (size_t)n_patterns, C = n_categories, KK = d.KK;
  const int nchunk = ceil_div(n_patterns, kTile);
  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  A(dalloc(&c->d_phi, n_epochs));
  {  // the per-step inputs: one device block, one pinned mirror
    size_t *o = c->in_off;
    o[IN_Q] = 0;                                       // Q [S][K][K]
    o[IN_PI] = o[IN_Q] + (size_t)d.S * KK;             // pi [K]
    o[IN_BOUND] = o[IN_PI] + d.K;                      // boundaries [E-1]
    o[IN_CATR] = o[IN_BOUND] + std::max(1, n_epochs - 1);  // category rates [C]
    o[IN_CATW] = o[IN_CATR] + C;                       // category weights [C]
    o[IN_HEIGHTS] = o[IN_CATW] + C;                    // heights [nn_max]
    o[IN_END] = o[IN_HEIGHTS] + nn_max;
    A(dalloc(&c->d_in, o[IN_END]));
    A(cudaMallocHost((void **)&c->h_in, sizeof(double) * o[IN_END]));
    A(cudaEventCreateWithFlags(&c->in_ev, cudaEventDisableTiming));
    if (ok) A(cudaHostGetDevicePointer((void **)&c->h_in_dev, c->h_in, 0));
    if (ok) {
      memset(c->h_in, 0, sizeof(double) * o[IN_END]);
      c->d_Qraw = c->d_in + o[IN_Q];
      c->d_pi = c->d_in + o[IN_PI];
      c->d_boundaries = c->d_in + o[IN_BOUND];
      c->d_catr = c->d_in + o[IN_CATR];
      c->d_catw = c->d_in + o[IN_CATW];
      c->d_heights = c->d_in + o[IN_HEIGHTS];
    }
  }
  A(dalloc(&c->d_Q, (size_t)d.S * KK));
  A(dalloc(&c->d_cnorm, d.S));
  A(dalloc(&c->d_lam, (size_t)d.S * d.K));
  A(dalloc(&c->d_V, (size_t)d.S * KK));
  A(cudaMalloc(&c->d_dfU, sizeof(float2) * (size_t)d.S * (KK + 2 * d.K)));
  A(cudaMalloc(&c->d_eig32, sizeof(float) * (size_t)d.S * (2 * KK + d.K)));
  A(dalloc(&c->d_Vinv, (size_t)d.S * KK));
  if (d.K > 8) A(dalloc(&c->d_eig, eig_scratch_doubles(d.K, d.S)));  // eigenvector refinement
  A(dalloc(&c->d_parent, nn_max));
  A(dalloc(&c->d_brate, nn_max));
  A(dalloc(&c->d_child, 2 * ni_max));
  A(dalloc(&c->d_level_nodes, ni_max));
  A(dalloc(&c->d_nseg, nn_max));
  A(dalloc(&c->d_seg_mat, (size_t)nn_max * d.E));
  A(dalloc(&c->d_seg_dt, (size_t)nn_max * d.E));
  A(dalloc(&c->d_seg_hi, (size_t)nn_max * d.E));
  A(dalloc(&c->d_seg_lo, (size_t)nn_max * d.E));
  A(dalloc(&c->d_P64, (size_t)nn_max * C * KK));
  A(cudaMalloc(&c->d_part, (size_t)ni_max * C * P * d.Kp * es));
  A(cudaMalloc(&c->d_pre, (size_t)ni_max * C * P * d.Kp * es));
  A(dalloc(&c->d_scale, (size_t)ni_max * d.Pp));
  A(dalloc(&c->d_tips, (size_t)max_taxa * d.Pp));
  A(dalloc(&c->d_pw, P));
  A(dalloc(&c->d_pwf, d.Pp));
  A(dalloc(&c->d_site_lnl, P));
  A(dalloc(&c->d_site_inv, P));
  A(dalloc(&c->d_lnl_part, ceil_div(n_patterns, 16)));  // one per block of >= 16 patterns
  if (precision == EPOCH_FP64 || states != 4 || n_categories > 8) {  // K = 4 FP32: per tree
    // G terms per pattern on the few-pattern path, else per tile of kTile
    const size_t nG = small_path(c) ? P : (size_t)nchunk;
    c->gpart_bytes = (size_t)ni_max * nG * 2 * C * KK * es;
    A(cudaMalloc(&c->d_Gpart, c->gpart_bytes));
  }
  A(dalloc(&c->d_G, (size_t)nn_max * C * KK));
  A(dalloc(&c->d_ctl, 8));
  A(dalloc(&c->d_level_off, max_taxa + 1));
  A(dalloc(&c->d_site_log, P));
  c->tips_staging_half = ((size_t)max_taxa * d.Pp + sizeof(float) * d.Pp + 255) & ~(size_t)255;
  A(cudaMallocHost((void **)&c->h_tips_staging, 2 * c->tips_staging_half));
  A(cudaEventCreateWithFlags(&c->tips_staging_ev[0], cudaEventDisableTiming));
  A(cudaEventCreateWithFlags(&c->tips_staging_ev[1], cudaEventDisableTiming));
  if (!ok) {
    cudaGetLastError();
    c->err = "device allocation failed";
    epoch_destroy(c);
    return EPOCH_ERR_CAPACITY;
  }
  // zero the partials once: padding lanes (state >= K) must stay zero
  A(cudaMemsetAsync(c->d_part, 0, (size_t)ni_max * C * P * d.Kp * es, c->stream));
  A(cudaMemsetAsync(c->d_pre, 0, (size_t)ni_max * C * P * d.Kp * es, c->stream));
  A(cudaMemsetAsync(c->d_P64, 0, (size_t)nn_max * C * KK * sizeof(double), c->stream));
  if (n_epochs > 1)
    memcpy(c->h_in + c->in_off[IN_BOUND], boundaries, sizeof(double) * (n_epochs - 1));
  A(launch_stage(c->h_in_dev, c->d_in, c->in_off[IN_END], nullptr, nullptr, 0, c->stream));
  A(cudaEventRecord(c->in_ev, c->stream));
  A(cudaMemcpyAsync(c->d_phi, phi.data(), sizeof(int) * n_epochs, cudaMemcpyHostToDevice,
                    c->stream));
  if (!ok || ensure_pt32(c) != EPOCH_OK || ensure_param_buffers(c) != EPOCH_OK) {
    cudaGetLastError();
    epoch_destroy(c);
    return EPOCH_ERR_CUDA;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    epoch_destroy(c);
    return EPOCH_ERR_CUDA;
  }
  *out = c;
  return EPOCH_OK;
}

// The input mirror (h_in) is written only once the last copy out of it has
// been made.
static epoch_status mirror_wait(epoch_ctx *c) {
  CK(cudaEventSynchronize(c->in_ev), "cudaEventSynchronize(inputs)");
  return EPOCH_OK;
}

// Copies doubles [lo, hi) of the input mirror to the device block and, when
// n_dq > 0, the first n_dq doubles of the dQ mirror to d_dQraw (one k_stage
// launch on the context's stream).
static epoch_status upload_inputs(epoch_ctx *c, size_t lo, size_t hi, size_t n_dq = 0) {
  if (hi < lo) hi = lo;
  if (hi == lo && n_dq == 0) return EPOCH_OK;
  CK(launch_stage(c->h_in_dev + lo, c->d_in + lo, hi - lo, c->h_dq_dev, c->d_dQraw, n_dq,
                  c->stream),
     "k_stage(inputs)");
  c->launches++;
  CK(cudaEventRecord(c->in_ev, c->stream), "cudaEventRecord(inputs)");
  return EPOCH_OK;
}

static epoch_status check_boundaries(epoch_ctx *c, const double *boundaries) {
  if (!boundaries) return fail(c, EPOCH_ERR_ARG, "boundaries is NULL");
  for (int j = 0; j < c->d.E - 1; j++) {
    if (!fin(boundaries[j])) return fail(c, EPOCH_ERR_ARG, "non-finite boundary");
    if (j > 0 && !(boundaries[j] > boundaries[j - 1]))
      return fail(c, EPOCH_ERR_ARG, "boundaries must be strictly increasing");
  }
  return EPOCH_OK;
}

epoch_status epoch_set_boundaries(epoch_ctx *c, const double *boundaries) {
  if (!c) return EPOCH_ERR_ARG;
  const int E = c->d.E;
  if (E == 1) return EPOCH_OK;
  epoch_status s = check_boundaries(c, boundaries);
  if (s != EPOCH_OK) return s;
  if ((s = mirror_wait(c)) != EPOCH_OK) return s;
  const size_t o = c->in_off[IN_BOUND];
  memcpy(c->h_in + o, boundaries, sizeof(double) * (E - 1));
  if ((s = upload_inputs(c, o, o + E - 1)) != EPOCH_OK) return s;
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

static epoch_status check_rates(epoch_ctx *c, const double *Q, const double *pi, int normalise,
                                int reversible) {
  if (!Q || !pi) return fail(c, EPOCH_ERR_ARG, "Q or pi is NULL");
  const Dims &d = c->d;
  const int K = d.K;
  double psum = 0.0;
  for (int i = 0; i < K; i++) {
    if (!fin(pi[i]) || !(pi[i] > 0.0)) return fail(c, EPOCH_ERR_NUMERIC, "pi must be > 0");
    psum += pi[i];
  }
  if (fabs(psum - 1.0) > 1e-9) return fail(c, EPOCH_ERR_NUMERIC, "pi must sum to 1");
  for (int s = 0; s < d.S; s++) {
    const double *q = Q + (size_t)s * d.KK;
    double qmax = 0.0;
    for (int i = 0; i < d.KK; i++) {
      if (!fin(q[i])) return fail(c, EPOCH_ERR_NUMERIC, "non-finite rate");
      qmax = fmax(qmax, fabs(q[i]));
    }
    double csum = 0.0;
    for (int i = 0; i < K; i++) {
      double row = 0.0;
      for (int j = 0; j < K; j++) {
        if (i != j && q[i * K + j] < 0.0)
          return fail(c, EPOCH_ERR_NUMERIC, "negative off-diagonal rate");
        row += q[i * K + j];
      }
      if (fabs(row) > 1e-9 * fmax(1.0, qmax))
        return fail(c, EPOCH_ERR_NUMERIC, "rows of Q must sum to zero");
      csum -= pi[i] * q[i * K + i];
    }
    if (normalise && !(csum > 0.0))
      return fail(c, EPOCH_ERR_NUMERIC, "cannot normalise a zero-rate matrix");
    if (reversible) {
      for (int i = 0; i < K; i++)
        for (int j = i + 1; j < K; j++) {
          double a = pi[i] * q[i * K + j], b = pi[j] * q[j * K + i];
          if (fabs(a - b) > 1e-8 * (fabs(a) + fabs(b)) + 1e-300)
            return fail(c, EPOCH_ERR_NUMERIC, "reversible=1 but pi_i q_ij != pi_j q_ji");
        }
    }
  }
  return EPOCH_OK;
}

// Q and pi into the input mirror (after mirror_wait); returns the end of
// the written range, which starts at in_off[IN_Q].
static size_t stage_rates(epoch_ctx *c, const double *Q, const double *pi) {
  const Dims &d = c->d;
  memcpy(c->h_in + c->in_off[IN_Q], Q, sizeof(double) * d.S * d.KK);
  memcpy(c->h_in + c->in_off[IN_PI], pi, sizeof(double) * d.K);
  c->have |= HAVE_RATES;
  return c->in_off[IN_PI] + d.K;
}

epoch_status epoch_set_rate_matrices(epoch_ctx *c, const double *Q, const double *pi,
                                     int normalise, int reversible) {
  if (!c) return EPOCH_ERR_ARG;
  epoch_status s = check_rates(c, Q, pi, normalise, reversible);
  if (s != EPOCH_OK) return s;
  if ((s = mirror_wait(c)) != EPOCH_OK) return s;
  c->normalise = normalise ? 1 : 0;
  if (c->d.reversible != (reversible ? 1 : 0)) invalidate_graphs(c);
  c->d.reversible = reversible ? 1 : 0;
  const size_t hi = stage_rates(c, Q, pi);
  if ((s = upload_inputs(c, c->in_off[IN_Q], hi)) != EPOCH_OK) return s;
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

// dQ through its pinned mirror (which shares the input mirror's event).
static epoch_status upload_dq(epoch_ctx *c, const double *dQ) {
  const size_t n = (size_t)c->d.np * c->d.S * c->d.KK;
  epoch_status s = mirror_wait(c);
  if (s != EPOCH_OK) return s;
  memcpy(c->h_dq, dQ, sizeof(double) * n);
  return upload_inputs(c, 0, 0, n);
}

epoch_status epoch_set_rate_derivatives(epoch_ctx *c, int n_params, const double *dQ) {
  if (!c) return EPOCH_ERR_ARG;
  if (n_params < 0 || n_params > 4096) return fail(c, EPOCH_ERR_ARG, "bad n_params");
  if (n_params > 0 && !dQ) return fail(c, EPOCH_ERR_ARG, "dQ is NULL");
  const Dims &d = c->d;
  for (size_t i = 0; i < (size_t)n_params * d.S * d.KK; i++)
    if (!fin(dQ[i])) return fail(c, EPOCH_ERR_NUMERIC, "non-finite dQ");
  if (n_params != c->d.np) {
    dfree(c->d_dQraw);
    dfree(c->d_Dth);
    dfree(c->d_Dth32);
    dfree(c->d_Dnz);
    c->d_dQraw = nullptr;
    c->d_Dth = nullptr;
    c->d_Dth32 = nullptr;
    c->d_Dnz = nullptr;
    c->d.np = n_params;
    if (c->h_dq) {
      CK(cudaEventSynchronize(c->in_ev), "cudaEventSynchronize(inputs)");
      cudaFreeHost(c->h_dq);
      c->h_dq = nullptr;
      c->h_dq_dev = nullptr;
    }
    if (n_params > 0) {
      const size_t n = (size_t)n_params * d.S * d.KK;
      CK(cudaMallocHost((void **)&c->h_dq, sizeof(double) * n), "cudaMallocHost(dQ)");
      CK(cudaHostGetDevicePointer((void **)&c->h_dq_dev, c->h_dq, 0), "cudaHostGetDevicePointer(dQ)");
      CK(dalloc(&c->d_dQraw, n), "cudaMalloc(dQ)");
      CK(dalloc(&c->d_Dth, n), "cudaMalloc(D)");
      CK(dalloc(&c->d_Dth32, n), "cudaMalloc(D32)");
      CK(dalloc(&c->d_Dnz, (size_t)n_params * d.S), "cudaMalloc(Dnz)");
    }
    epoch_status s = ensure_param_buffers(c);
    if (s != EPOCH_OK) return s;
    invalidate_graphs(c);
  }
  if (n_params > 0) {
    epoch_status s = upload_dq(c, dQ);
    if (s != EPOCH_OK) return s;
  }
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

static epoch_status check_categories(epoch_ctx *c, const double *rates, const double *weights) {
  if (!rates || !weights) return fail(c, EPOCH_ERR_ARG, "rates or weights is NULL");
  double ws = 0.0;
  for (int k = 0; k < c->d.C; k++) {
    if (!fin(rates[k]) || rates[k] < 0.0) return fail(c, EPOCH_ERR_ARG, "bad category rate");
    if (!fin(weights[k]) || weights[k] < 0.0)
      return fail(c, EPOCH_ERR_ARG, "bad category weight");
    ws += weights[k];
  }
  if (!(ws > 0.0)) return fail(c, EPOCH_ERR_ARG, "category weights sum to zero");
  return EPOCH_OK;
}

// Category rates and weights into the input mirror (after mirror_wait);
// returns the end of the written range, which starts at in_off[IN_CATR].
static size_t stage_categories(epoch_ctx *c, const double *rates, const double *weights) {
  memcpy(c->h_in + c->in_off[IN_CATR], rates, sizeof(double) * c->d.C);
  memcpy(c->h_in + c->in_off[IN_CATW], weights, sizeof(double) * c->d.C);
  c->have |= HAVE_CATS;
  return c->in_off[IN_CATW] + c->d.C;
}

epoch_status epoch_set_categories(epoch_ctx *c, const double *rates, const double *weights) {
  if (!c) return EPOCH_ERR_ARG;
  epoch_status s = check_categories(c, rates, weights);
  if (s != EPOCH_OK) return s;
  if ((s = mirror_wait(c)) != EPOCH_OK) return s;
  const size_t hi = stage_categories(c, rates, weights);
  if ((s = upload_inputs(c, c->in_off[IN_CATR], hi)) != EPOCH_OK) return s;
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

epoch_status epoch_set_ambiguity_masks(epoch_ctx *c, int n_masks, const unsigned long long *masks) {
  if (!c) return EPOCH_ERR_ARG;
  const int K = c->d.K;
  if (n_masks < 0 || K + 1 + n_masks > 255) return fail(c, EPOCH_ERR_ARG, "too many masks");
  if (n_masks > 0 && (!masks || K > 64)) return fail(c, EPOCH_ERR_ARG, "masks need K <= 64");
  for (int m = 0; m < n_masks; m++) {
    unsigned long long valid = (K == 64) ? ~0ull : ((1ull << K) - 1ull);
    if ((masks[m] & ~valid) != 0 || masks[m] == 0)
      return fail(c, EPOCH_ERR_ARG, "mask selects no state or a state >= K");
  }
  dfree(c->d_masks);
  c->d_masks = nullptr;
  if (n_masks > 0) {
    CK(dalloc(&c->d_masks, n_masks), "cudaMalloc(masks)");
    c->h_masks.assign(masks, masks + n_masks);
    CK(cudaMemcpyAsync(c->d_masks, c->h_masks.data(), sizeof(unsigned long long) * n_masks,
                       cudaMemcpyHostToDevice, c->stream),
       "cudaMemcpyAsync(masks)");
  } else {
    c->h_masks.clear();
  }
  c->d.n_masks = n_masks;
  c->d.NR = K + 1 + n_masks;
  epoch_status s = ensure_pt32(c);
  if (s != EPOCH_OK) return s;
  invalidate_graphs(c);
  // the kernel path can depend on the number of masks: the tree must be set
  // again (re-planned), then the tip data
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT | HAVE_TIPS | HAVE_TREE);
  c->h_parent.clear();
  c->d.N = 0;
  return EPOCH_OK;
}

static epoch_status validate_heights(epoch_ctx *c, int N, const double *heights, const int *parent) {
  const int nn = 2 * N - 1;
  for (int v = 0; v < nn; v++) {
    if (!fin(heights[v])) return fail(c, EPOCH_ERR_ARG, "non-finite height");
    int u = parent[v];
    if (u >= 0 && !(heights[u] >= heights[v]))
      return fail(c, EPOCH_ERR_ARG, "a parent is younger than its child");
  }
  return EPOCH_OK;
}

epoch_status epoch_set_tree(epoch_ctx *c, int n_taxa, const double *heights, const int *parent,
                            const double *branch_rates) {
  if (!c) return EPOCH_ERR_ARG;
  if (!heights || !parent) return fail(c, EPOCH_ERR_ARG, "heights or parent is NULL");
  if (n_taxa < 2) return fail(c, EPOCH_ERR_ARG, "need at least 2 taxa");
  if (n_taxa > c->max_taxa) return fail(c, EPOCH_ERR_CAPACITY, "more taxa than max_taxa");
  const int N = n_taxa, nn = 2 * N - 1;
  std::vector<int> child;
  int root = -1;
  std::string msg;
  epoch_status s = check_tree(N, heights, parent, branch_rates, &root, &child, nullptr, &msg);
  if (s != EPOCH_OK) return fail(c, s, msg);

  const bool same_topo = (N == c->d.N) && c->h_parent.size() == (size_t)nn &&
                         std::equal(c->h_parent.begin(), c->h_parent.end(), parent);
  if (!same_topo) {
    std::vector<int> level;
    check_tree(N, heights, parent, branch_rates, &root, &child, &level, &msg);
    // group internal nodes by post-order level (1..L); level l-1 of the
    // schedule holds the nodes whose children all lie in earlier levels
    const int L = level[root];
    std::vector<int> count(L + 1, 0), nodes(N - 1);
    for (int u = N; u < nn; u++) count[level[u]]++;
    std::vector<int> start(L + 2, 0);
    for (int l = 1; l <= L; l++) start[l + 1] = start[l] + count[l];
    std::vector<int> fillp(start.begin(), start.end());
    for (int u = N; u < nn; u++) nodes[fillp[level[u]]++] = u;
    c->h_level_off.assign(start.begin() + 1, start.end());  // L+1 entries
    c->h_level_nodes = nodes;
    c->h_child = child;
    c->h_parent.assign(parent, parent + nn);
    int maxw = 0;
    for (int l = 0; l < L; l++) maxw = std::max(maxw, c->h_level_off[l + 1] - c->h_level_off[l]);
    c->max_level_width = maxw;
    c->d.N = N;
    c->d.nn = nn;
    c->topo_version++;
    invalidate_graphs(c);
    // generic adjoint scratch (two children per node of the widest level)
    if (generic_path(c)) {
      dfree(c->d_xbuf);
      c->d_xbuf = nullptr;
      const size_t n = (size_t)2 * maxw * c->d.C * c->d.P * c->d.Kp * elem_size(c->precision);
      CK(cudaMalloc(&c->d_xbuf, n), "cudaMalloc(adjoint scratch)");
    }
    CK(cudaMemcpyAsync(c->d_parent, c->h_parent.data(), sizeof(int) * nn, cudaMemcpyHostToDevice,
                       c->stream),
       "cudaMemcpyAsync(parent)");
    CK(cudaMemcpyAsync(c->d_child, c->h_child.data(), sizeof(int) * 2 * (N - 1),
                       cudaMemcpyHostToDevice, c->stream),
       "cudaMemcpyAsync(child)");
    CK(cudaMemcpyAsync(c->d_level_nodes, c->h_level_nodes.data(), sizeof(int) * (N - 1),
                       cudaMemcpyHostToDevice, c->stream),
       "cudaMemcpyAsync(levels)");
    CK(cudaMemcpyAsync(c->d_level_off, c->h_level_off.data(), sizeof(int) * (L + 1),
                       cudaMemcpyHostToDevice, c->stream),
       "cudaMemcpyAsync(level offsets)");
    c->root = root;
    if (fast_k4(c)) {
      s = plan_k4(c);
      if (s != EPOCH_OK) return s;
    }
    if (small_path(c)) {  // G terms per (branch, pattern)
      const size_t need = (size_t)(c->max_taxa - 1) * c->d.P * 2 * c->d.C * c->d.KK *
                          elem_size(c->precision);
      if (c->gpart_bytes < need) {
        dfree(c->d_Gpart);
        c->d_Gpart = nullptr;
        c->gpart_bytes = need;
        CK(cudaMalloc(&c->d_Gpart, need), "cudaMalloc(G terms)");
      }
    }
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");  // host vectors reused
    c->have &= ~HAVE_TIPS;
  }
  if ((s = mirror_wait(c)) != EPOCH_OK) return s;
  memcpy(c->h_in + c->in_off[IN_HEIGHTS], heights, sizeof(double) * nn);
  s = upload_inputs(c, c->in_off[IN_HEIGHTS], c->in_off[IN_HEIGHTS] + nn);
  if (s != EPOCH_OK) return s;
  if (branch_rates) {
    c->h_brate.assign(branch_rates, branch_rates + nn);
    CK(cudaMemcpyAsync(c->d_brate, c->h_brate.data(), sizeof(double) * nn, cudaMemcpyHostToDevice,
                       c->stream),
       "cudaMemcpyAsync(branch rates)");
  } else {
    std::vector<double> ones(nn, 1.0);
    CK(cudaMemcpyAsync(c->d_brate, ones.data(), sizeof(double) * nn, cudaMemcpyHostToDevice,
                       c->stream),
       "cudaMemcpyAsync(branch rates)");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  }
  c->have |= HAVE_TREE;
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

epoch_status epoch_set_heights(epoch_ctx *c, const double *heights) {
  if (!c) return EPOCH_ERR_ARG;
  if (!(c->have & HAVE_TREE)) return fail(c, EPOCH_ERR_ORDER, "set_heights before set_tree");
  if (!heights) return fail(c, EPOCH_ERR_ARG, "heights is NULL");
  epoch_status s = validate_heights(c, c->d.N, heights, c->h_parent.data());
  if (s != EPOCH_OK) return s;
  if ((s = mirror_wait(c)) != EPOCH_OK) return s;
  memcpy(c->h_in + c->in_off[IN_HEIGHTS], heights, sizeof(double) * c->d.nn);
  s = upload_inputs(c, c->in_off[IN_HEIGHTS], c->in_off[IN_HEIGHTS] + c->d.nn);
  if (s != EPOCH_OK) return s;
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

epoch_status epoch_set_tip_data(epoch_ctx *c, const int *tip_codes, const double *pattern_weights) {
  if (!c) return EPOCH_ERR_ARG;
  if (!(c->have & HAVE_TREE)) return fail(c, EPOCH_ERR_ORDER, "set_tip_data before set_tree");
  if (!tip_codes || !pattern_weights) return fail(c, EPOCH_ERR_ARG, "codes or weights is NULL");
  const Dims &d = c->d;
  const int maxcode = d.K + d.n_masks;
  // marshal int codes into the one-byte device layout [N][Pp] (row stride
  // padded to 16 bytes; padding holds code 0 and is never used as a pattern).
  // The pinned staging area has two halves used in turn; a half is refilled
  // only after the copy out of it (two calls ago) has finished, so this call
  // does not wait for the work queued on the stream.
  uint8_t *stage = c->h_tips_staging + c->tips_staging_cur * c->tips_staging_half;
  CK(cudaEventSynchronize(c->tips_staging_ev[c->tips_staging_cur]), "cudaEventSynchronize");
  std::vector<unsigned> bad(1, 0u);
  for (int x = 0; x < d.N; x++) {  // branch-free so that the loop vectorises
    uint8_t *row = stage + (size_t)x * d.Pp;
    const int *src = tip_codes + (size_t)x * d.P;
    unsigned b = 0;
    for (int p = 0; p < d.P; p++) {
      const unsigned code = (unsigned)src[p];
      b |= (unsigned)(code > (unsigned)maxcode);
      row[p] = (uint8_t)code;
    }
    for (int p = d.P; p < d.Pp; p++) row[p] = 0;
    bad[0] |= b;
  }
  for (unsigned b : bad)
    if (b) return fail(c, EPOCH_ERR_ARG, "tip code out of range");
  float *wf = reinterpret_cast<float *>(stage + (size_t)c->max_taxa * d.Pp);
  for (int p = 0; p < d.P; p++) {
    if (!fin(pattern_weights[p]) || pattern_weights[p] < 0.0)
      return fail(c, EPOCH_ERR_ARG, "bad pattern weight");
    wf[p] = (float)pattern_weights[p];
  }
  for (int p = d.P; p < d.Pp; p++) wf[p] = 0.f;
  CK(cudaMemcpyAsync(c->d_tips, stage, (size_t)d.N * d.Pp, cudaMemcpyHostToDevice, c->stream),
     "cudaMemcpyAsync(tips)");
  CK(cudaMemcpyAsync(c->d_pwf, wf, sizeof(float) * d.Pp, cudaMemcpyHostToDevice, c->stream),
     "cudaMemcpyAsync(weights)");
  c->h_pw.assign(pattern_weights, pattern_weights + d.P);
  CK(cudaMemcpyAsync(c->d_pw, c->h_pw.data(), sizeof(double) * d.P, cudaMemcpyHostToDevice,
                     c->stream),
     "cudaMemcpyAsync(weights)");
  CK(cudaEventRecord(c->tips_staging_ev[c->tips_staging_cur], c->stream), "cudaEventRecord");
  c->tips_staging_cur ^= 1;
  c->have |= HAVE_TIPS;
  c->have &= ~(HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

epoch_status epoch_compute_branch_matrices(epoch_ctx *c) {
  if (!c) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_RATES | HAVE_CATS | HAVE_TREE, "compute_branch_matrices");
  if (s != EPOCH_OK) return s;
  s = enqueue_branch(c);
  if (s != EPOCH_OK) return s;
  CK(join_sides(c), "join");
  c->have |= HAVE_BRANCH;
  c->have &= ~(HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

epoch_status epoch_update_partials(epoch_ctx *c) {
  if (!c) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_BRANCH | HAVE_TIPS, "update_partials");
  if (s != EPOCH_OK) return s;
  s = replay(c, 2, [&] { return enqueue_partials(c); });
  if (s != EPOCH_OK) return s;
  c->have |= HAVE_PARTIALS;
  c->have &= ~HAVE_GRADIENT;
  return EPOCH_OK;
}

epoch_status epoch_log_likelihood(epoch_ctx *c, double *out_lnL) {
  if (!c || !out_lnL) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_PARTIALS, "log_likelihood");
  if (s != EPOCH_OK) return s;
  s = read_status(c);  // the lnL comes back with the status word
  if (s != EPOCH_OK) return s;
  *out_lnL = *c->h_lnl_pinned;
  return EPOCH_OK;
}

epoch_status epoch_site_log_likelihoods(epoch_ctx *c, double *out) {
  if (!c || !out) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_PARTIALS, "site_log_likelihoods");
  if (s != EPOCH_OK) return s;
  CK(cudaMemcpyAsync(out, c->d_site_lnl, sizeof(double) * c->d.P, cudaMemcpyDeviceToHost,
                     c->stream),
     "cudaMemcpyAsync(site lnL)");
  return read_status(c);
}

epoch_status epoch_gradient(epoch_ctx *c, double *d_heights, double *d_boundaries,
                            double *d_params, double *d_branch_rates) {
  if (!c) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_PARTIALS, "gradient");
  if (s != EPOCH_OK) return s;
  if (d_params && c->d.np > 0 && !c->d.reversible)
    return fail(c, EPOCH_ERR_UNSUPPORTED, "parameter gradients need reversible=1");
  s = replay(c, 3, [&] { return enqueue_gradient(c); });
  if (s != EPOCH_OK) return s;
  c->have |= HAVE_GRADIENT;
  return copy_grad_out(c, d_heights, d_boundaries, d_params, d_branch_rates);
}

epoch_status epoch_set_heights_device(epoch_ctx *c, const double *d_heights) {
  if (!c) return EPOCH_ERR_ARG;
  if (!(c->have & HAVE_TREE)) return fail(c, EPOCH_ERR_ORDER, "set_heights_device before set_tree");
  if (!d_heights) return fail(c, EPOCH_ERR_ARG, "heights is NULL");
  CK(cudaMemcpyAsync(c->d_heights, d_heights, sizeof(double) * c->d.nn, cudaMemcpyDeviceToDevice,
                     c->stream),
     "cudaMemcpyAsync(heights)");
  CK(launch_check_heights(c), "height check kernel");
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT);
  return EPOCH_OK;
}

epoch_status epoch_read_results_device(epoch_ctx *c, double *d_lnL, double *d_grad) {
  if (!c) return EPOCH_ERR_ARG;
  if (d_lnL)
    CK(cudaMemcpyAsync(d_lnL, c->d_lnl, sizeof(double), cudaMemcpyDeviceToDevice, c->stream),
       "cudaMemcpyAsync(lnL)");
  if (d_grad) {
    const size_t n = (size_t)2 * c->d.nn + (c->d.E - 1) + c->d.np;
    CK(cudaMemcpyAsync(d_grad, c->d_grad, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                       c->stream),
       "cudaMemcpyAsync(gradient)");
  }
  return EPOCH_OK;
}

epoch_status epoch_get_branch_matrix(epoch_ctx *c, int node, int category, double *out) {
  if (!c || !out) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_BRANCH, "get_branch_matrix");
  if (s != EPOCH_OK) return s;
  if (node < 0 || node >= c->d.nn || c->h_parent[node] < 0)
    return fail(c, EPOCH_ERR_ARG, "node has no branch above it");
  if (category < 0 || category >= c->d.C) return fail(c, EPOCH_ERR_ARG, "bad category");
  CK(cudaMemcpyAsync(out, c->d_P64 + ((size_t)node * c->d.C + category) * c->d.KK,
                     sizeof(double) * c->d.KK, cudaMemcpyDeviceToHost, c->stream),
     "cudaMemcpyAsync(branch matrix)");
  return read_status(c);
}

epoch_status epoch_expected_counts(epoch_ctx *c, double *per_branch, double *per_epoch) {
  if (!c) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_GRADIENT, "expected_counts");
  if (s != EPOCH_OK) return s;
  if (!c->d.reversible)
    return fail(c, EPOCH_ERR_UNSUPPORTED, "expected counts need reversible=1");
  const Dims &d = c->d;
  if (!c->d_jumps) {
    const size_t nn_max = (size_t)(2 * c->max_taxa - 1);
    if (dalloc(&c->d_jumps, nn_max * d.E * d.C * d.KK) != cudaSuccess ||
        dalloc(&c->d_jump_out, (nn_max + d.E) * d.KK) != cudaSuccess) {
      cudaGetLastError();
      dfree(c->d_jumps);
      dfree(c->d_jump_out);
      c->d_jumps = c->d_jump_out = nullptr;
      return fail(c, EPOCH_ERR_CAPACITY, "cannot allocate the expected-count buffers");
    }
  }
  double *d_branch = c->d_jump_out, *d_epoch = c->d_jump_out + (size_t)d.nn * d.KK;
  CK(launch_expected_counts(c, d_branch, d_epoch), "expected-count kernels");
  if (per_branch)
    CK(cudaMemcpyAsync(per_branch, d_branch, sizeof(double) * d.nn * d.KK, cudaMemcpyDeviceToHost,
                       c->stream),
       "cudaMemcpyAsync(counts per branch)");
  if (per_epoch)
    CK(cudaMemcpyAsync(per_epoch, d_epoch, sizeof(double) * d.E * d.KK, cudaMemcpyDeviceToHost,
                       c->stream),
       "cudaMemcpyAsync(counts per epoch)");
  return read_status(c);
}

epoch_status epoch_ancestral_states(epoch_ctx *c, double *out) {
  if (!c || !out) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_GRADIENT, "ancestral_states");
  if (s != EPOCH_OK) return s;
  const Dims &d = c->d;
  if (!c->d_anc &&
      dalloc(&c->d_anc, (size_t)(c->max_taxa - 1) * d.P * d.K) != cudaSuccess) {
    cudaGetLastError();
    c->d_anc = nullptr;
    return fail(c, EPOCH_ERR_CAPACITY, "cannot allocate the ancestral-state buffer");
  }
  CK(launch_ancestral(c, c->d_anc), "ancestral-state kernel");
  CK(cudaMemcpyAsync(out, c->d_anc, sizeof(double) * (d.N - 1) * d.P * d.K,
                     cudaMemcpyDeviceToHost, c->stream),
     "cudaMemcpyAsync(ancestral states)");
  return read_status(c);
}

epoch_status epoch_evaluate_async(epoch_ctx *c, int with_gradient) {
  if (!c) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_RATES | HAVE_CATS | HAVE_TREE | HAVE_TIPS, "evaluate_async");
  if (s != EPOCH_OK) return s;
  const int g = with_gradient ? 1 : 0;
  s = replay(c, g, [&] {
    epoch_status es = enqueue_branch(c);
    if (es == EPOCH_OK) es = enqueue_partials(c);
    if (es == EPOCH_OK && g) es = enqueue_gradient(c);
    return es;
  });
  if (s != EPOCH_OK) return s;
  c->have |= HAVE_BRANCH | HAVE_PARTIALS;
  if (g)
    c->have |= HAVE_GRADIENT;
  else
    c->have &= ~HAVE_GRADIENT;
  return EPOCH_OK;
}

epoch_status epoch_evaluate_step(epoch_ctx *c, const double *Q, const double *pi, const double *dQ,
                                 const double *boundaries, const double *cat_rates,
                                 const double *cat_weights, const double *heights,
                                 int with_gradient, double *lnL, double *d_heights,
                                 double *d_boundaries, double *d_params, double *d_branch_rates) {
  if (!c) return EPOCH_ERR_ARG;
  const Dims &d = c->d;
  // every given input is checked before any is taken
  epoch_status s = EPOCH_OK;
  if ((Q != nullptr) != (pi != nullptr)) return fail(c, EPOCH_ERR_ARG, "Q and pi go together");
  if ((cat_rates != nullptr) != (cat_weights != nullptr))
    return fail(c, EPOCH_ERR_ARG, "category rates and weights go together");
  if (Q && (s = check_rates(c, Q, pi, c->normalise, d.reversible)) != EPOCH_OK) return s;
  if (dQ && d.np > 0)
    for (size_t i = 0; i < (size_t)d.np * d.S * d.KK; i++)
      if (!fin(dQ[i])) return fail(c, EPOCH_ERR_NUMERIC, "non-finite dQ");
  if (boundaries && d.E > 1 && (s = check_boundaries(c, boundaries)) != EPOCH_OK) return s;
  if (cat_rates && (s = check_categories(c, cat_rates, cat_weights)) != EPOCH_OK) return s;
  if (heights) {
    if (!(c->have & HAVE_TREE)) return fail(c, EPOCH_ERR_ORDER, "heights before set_tree");
    if ((s = validate_heights(c, d.N, heights, c->h_parent.data())) != EPOCH_OK) return s;
  }
  // all of them into the mirror, then one copy over the span they cover:
  // the regions in between hold what the device block holds
  if ((s = mirror_wait(c)) != EPOCH_OK) return s;
  size_t lo = c->in_off[IN_END], hi = 0;
  auto span = [&](size_t a, size_t b) {
    lo = std::min(lo, a);
    hi = std::max(hi, b);
  };
  if (Q) span(c->in_off[IN_Q], stage_rates(c, Q, pi));
  if (boundaries && d.E > 1) {
    memcpy(c->h_in + c->in_off[IN_BOUND], boundaries, sizeof(double) * (d.E - 1));
    span(c->in_off[IN_BOUND], c->in_off[IN_BOUND] + d.E - 1);
  }
  if (cat_rates) span(c->in_off[IN_CATR], stage_categories(c, cat_rates, cat_weights));
  if (heights) {
    memcpy(c->h_in + c->in_off[IN_HEIGHTS], heights, sizeof(double) * d.nn);
    span(c->in_off[IN_HEIGHTS], c->in_off[IN_HEIGHTS] + d.nn);
  }
  size_t n_dq = 0;
  if (dQ && d.np > 0) {
    n_dq = (size_t)d.np * d.S * d.KK;
    memcpy(c->h_dq, dQ, sizeof(double) * n_dq);
  }
  if ((s = upload_inputs(c, lo, hi, n_dq)) != EPOCH_OK) return s;
  c->have &= ~(HAVE_BRANCH | HAVE_PARTIALS | HAVE_GRADIENT);
  s = epoch_evaluate_async(c, with_gradient);
  if (s != EPOCH_OK) return s;
  if (!with_gradient) return epoch_read_results(c, lnL, nullptr, nullptr, nullptr, nullptr);
  return epoch_read_results(c, lnL, d_heights, d_boundaries, d_params, d_branch_rates);
}

epoch_status epoch_read_results(epoch_ctx *c, double *lnL, double *d_heights,
                                double *d_boundaries, double *d_params, double *d_branch_rates) {
  if (!c) return EPOCH_ERR_ARG;
  epoch_status s = need(c, HAVE_PARTIALS, "read_results");
  if (s != EPOCH_OK) return s;
  // the lnL comes back with the status word (and the gradient) in one copy
  if (d_heights || d_boundaries || d_params || d_branch_rates) {
    s = copy_grad_out(c, d_heights, d_boundaries, d_params, d_branch_rates);
  } else {
    s = read_status(c);
  }
  if (s != EPOCH_OK) return s;
  if (lnL) *lnL = *c->h_lnl_pinned;
  return EPOCH_OK;
}

}  // extern "C"
