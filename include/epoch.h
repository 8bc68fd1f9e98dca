/*
 * epoch.h -- C ABI of libepoch, a B300 (sm_103a) library for the tree
 * likelihood and its gradient under the epoch (time-heterogeneous)
 * substitution model of Bielejec, Lemey, Baele, Rambaut and Suchard,
 * "Inferring heterogeneous evolutionary processes through time"
 * (arXiv 1309.3075).
 *
 * Model (paper, Methods and "Relaxing time-homogeneity"):
 *   S rate matrices Q_s (K x K, rows sum to zero); epoch boundaries
 *   b_1 < ... < b_{E-1}; epoch e is governed by Q_{phi(e)}.  For the branch
 *   above node v (parent u) and rate category c the transition matrix is the
 *   time-ordered product of exp(r_v rho_c dt_k Q_{phi(e_k)}) over the epoch
 *   segments k the branch spans, the segment at the parent end on the left
 *   (Eq. matrixProduct, Eq. convolution).  Felsenstein pruning
 *   (Eq. partial_likelihood) runs over all site patterns and categories and
 *   lnL = sum_p n_p log sum_c w_c sum_i pi_i L_root(c,p,i).
 *
 * Conventions used by every entry point:
 *   - Times are HEIGHTS before the youngest tip (>= 0 not required, only
 *     parent height >= child height).  Epoch 0 = [0, b_1) is the youngest,
 *     epoch E-1 = [b_{E-1}, +inf) the oldest.  A segment belongs to the epoch
 *     of its lower end; pieces of zero length are dropped, except that a
 *     zero-length branch keeps one zero-length segment (P = I) so its height
 *     derivatives are one-sided.
 *   - Matrices are row-major FP64, row = parent (ancestral) state.
 *   - Nodes: tips 0..N-1, internal nodes N..2N-2; parent[root] = -1; the tree
 *     is binary (every internal node has exactly two children).
 *   - Tip codes: 0..K-1 observed state, K = missing (every state allowed),
 *     K+1+m = ambiguity mask m (see epoch_set_ambiguity_masks).
 *   - Every Q_s is normalised separately (when asked) so that
 *     sum_i pi_i q_ii = -1 (Methods, after Eq. makeprobs); pi is also the root
 *     distribution.
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership.  The context owns all device memory it allocates.
 *   - Calls are ordered: create -> set_rate_matrices -> set_categories ->
 *     set_tree -> set_tip_data -> compute_branch_matrices -> update_partials
 *     -> log_likelihood / gradient.  A call whose inputs are not yet set
 *     returns EPOCH_ERR_ORDER.  Setting an input again invalidates the
 *     results that depend on it.
 *   - Nothing aborts.  Invalid arguments are rejected on the host before any
 *     device work (EPOCH_ERR_ARG, EPOCH_ERR_NUMERIC); device-side failures
 *     (non-finite partials, an eigensolver that did not converge, a bounded
 *     wait that ran out) are reported through a device status word read at
 *     the next synchronising call.  epoch_last_error() gives a message.
 *     lnL = -inf for an impossible pattern is a valid result, not an error.
 *   - All device work is enqueued on the context's CUDA stream.  Calls
 *     documented "async" return without synchronising; calls that return
 *     host results synchronise that stream.
 */
#ifndef EPOCH_H
#define EPOCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPOCH_MAX_STATES 64   /* K <= 64                                   */
#define EPOCH_MAX_EPOCHS 32   /* E <= 32                                   */
#define EPOCH_MAX_CATEGORIES 16
#define EPOCH_NOALLOC_MAX_PATTERNS 262144 /* epoch_site_log_sum_noalloc */

typedef struct epoch_ctx epoch_ctx; /* opaque; owns all device memory */

typedef enum {
  EPOCH_OK = 0,
  EPOCH_ERR_ARG = 1,      /* invalid argument (size, index, NULL, order of heights) */
  EPOCH_ERR_ORDER = 2,    /* an input this call needs has not been set        */
  EPOCH_ERR_CAPACITY = 3, /* more taxa/patterns than the context was made for */
  EPOCH_ERR_NUMERIC = 4,  /* NaN/negative rates, rows not summing to 0, ...   */
  EPOCH_ERR_CUDA = 5,     /* a CUDA runtime call failed                       */
  EPOCH_ERR_TIMEOUT = 6,  /* a bounded device-side wait ran out               */
  EPOCH_ERR_UNSUPPORTED = 7 /* valid request the library does not support     */
} epoch_status;

typedef enum {
  EPOCH_FP64 = 0,     /* plain FP64 path: one thread per (pattern, category, state) */
  EPOCH_FP32 = 1,     /* FP32 partials with per-pattern power-of-two rescaling,
                         contractions on the FP32 SIMT pipes */
  EPOCH_FP32_TC = 2,  /* FP32 partials; for 8 < K <= 64 and at most 4
                         categories the partials contractions (S = P L in
                         pruning, S and U = P^T X in the adjoint) run on the
                         tensor cores (tcgen05, tiles 16, 32 or 64 states
                         wide) as three TF32 products of the split
                         x = hi + lo (hi hi + hi lo + lo hi), FP32
                         accumulate; other shapes as EPOCH_FP32 */
  EPOCH_FP32_AUTO = 3, /* EPOCH_FP32, EPOCH_FP32_TC or EPOCH_FP32_TC_BF16,
                         whichever evaluates lnL + gradient fastest for this
                         shape on this device: the first context of a (K,
                         categories, pattern-count bucket) times each on a
                         synthetic problem of that shape and the choice is
                         kept for the process
                         (epoch_path_info reports it).  K <= 8 or more than
                         4 categories: EPOCH_FP32 without a probe */
  EPOCH_FP32_TC_BF16 = 4 /* as EPOCH_FP32_TC, with the tile products as BF16 x 3:
                         x = x1 + x2 + x3 (each part the rest rounded to
                         BF16), A B ~ A1 B1 + A1 B2 + A2 B1 + A1 B3 + A2 B2 +
                         A3 B1 on tcgen05 kind::f16, FP32 accumulate */
} epoch_precision;

/* ---- context ----------------------------------------------------------- */

/* Create a context.
 *   states       K, 2..EPOCH_MAX_STATES
 *   n_epochs     E >= 1
 *   boundaries   [E-1] heights, strictly increasing (NULL if E == 1)
 *   epoch_to_matrix [E] phi(e) in 0..n_matrices-1, or NULL = identity (S = E)
 *   n_matrices   S
 *   max_taxa     largest N a later epoch_set_tree may use (>= 2)
 *   n_patterns   P >= 1 (site patterns)
 *   n_categories C, 1..EPOCH_MAX_CATEGORIES
 *   precision    an epoch_precision value
 *   cuda_stream  cudaStream_t to enqueue on, or NULL for a private stream
 * Allocates every device buffer the path needs (partials, scale exponents,
 * branch matrices, work lists).  On error *out is NULL. */
epoch_status epoch_create(epoch_ctx **out, int states, int n_epochs,
                          const double *boundaries, const int *epoch_to_matrix,
                          int n_matrices, int max_taxa, int n_patterns,
                          int n_categories, int precision, void *cuda_stream);

void epoch_destroy(epoch_ctx *ctx);

/* The path a context runs (an epoch_precision value; EPOCH_FP32_AUTO is
 * resolved at creation) and, for EPOCH_FP32_AUTO, the probe's lnL + gradient
 * times in ms on the SIMT, the TF32 x 3 and the BF16 x 3 tensor-core paths
 * (-1 when no probe ran or a path could not run).  Any pointer may be NULL.
 * Not in the paper: a report of the library's own choice between
 * implementations of the same computation. */
epoch_status epoch_path_info(const epoch_ctx *ctx, int *precision_in_use, double *probe_ms_simt,
                             double *probe_ms_tc, double *probe_ms_tc_bf16);

/* Human-readable text of the last failure on this context ("" if none). */
const char *epoch_last_error(const epoch_ctx *ctx);
const char *epoch_status_string(epoch_status s);

/* ---- model inputs ------------------------------------------------------- */

/* Replace the epoch boundaries (same E).  [E-1] heights, strictly increasing. */
epoch_status epoch_set_boundaries(epoch_ctx *ctx, const double *boundaries);

/* Rate matrices Q [S][K][K] (off-diagonals >= 0, rows sum to 0 within
 * 1e-9 * max|q|) and pi [K] (> 0, sums to 1).  normalise = 1 scales each Q_s
 * to sum_i pi_i q_ii = -1 (Methods).  reversible = 1 promises
 * pi_i q_ij = pi_j q_ji (checked) and selects the eigen path (symmetric
 * Jacobi on Pi^{1/2} Q Pi^{-1/2}, P = V diag(exp(tau lambda)) V^{-1});
 * reversible = 0 selects uniformisation for general Q.  The decomposition
 * itself runs on the device in epoch_compute_branch_matrices. */
epoch_status epoch_set_rate_matrices(epoch_ctx *ctx, const double *Q,
                                     const double *pi, int normalise,
                                     int reversible);

/* Model parameters theta_a for the gradient: dQ [n_params][S][K][K] holds
 * d Q_s / d theta_a of the matrices passed to epoch_set_rate_matrices
 * (before normalisation; the derivative of the normalising constant is
 * added by the library).  n_params = 0 clears them.  Parameter gradients
 * need reversible = 1. */
epoch_status epoch_set_rate_derivatives(epoch_ctx *ctx, int n_params,
                                        const double *dQ);

/* Among-site rate categories: rates rho_c [C] (>= 0) and weights w_c [C]
 * (>= 0).  The paper leaves the distribution open; callers typically pass
 * discrete-gamma rates with equal weights. */
epoch_status epoch_set_categories(epoch_ctx *ctx, const double *rates,
                                  const double *weights);

/* Ambiguity masks for tip codes K+1 .. K+n_masks: bit j of masks[m] set =
 * state j allowed.  Needs K <= 64 and K + 1 + n_masks <= 255. */
epoch_status epoch_set_ambiguity_masks(epoch_ctx *ctx, int n_masks,
                                       const unsigned long long *masks);

/* Tree: n_taxa N (2..max_taxa), heights [2N-1], parent [2N-1] (root -1;
 * tips 0..N-1, internal N..2N-2, binary), branch_rates [2N-1] (r_v of the
 * branch above v; NULL = all 1).  The host validates the topology and
 * builds the post-order level schedule; heights are copied to the device
 * where the branches are cut at the epoch boundaries. */
epoch_status epoch_set_tree(epoch_ctx *ctx, int n_taxa, const double *heights,
                            const int *parent, const double *branch_rates);

/* Host-only check of a tree (no context, no device): the same topology,
 * height-order and branch-rate checks epoch_set_tree makes.  On success
 * *n_levels (if not NULL) = number of post-order levels of internal nodes
 * (tips are level 0, an internal node 1 + the max of its children's). */
epoch_status epoch_check_tree(int n_taxa, const double *heights, const int *parent,
                              const double *branch_rates, int *n_levels);

/* New heights for the current topology ([2N-1], parent >= child). */
epoch_status epoch_set_heights(epoch_ctx *ctx, const double *heights);

/* Tip data: codes [N][P] (see conventions) and pattern weights n_p [P] >= 0. */
epoch_status epoch_set_tip_data(epoch_ctx *ctx, const int *tip_codes,
                                const double *pattern_weights);

/* ---- the hot path ------------------------------------------------------- */

/* Async.  Cuts every branch at the boundaries, normalises and decomposes
 * the Q_s (FP64), and forms P_{v,c} for every branch and category as the
 * time-ordered product of segment exponentials (FP64, Eq. convolution). */
epoch_status epoch_compute_branch_matrices(epoch_ctx *ctx);

/* Async.  Post-order pruning over all patterns and categories with
 * per-pattern power-of-two rescaling after every internal node, then the
 * root sum and the weighted FP64 log-sum.  Replayed from a CUDA graph that
 * the context captures on the first call and again after the topology or a
 * size changes. */
epoch_status epoch_update_partials(epoch_ctx *ctx);

/* Synchronises; returns lnL of the last epoch_update_partials. */
epoch_status epoch_log_likelihood(epoch_ctx *ctx, double *out_lnL);

/* Synchronises; per-pattern log-likelihoods [P] (scale factors included). */
epoch_status epoch_site_log_likelihoods(epoch_ctx *ctx, double *out);

/* Gradient of lnL by a pre-order adjoint pass over the stored post-order
 * partials, per-branch dlnL/dP, then the chain rule through the segment
 * products, replayed from a CUDA graph captured on the first call (and again
 * after the topology or a size changes).  Synchronises.  Each output may be
 * NULL (not wanted):
 *   d_heights      [2N-1]  d lnL / d height of every node
 *   d_boundaries   [E-1]   d lnL / d b_k
 *   d_params       [n_params] d lnL / d theta_a (needs reversible = 1)
 *   d_branch_rates [2N-1]  d lnL / d r_v (entry of the root is 0)
 * Derivatives at a height that coincides with a boundary are one-sided
 * (taken from the segment that exists). */
epoch_status epoch_gradient(epoch_ctx *ctx, double *d_heights,
                            double *d_boundaries, double *d_params,
                            double *d_branch_rates);

/* Expected numbers of transitions i -> j ("Markov jumps") given the data,
 * summed over the weighted patterns (n_p) and the rate categories, for the
 * inputs of the last gradient evaluation (epoch_gradient, or
 * epoch_evaluate_async with with_gradient = 1; EPOCH_ERR_ORDER otherwise).
 * Not in the paper: it uses the per-branch adjoints G = d lnL / d P of the
 * gradient.  For a segment with E = exp(tau Q_s) (tau = r_v rho_c dt) the
 * expected count given both end states is q_ij d log E_ab / d q_ij with
 * q_ii held fixed (a path's density is a product of jump factors q_ij and
 * holding factors); over the data this is
 *   N_ij = q_ij < A^T G Z^T , dE/dq_ij >,
 * A / Z the products of the segment exponentials above / below (Eq.
 * convolution), dE/dq_ij by the Daleckii-Krein form of the eigensystem.
 * q is the normalised Q_s, so counts do not depend on the normalisation.
 * Outputs (host, caller-owned, either may be NULL), diagonal entries 0:
 *   per_branch [2N-1][K][K]  summed over the branch's segments (root: 0);
 *   per_epoch  [E][K][K]     summed over the segments lying in epoch e.
 * FP64 on every precision (from the path's G).  Needs reversible = 1
 * (EPOCH_ERR_UNSUPPORTED otherwise).  Synchronises.  Allocates a per-
 * segment buffer [2N-1][E][C][K][K] doubles on first use
 * (EPOCH_ERR_CAPACITY if that fails). */
epoch_status epoch_expected_counts(epoch_ctx *ctx, double *per_branch, double *per_epoch);

/* Marginal posterior probability of the state of every internal node given
 * each pattern, for the inputs of the last gradient evaluation
 * (EPOCH_ERR_ORDER otherwise).  Not in the paper: with L_u the post-order
 * partials (Eq. partial_likelihood) and U_u the outside partials of the
 * adjoint pass, Pr(x_u = i | data_p) = sum_c U_u(c,p,i) L_u(c,p,i) / (its
 * sum over i), the root's U being w_c pi_i.  Any model and precision.
 *   out [N-1][P][K]  host, caller-owned, FP64; row u - N is internal node u.
 * Synchronises.  Allocates an [N-1][P][K] FP64 device buffer on first use
 * (EPOCH_ERR_CAPACITY if that fails). */
epoch_status epoch_ancestral_states(epoch_ctx *ctx, double *out);

/* Test hook: P_{node,cat} [K][K] of the last epoch_compute_branch_matrices. */
epoch_status epoch_get_branch_matrix(epoch_ctx *ctx, int node, int category,
                                     double *out);

/* ---- device-resident evaluation (no host copies) ------------------------ */

/* Async.  The whole path (branch matrices, partials, root and, when
 * with_gradient = 1, the adjoint pass and the chain rule) replayed from a
 * CUDA graph that the context captures on first use and re-captures when
 * the topology or a size changes.  Results stay on the device until
 * epoch_read_results. */
epoch_status epoch_evaluate_async(epoch_ctx *ctx, int with_gradient);

/* Synchronises and copies the results of the last evaluation (any pointer
 * may be NULL). */
epoch_status epoch_read_results(epoch_ctx *ctx, double *lnL, double *d_heights,
                                double *d_boundaries, double *d_params,
                                double *d_branch_rates);

/* Zero-copy variants for callers whose arrays live on the device (a torch
 * tensor's data pointer, on this context's device).  Both are async on the
 * context's stream; order other streams after it with an event.
 *
 * epoch_set_heights_device: d_heights [2N-1] DEVICE pointer, copied on the
 * device.  The tree check runs on the device too: a non-finite height or a
 * parent below its child makes the next synchronising call (read_results,
 * log_likelihood, gradient) return EPOCH_ERR_ARG.
 *
 * epoch_read_results_device: copies the results of the last
 * epoch_evaluate_async into caller DEVICE memory, either pointer may be NULL:
 *   d_lnL  [1]
 *   d_grad [2(2N-1) + (E-1) + n_params]: d/d heights [2N-1], d/d boundaries
 *          [E-1], d/d parameters [n_params], d/d branch rates [2N-1]
 *          (the gradient part holds values only for with_gradient = 1).
 * No status check: call epoch_read_results (or any synchronising call) to
 * see device errors. */
epoch_status epoch_set_heights_device(epoch_ctx *ctx, const double *d_heights);
epoch_status epoch_read_results_device(epoch_ctx *ctx, double *d_lnL, double *d_grad);

/* One step of an inference loop in one call: the per-step inputs that are
 * not NULL replace the current ones exactly as the setters would (Q and pi
 * together, with the context's normalise and reversible flags; dQ with the
 * context's parameter count; category rates and weights together; node
 * heights of the current topology), then lnL (and, with_gradient, the
 * gradient) is evaluated and read back as epoch_read_results.  Synchronises.
 * The same checks and error codes as the separate calls.  Every given input
 * is checked before any is taken, so an invalid input changes nothing; an
 * error of the evaluation itself (a missing set-up call, a device status)
 * comes after the inputs were taken, as with the separate calls.
 * Host arrays (pinned or not) are free again when the call returns: they are
 * copied into the context's pinned staging area, which one small kernel on
 * the context's stream reads into device memory (the results come back the
 * same way), so a step makes no copy-engine transfer. */
epoch_status epoch_evaluate_step(epoch_ctx *ctx, const double *Q, const double *pi,
                                 const double *dQ, const double *boundaries,
                                 const double *cat_rates, const double *cat_weights,
                                 const double *heights, int with_gradient, double *lnL,
                                 double *d_heights, double *d_boundaries, double *d_params,
                                 double *d_branch_rates);

/* Counters: kernels launched by this context since creation (graph
 * replays count their kernels), and graph captures made. */
epoch_status epoch_counters(const epoch_ctx *ctx, long long *kernel_launches,
                            long long *graph_captures);

/* ---- many trees in one launch (the batched trait workload) ---------------- */

/* Log-likelihoods of n_trees independent trees, each with its own taxa,
 * epochs (own boundaries and one K x K rate matrix per epoch), root
 * distribution and at most 4 site patterns, one rate category.  One
 * persistent kernel evaluates all of them (trees are taken from a queue
 * longest first); the launch is captured in a CUDA graph and replayed.  The
 * branch products of Eq. convolution are applied to the partial vectors by
 * uniformisation, so Q need not be reversible.  FP32 partials with
 * per-pattern power-of-two rescaling; FP64 root log-sum.
 * Sizes: 2 <= states <= 64; per tree n_taxa >= 2, 1 <= n_epochs <= 32,
 * 1 <= n_patterns <= 4; the R matrices of the largest tree's epochs must
 * fit in shared memory (n_epochs * K * K * 4 bytes, about 200 KB), else
 * EPOCH_ERR_CAPACITY.  cuda_stream as in epoch_create. */
typedef struct epoch_batch epoch_batch;
epoch_status epoch_batch_create(epoch_batch **out, int states, int n_trees,
                                const int *n_taxa, const int *n_epochs,
                                const int *n_patterns, void *cuda_stream);
void epoch_batch_destroy(epoch_batch *b);
const char *epoch_batch_last_error(const epoch_batch *b);

/* Models of every tree, concatenated in tree order (host arrays, copied):
 *   boundaries [sum_t (E_t - 1)] heights, strictly increasing per tree
 *   Q          [sum_t E_t][K][K] row-major, rows summing to zero; epoch e of
 *              tree t uses its e-th matrix
 *   pi         [n_trees][K] root distribution (and normalisation weights)
 *   normalise  1: each Q scaled so that sum_i pi_i q_ii = -1 */
epoch_status epoch_batch_set_models(epoch_batch *b, const double *boundaries,
                                    const double *Q, const double *pi,
                                    int normalise);

/* Trees, concatenated: heights [sum_t (2 N_t - 1)] and parent (local node
 * indices, tips 0..N_t-1, root -1), same conventions as epoch_set_tree. */
epoch_status epoch_batch_set_trees(epoch_batch *b, const double *heights,
                                   const int *parent);

/* Tip codes [sum_t N_t * P_t] (tree t: [N_t][P_t], 0..K-1, K = missing) and
 * pattern weights [sum_t P_t]. */
epoch_status epoch_batch_set_tip_data(epoch_batch *b, const int *codes,
                                      const double *weights);

/* Async.  The first call times a few launch shapes on the current inputs
 * and keeps the fastest (epoch_batch_launch_shape reports it), then
 * captures the launch in a graph; later calls replay it. */
epoch_status epoch_batch_evaluate_async(epoch_batch *b);

/* Synchronises; lnL [n_trees] of the last evaluation.  EPOCH_ERR_NUMERIC
 * when a partial became non-finite or a branch needed more than 4096
 * uniformisation terms. */
epoch_status epoch_batch_read(epoch_batch *b, double *lnL);

epoch_status epoch_batch_launch_shape(const epoch_batch *b, int *warps_per_cta,
                                      int *ctas_per_sm);

/* lnL and its gradient for every tree in one persistent launch: after a
 * tree's post-order pass, the same CTA runs its pre-order adjoint (outside
 * vectors moved down each branch segment by segment with the transposed
 * uniformised exponential) and differentiates each segment's length,
 * d log L / d dt = ub . Q_e z (Eq. convolution differentiated; Relaxing
 * time-homogeneity).  Height derivatives collect the terms of the segments a
 * node ends; boundary derivatives the terms of the segments on both sides of
 * each crossed boundary.  Sums run in a fixed order (no atomics), so replays
 * are bitwise reproducible.  Async; the first call tunes the launch shape of
 * this variant and captures it in a graph, and allocates the gradient's
 * device buffers (about (sum 2N_t - 1) (E_max + 3) doubles and a scratch of
 * forward vectors per resident warp).  Errors as epoch_batch_evaluate_async. */
epoch_status epoch_batch_evaluate_gradient_async(epoch_batch *b);

/* Synchronises; lnL [n_trees], d lnL_t / d height [sum_t (2 N_t - 1)] (tree
 * order, local node order within a tree; tips included) and d lnL_t / d
 * boundary [sum_t (E_t - 1)] (NULL allowed when every tree has one epoch) of
 * the last evaluation.  EPOCH_ERR_ORDER unless that evaluation was
 * epoch_batch_evaluate_gradient_async with the current inputs;
 * EPOCH_ERR_NUMERIC as epoch_batch_read. */
epoch_status epoch_batch_read_gradient(epoch_batch *b, double *lnL, double *d_heights,
                                       double *d_boundaries);

/* ---- allocation-free root log-sum (no counterpart in the paper) ---------- */

/* The weighted log-sum that ends the root step, for callers that must not
 * have a library allocate device memory (a fixed-footprint sampler loop, a
 * program whose own pool already holds the HBM).  The call allocates
 * nothing: its block sums and counter live in one static device array sized
 * for EPOCH_NOALLOC_MAX_PATTERNS patterns.  Async on cuda_stream (NULL =
 * legacy default stream); no context needed.
 *
 * All pointers are DEVICE pointers owned by the caller:
 *   site_log   [n_patterns]  log of the scaled root sum of each pattern
 *   exponents  [n_rows][row_stride] int16 power-of-two scale exponents of
 *              each pattern (row_stride >= n_patterns); may be NULL when
 *              n_rows = 0
 *   weights    [n_patterns]  pattern weights n_p
 *   site_out   [n_patterns]  out: site_log[p] + ln2 * sum_u exponents[u][p]
 *              (may be NULL)
 *   lnL_out    [1]           out: sum_p n_p site_out[p] (terms with n_p = 0
 *              skipped), summed in a fixed order
 * Returns EPOCH_ERR_ARG for a negative size, a NULL input that is needed or
 * row_stride < n_patterns; EPOCH_ERR_CAPACITY when n_patterns exceeds
 * EPOCH_NOALLOC_MAX_PATTERNS (nothing is launched); EPOCH_ERR_CUDA when the
 * launch fails.
 * The first call on a device looks up the scratch array's address and
 * zeroes its counter (on cuda_stream); make that first call before any
 * stream capture begins.  Calls on the same device that can overlap in time
 * share the scratch and race: order them (one stream, or events). */
epoch_status epoch_site_log_sum_noalloc(const double *site_log,
                                        const int16_t *exponents, int n_rows,
                                        long long row_stride,
                                        const double *weights, int n_patterns,
                                        double *site_out, double *lnL_out,
                                        void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* EPOCH_H */
