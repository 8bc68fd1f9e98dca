/*
 * epoch_oracle.c -- plain, slow, FP64 CPU oracle for the epoch-model tree
 * likelihood of Bielejec et al., "Inferring heterogeneous evolutionary
 * processes through time" (arXiv 1309.3075).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file (through oracle/__init__.py).
 * The product library shares no code, header, table or helper with it.
 *
 * What it computes, each piece following the paper's definition:
 *   - rate normalisation  sum_i pi_i q_ii = -1            (Methods, after Eq. makeprobs)
 *   - P(t) = exp(r t Q)                                  (Methods, Eq. makeprobs)
 *     reversible Q: symmetric eigendecomposition of Pi^{1/2} Q Pi^{-1/2}
 *       (cyclic Jacobi), P = V diag(exp(r t lambda)) V^{-1}
 *       (the eigen-decomposition reuse of Appendix A);
 *     any Q: uniformisation (Jensen 1953), with repeated multiplication when
 *       mu*t is large.
 *   - branch segmentation at the epoch boundaries          (Relaxing time-homogeneity)
 *   - P(t_u,t_v) = product of segment exponentials, parent end first
 *                                                         (Eq. matrixProduct, Eq. convolution)
 *   - Felsenstein pruning                                  (Eq. partial_likelihood)
 *   - root sum  sum_i pi_i L_root(i), sites x categories aggregated
 *                                                         (Methods, after Eq. partial_likelihood)
 *   - brute-force sum over all internal-node states (small trees only)
 *   - analytic gradient: pre-order adjoint, then the derivative of every
 *     branch product formed explicitly and contracted with dlnL/dP.
 *     The paper gives no gradient; the derivative of Eq. convolution is
 *     taken term by term (product rule), and d exp(X)/d theta uses the
 *     block-triangular exponential exp([[X, Y], [0, X]]) (Van Loan 1978).
 *
 * Conventions (readings of the paper where it is silent or garbled):
 *   - times are heights before the youngest tip; epoch 0 = [0, b_1) is the
 *     youngest, epoch E-1 = [b_{E-1}, inf) the oldest;
 *   - P rows = parent (ancestral) state; the left factor of the product is
 *     the segment at the parent end;
 *   - the garbled middle/last factors of Eq. convolution are read as full
 *     epochs T_nu - T_{nu-1} and the final piece from the last boundary to
 *     the child;
 *   - a zero-length branch keeps one zero-length segment (P = I) so that
 *     height derivatives are one-sided; other zero-length pieces are dropped;
 *   - every Q_s is normalised separately with the one pi (flag);
 *   - tip code K = missing (all ones), codes > K index ambiguity masks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "epoch_oracle.h"

/* ------------------------------------------------------------------ */
/* small dense helpers (row-major, n x n)                              */
/* ------------------------------------------------------------------ */

static void mat_identity(int n, double *A) {
  memset(A, 0, sizeof(double) * n * n);
  for (int i = 0; i < n; i++) A[i * n + i] = 1.0;
}

/* C = A * B (C may not alias A or B) */
static void mat_mul(int n, const double *A, const double *B, double *C) {
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      double s = 0.0;
      for (int k = 0; k < n; k++) s += A[i * n + k] * B[k * n + j];
      C[i * n + j] = s;
    }
}

/* A <- A * B using scratch T */
static void mat_mul_right(int n, double *A, const double *B, double *T) {
  mat_mul(n, A, B, T);
  memcpy(A, T, sizeof(double) * n * n);
}

static double frob_dot(int n, const double *A, const double *B) {
  double s = 0.0;
  for (int i = 0; i < n * n; i++) s += A[i] * B[i];
  return s;
}

/* ------------------------------------------------------------------ */
/* Rate normalisation: scale Q so that sum_i pi_i q_ii = -1.           */
/* (Methods: "reparametrizes ... through the constraint")              */
/* ------------------------------------------------------------------ */
double or_normalise(int K, const double *Qraw, const double *pi, double *Qout) {
  double c = 0.0;
  for (int i = 0; i < K; i++) c -= pi[i] * Qraw[i * K + i];
  if (!(c > 0.0)) return c;
  for (int i = 0; i < K * K; i++) Qout[i] = Qraw[i] / c;
  return c;
}

/* ------------------------------------------------------------------ */
/* Symmetric eigendecomposition of a reversible Q.                     */
/* S = Pi^{1/2} Q Pi^{-1/2} is symmetric when pi_i q_ij = pi_j q_ji    */
/* (detailed balance, Methods).  Cyclic Jacobi rotations diagonalise   */
/* S = U diag(lambda) U^T; then Q = V diag(lambda) V^{-1} with          */
/* V = Pi^{-1/2} U and V^{-1} = U^T Pi^{1/2}.                          */
/* Returns the number of sweeps used, or -1 if it did not converge.    */
/* ------------------------------------------------------------------ */
int or_eig_sym(int K, const double *Q, const double *pi, double *lam,
               double *V, double *Vinv) {
  double *S = (double *)malloc(sizeof(double) * K * K);
  double *U = (double *)malloc(sizeof(double) * K * K);
  for (int i = 0; i < K; i++)
    for (int j = 0; j < K; j++)
      S[i * K + j] = sqrt(pi[i]) * Q[i * K + j] / sqrt(pi[j]);
  /* enforce exact symmetry (removes rounding asymmetry only) */
  for (int i = 0; i < K; i++)
    for (int j = i + 1; j < K; j++) {
      double a = 0.5 * (S[i * K + j] + S[j * K + i]);
      S[i * K + j] = a;
      S[j * K + i] = a;
    }
  mat_identity(K, U);
  double scale = 0.0;
  for (int i = 0; i < K * K; i++) scale += S[i] * S[i];
  scale = sqrt(scale);
  int sweep;
  int converged = 0;
  for (sweep = 0; sweep < 100; sweep++) {
    double off = 0.0;
    for (int p = 0; p < K; p++)
      for (int q = p + 1; q < K; q++) off += S[p * K + q] * S[p * K + q];
    if (sqrt(off) <= 1e-16 * scale || off == 0.0) {
      converged = 1;
      break;
    }
    for (int p = 0; p < K; p++) {
      for (int q = p + 1; q < K; q++) {
        double apq = S[p * K + q];
        if (apq == 0.0) continue;
        double app = S[p * K + p], aqq = S[q * K + q];
        /* rotation angle that zeroes the (p,q) entry */
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) /
                   (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0);
        double s = t * c;
        /* S <- J^T S J with J the rotation in the (p,q) plane */
        for (int k = 0; k < K; k++) {
          double skp = S[k * K + p], skq = S[k * K + q];
          S[k * K + p] = c * skp - s * skq;
          S[k * K + q] = s * skp + c * skq;
        }
        for (int k = 0; k < K; k++) {
          double spk = S[p * K + k], sqk = S[q * K + k];
          S[p * K + k] = c * spk - s * sqk;
          S[q * K + k] = s * spk + c * sqk;
        }
        S[p * K + q] = 0.0;
        S[q * K + p] = 0.0;
        for (int k = 0; k < K; k++) {
          double ukp = U[k * K + p], ukq = U[k * K + q];
          U[k * K + p] = c * ukp - s * ukq;
          U[k * K + q] = s * ukp + c * ukq;
        }
      }
    }
  }
  for (int i = 0; i < K; i++) lam[i] = S[i * K + i];
  for (int i = 0; i < K; i++)
    for (int j = 0; j < K; j++) {
      V[i * K + j] = U[i * K + j] / sqrt(pi[i]);
      Vinv[i * K + j] = U[j * K + i] * sqrt(pi[j]);
    }
  /* accept a rounding-level remainder if the sweep limit was hit */
  double off = 0.0;
  for (int p = 0; p < K; p++)
    for (int q = p + 1; q < K; q++) off += S[p * K + q] * S[p * K + q];
  if (!converged && sqrt(off) <= 1e-13 * scale) converged = 1;
  free(S);
  free(U);
  return converged ? sweep : -1;
}

/* P = V diag(exp(tau*lambda)) V^{-1}   (Eq. makeprobs via the eigen-decomposition) */
void or_expm_eig(int K, const double *lam, const double *V, const double *Vinv,
                 double tau, double *P) {
  for (int i = 0; i < K; i++)
    for (int j = 0; j < K; j++) {
      double s = 0.0;
      for (int k = 0; k < K; k++) s += V[i * K + k] * exp(tau * lam[k]) * Vinv[k * K + j];
      P[i * K + j] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Uniformisation: exp(tau Q) = sum_m Pois(m; mu tau) B^m,             */
/* B = I + Q/mu, mu >= max_i |q_ii|.  For mu*tau > 30 the interval is  */
/* split into n equal pieces and the piece result raised to the n-th  */
/* power by repeated multiplication.                                  */
/* ------------------------------------------------------------------ */
static void expm_unif_piece(int K, const double *B, double mt, double *P,
                            double *Bm, double *T) {
  /* P = sum_m e^{-mt} mt^m / m! B^m,  truncated far in the Poisson tail */
  int mmax = (int)ceil(mt + 12.0 * sqrt(mt) + 30.0);
  double w = exp(-mt);
  mat_identity(K, Bm);
  memset(P, 0, sizeof(double) * K * K);
  for (int m = 0; m <= mmax; m++) {
    for (int i = 0; i < K * K; i++) P[i] += w * Bm[i];
    mat_mul_right(K, Bm, B, T);
    w = w * mt / (double)(m + 1);
  }
}

void or_expm_unif(int K, const double *Q, double tau, double *P) {
  double mu = 0.0;
  for (int i = 0; i < K; i++) mu = fmax(mu, fabs(Q[i * K + i]));
  if (mu == 0.0 || tau == 0.0) {
    mat_identity(K, P);
    return;
  }
  double *B = (double *)malloc(sizeof(double) * K * K);
  double *Bm = (double *)malloc(sizeof(double) * K * K);
  double *T = (double *)malloc(sizeof(double) * K * K);
  double *Pp = (double *)malloc(sizeof(double) * K * K);
  for (int i = 0; i < K * K; i++) B[i] = Q[i] / mu;
  for (int i = 0; i < K; i++) B[i * K + i] += 1.0;
  double mt = mu * tau;
  int n = (int)ceil(mt / 30.0);
  if (n < 1) n = 1;
  expm_unif_piece(K, B, mt / n, Pp, Bm, T);
  memcpy(P, Pp, sizeof(double) * K * K);
  for (int r = 1; r < n; r++) mat_mul_right(K, P, Pp, T);
  free(B);
  free(Bm);
  free(T);
  free(Pp);
}

/* ------------------------------------------------------------------ */
/* exp of a general real matrix by scaling and squaring with a long   */
/* Taylor series.  Used only for the block-triangular Frechet         */
/* derivative below (the matrices are small and well scaled).         */
/* ------------------------------------------------------------------ */
static void expm_taylor(int n, const double *A, double *X) {
  double norm = 0.0;
  for (int j = 0; j < n; j++) {
    double col = 0.0;
    for (int i = 0; i < n; i++) col += fabs(A[i * n + j]);
    norm = fmax(norm, col);
  }
  int s = 0;
  while (norm / ldexp(1.0, s) > 0.25) s++;
  double *As = (double *)malloc(sizeof(double) * n * n);
  double *term = (double *)malloc(sizeof(double) * n * n);
  double *T = (double *)malloc(sizeof(double) * n * n);
  for (int i = 0; i < n * n; i++) As[i] = A[i] / ldexp(1.0, s);
  mat_identity(n, X);
  mat_identity(n, term);
  for (int k = 1; k <= 30; k++) {
    mat_mul(n, term, As, T);
    for (int i = 0; i < n * n; i++) term[i] = T[i] / (double)k;
    for (int i = 0; i < n * n; i++) X[i] += term[i];
  }
  for (int r = 0; r < s; r++) mat_mul_right(n, X, X, T);
  free(As);
  free(term);
  free(T);
}

/* Frechet derivative L(X, Y) of exp at X in direction Y, read off the  */
/* upper-right block of exp([[X, Y], [0, X]]).                          */
static void expm_frechet(int K, const double *X, const double *Y, double *L) {
  int n = 2 * K;
  double *M = (double *)calloc((size_t)n * n, sizeof(double));
  double *EM = (double *)malloc(sizeof(double) * n * n);
  for (int i = 0; i < K; i++)
    for (int j = 0; j < K; j++) {
      M[i * n + j] = X[i * K + j];
      M[(i + K) * n + (j + K)] = X[i * K + j];
      M[i * n + (j + K)] = Y[i * K + j];
    }
  expm_taylor(n, M, EM);
  for (int i = 0; i < K; i++)
    for (int j = 0; j < K; j++) L[i * K + j] = EM[i * n + (j + K)];
  free(M);
  free(EM);
}

/* ------------------------------------------------------------------ */
/* Branch segmentation (Relaxing time-homogeneity; Coarse-grain        */
/* parallel implementation: "weights that measure the times that each */
/* of the substitution processes is active on that branch").          */
/* Branch from the parent at height h_hi down to the child at h_lo.   */
/* Segments are listed from the parent end.  Epoch of a segment =      */
/* number of boundaries <= its lower end.  hi_ref/lo_ref name what     */
/* bounds the segment: a node id (>= 0) or boundary j as -(j+1).        */
/* ------------------------------------------------------------------ */
int or_segments(int E, const double *b, double h_lo, double h_hi, int parent,
                int child, int maxseg, int *seg_epoch, double *seg_dt,
                int *hi_ref, int *lo_ref) {
  int n = 0;
  if (h_hi == h_lo) {
    int e = 0;
    for (int j = 0; j < E - 1; j++)
      if (b[j] <= h_lo) e++;
    if (maxseg < 1) return -1;
    seg_epoch[0] = e;
    seg_dt[0] = 0.0;
    hi_ref[0] = parent;
    lo_ref[0] = child;
    return 1;
  }
  double top = h_hi;
  int top_ref = parent;
  /* boundaries strictly inside (h_lo, h_hi), visited from the top down */
  for (int j = E - 2; j >= 0; j--) {
    if (b[j] > h_lo && b[j] < h_hi) {
      if (n >= maxseg) return -1;
      int e = 0;
      for (int k = 0; k < E - 1; k++)
        if (b[k] <= b[j]) e++;
      seg_epoch[n] = e;
      seg_dt[n] = top - b[j];
      hi_ref[n] = top_ref;
      lo_ref[n] = -(j + 1);
      n++;
      top = b[j];
      top_ref = -(j + 1);
    }
  }
  if (n >= maxseg) return -1;
  int e = 0;
  for (int k = 0; k < E - 1; k++)
    if (b[k] <= h_lo) e++;
  seg_epoch[n] = e;
  seg_dt[n] = top - h_lo;
  hi_ref[n] = top_ref;
  lo_ref[n] = child;
  n++;
  return n;
}

/* ------------------------------------------------------------------ */
/* Prepared model: normalised Q_s, eigen systems, per-(branch,cat) P.  */
/* ------------------------------------------------------------------ */
typedef struct {
  const or_problem *pr;
  int K, S, nn, root;
  double *Q;      /* [S][K][K] normalised (or raw if normalise == 0) */
  double *cnorm;  /* [S] normalising constants (1 if not normalised) */
  double *lam, *V, *Vinv; /* eigen systems (reversible only) */
  int *child_off;         /* [nn+1] CSR offsets of the child lists */
  int *child;             /* children of u: child[child_off[u] .. child_off[u+1]) */
  int *post;              /* post-order node list (children before parents) */
} prep_t;

static int node_count(const or_problem *pr) { return 2 * pr->n_taxa - 1; }

static void segment_exp(const prep_t *m, int s, double tau, double *E) {
  int K = m->K;
  if (m->pr->reversible)
    or_expm_eig(K, m->lam + s * K, m->V + s * K * K, m->Vinv + s * K * K, tau, E);
  else
    or_expm_unif(K, m->Q + s * K * K, tau, E);
}

static int prep_init(prep_t *m, const or_problem *pr) {
  memset(m, 0, sizeof(*m));
  m->pr = pr;
  int K = pr->K, S = pr->n_matrices;
  m->K = K;
  m->S = S;
  m->nn = node_count(pr);
  m->Q = (double *)malloc(sizeof(double) * S * K * K);
  m->cnorm = (double *)malloc(sizeof(double) * S);
  for (int s = 0; s < S; s++) {
    if (pr->normalise) {
      double c = or_normalise(K, pr->Q + s * K * K, pr->pi, m->Q + s * K * K);
      if (!(c > 0.0)) return -1;
      m->cnorm[s] = c;
    } else {
      memcpy(m->Q + s * K * K, pr->Q + s * K * K, sizeof(double) * K * K);
      m->cnorm[s] = 1.0;
    }
  }
  if (pr->reversible) {
    m->lam = (double *)malloc(sizeof(double) * S * K);
    m->V = (double *)malloc(sizeof(double) * S * K * K);
    m->Vinv = (double *)malloc(sizeof(double) * S * K * K);
    for (int s = 0; s < S; s++)
      if (or_eig_sym(K, m->Q + s * K * K, pr->pi, m->lam + s * K, m->V + s * K * K,
                     m->Vinv + s * K * K) < 0)
        return -2;
  }
  /* child lists (CSR) */
  int nn = m->nn;
  m->child_off = (int *)calloc(nn + 1, sizeof(int));
  m->root = -1;
  for (int v = 0; v < nn; v++) {
    int u = pr->parent[v];
    if (u < 0) {
      m->root = v;
      continue;
    }
    m->child_off[u + 1]++;
  }
  if (m->root < 0) return -4;
  for (int u = 0; u < nn; u++) m->child_off[u + 1] += m->child_off[u];
  m->child = (int *)malloc(sizeof(int) * (m->child_off[nn] + 1));
  int *fill = (int *)calloc(nn, sizeof(int));
  for (int v = 0; v < nn; v++) {
    int u = pr->parent[v];
    if (u >= 0) m->child[m->child_off[u] + fill[u]++] = v;
  }
  free(fill);
  /* iterative post-order from the root */
  m->post = (int *)malloc(sizeof(int) * nn);
  int *stack = (int *)malloc(sizeof(int) * nn);
  char *seen = (char *)calloc(nn, 1);
  int sp = 0, np = 0;
  stack[sp++] = m->root;
  while (sp > 0) {
    int u = stack[sp - 1];
    if (!seen[u]) {
      seen[u] = 1;
      for (int k = m->child_off[u + 1] - 1; k >= m->child_off[u]; k--)
        stack[sp++] = m->child[k];
    } else {
      sp--;
      m->post[np++] = u;
    }
  }
  free(stack);
  free(seen);
  return np == nn ? 0 : -5;
}

static const int *children_of(const prep_t *m, int u, int *n) {
  *n = m->child_off[u + 1] - m->child_off[u];
  return m->child + m->child_off[u];
}

static void prep_free(prep_t *m) {
  free(m->Q);
  free(m->cnorm);
  free(m->lam);
  free(m->V);
  free(m->Vinv);
  free(m->child_off);
  free(m->child);
  free(m->post);
}

/* segments of the branch above node v */
static int branch_segments(const prep_t *m, int v, int *ep, double *dt, int *hi,
                           int *lo) {
  const or_problem *pr = m->pr;
  int u = pr->parent[v];
  return or_segments(pr->n_epochs, pr->boundaries, pr->heights[v], pr->heights[u], u,
                     v, 64, ep, dt, hi, lo);
}

static double branch_rate(const or_problem *pr, int v) {
  return pr->branch_rates ? pr->branch_rates[v] : 1.0;
}

static int matrix_of_epoch(const or_problem *pr, int e) {
  return pr->epoch_to_matrix ? pr->epoch_to_matrix[e] : e;
}

/* P(t_u, t_v, r_v) for category c: the time-ordered product of Eq. convolution */
static int branch_matrix(const prep_t *m, int v, int c, double *P) {
  const or_problem *pr = m->pr;
  int K = m->K;
  int ep[64], hi[64], lo[64];
  double dt[64];
  int n = branch_segments(m, v, ep, dt, hi, lo);
  if (n < 0) return -1;
  double r = branch_rate(pr, v) * pr->cat_rates[c];
  double *E = (double *)malloc(sizeof(double) * K * K);
  double *T = (double *)malloc(sizeof(double) * K * K);
  mat_identity(K, P);
  for (int k = 0; k < n; k++) {
    segment_exp(m, matrix_of_epoch(pr, ep[k]), r * dt[k], E);
    mat_mul_right(K, P, E, T);
  }
  free(E);
  free(T);
  return 0;
}

int or_branch_matrix(const or_problem *pr, int node, int cat, double *P) {
  prep_t m;
  if (prep_init(&m, pr) != 0) {
    prep_free(&m);
    return -1;
  }
  int rc = branch_matrix(&m, node, cat, P);
  prep_free(&m);
  return rc;
}

/* tip indicator vector: 1 for every state the code allows */
static int tip_allows(const or_problem *pr, int code, int j) {
  int K = pr->K;
  if (code < K) return code == j;
  if (code == K) return 1;
  int mi = code - K - 1;
  if (mi < pr->n_masks) return (int)((pr->masks[mi] >> j) & 1ull);
  return 0;
}

/* all branch matrices, [node][cat][K][K] */
static double *all_branch_matrices(const prep_t *m) {
  const or_problem *pr = m->pr;
  int K = m->K, C = pr->n_categories, nn = m->nn;
  double *P = (double *)calloc((size_t)nn * C * K * K, sizeof(double));
  for (int v = 0; v < nn; v++) {
    if (pr->parent[v] < 0) continue;
    for (int c = 0; c < C; c++) branch_matrix(m, v, c, P + ((size_t)v * C + c) * K * K);
  }
  return P;
}

/* ------------------------------------------------------------------ */
/* One pattern's post-order pass (Eq. partial_likelihood).             */
/* L: [nn][C][K] partials, scaled per node by the max over (c,i) when   */
/* pr->scaling != 0; mscale[u] = that max (1 when not scaled).          */
/* Returns the scaled site value sum_c w_c sum_i pi_i L_root(c,i) and   */
/* the accumulated log of the scale factors in *logscale.              */
/* ------------------------------------------------------------------ */
static double pattern_forward(const prep_t *m, const double *P, int p, double *L,
                              double *mscale, double *logscale) {
  const or_problem *pr = m->pr;
  int K = m->K, C = pr->n_categories, N = pr->n_taxa;
  *logscale = 0.0;
  for (int a = 0; a < m->nn; a++) {
    int u = m->post[a];
    double *Lu = L + (size_t)u * C * K;
    mscale[u] = 1.0;
    if (u < N) {
      int code = pr->tips[(size_t)u * pr->n_patterns + p];
      for (int c = 0; c < C; c++)
        for (int i = 0; i < K; i++) Lu[c * K + i] = tip_allows(pr, code, i) ? 1.0 : 0.0;
      continue;
    }
    int nc;
    const int *ch = children_of(m, u, &nc);
    for (int c = 0; c < C; c++)
      for (int i = 0; i < K; i++) Lu[c * K + i] = 1.0;
    for (int k = 0; k < nc; k++) {
      int v = ch[k];
      const double *Lv = L + (size_t)v * C * K;
      for (int c = 0; c < C; c++) {
        const double *Pv = P + ((size_t)v * C + c) * K * K;
        for (int i = 0; i < K; i++) {
          double s = 0.0;
          for (int j = 0; j < K; j++) s += Pv[i * K + j] * Lv[c * K + j];
          Lu[c * K + i] *= s;
        }
      }
    }
    if (pr->scaling) {
      double mx = 0.0;
      for (int q = 0; q < C * K; q++) mx = fmax(mx, Lu[q]);
      if (mx > 0.0) {
        for (int q = 0; q < C * K; q++) Lu[q] /= mx;
        mscale[u] = mx;
        *logscale += log(mx);
      }
    }
  }
  const double *Lr = L + (size_t)m->root * C * K;
  double site = 0.0;
  for (int c = 0; c < C; c++) {
    double sc = 0.0;
    for (int i = 0; i < K; i++) sc += pr->pi[i] * Lr[c * K + i];
    site += pr->cat_weights[c] * sc;
  }
  return site;
}

double or_log_likelihood(const or_problem *pr, double *site_lnl) {
  prep_t m;
  if (prep_init(&m, pr) != 0) {
    prep_free(&m);
    return NAN;
  }
  int K = pr->K, C = pr->n_categories;
  double *P = all_branch_matrices(&m);
  double *L = (double *)malloc(sizeof(double) * m.nn * C * K);
  double *ms = (double *)malloc(sizeof(double) * m.nn);
  long double total = 0.0L;
  for (int p = 0; p < pr->n_patterns; p++) {
    double ls;
    double site = pattern_forward(&m, P, p, L, ms, &ls);
    double lp = log(site) + ls;
    if (site_lnl) site_lnl[p] = lp;
    total += (long double)pr->pattern_weights[p] * (long double)lp;
  }
  free(P);
  free(L);
  free(ms);
  prep_free(&m);
  return (double)total;
}

/* ------------------------------------------------------------------ */
/* Brute force: sum over every joint assignment of internal-node states */
/* of pi(root state) * prod over branches of the branch factor, where   */
/* a branch into an internal node contributes p_{state(u), state(v)}    */
/* and a branch into a tip contributes sum over the tip's allowed       */
/* states j of p_{state(u), j}.  No pruning, no scaling.  Exponential   */
/* cost: small trees only.                                             */
/* ------------------------------------------------------------------ */
double or_brute_force(const or_problem *pr, double *site_lnl) {
  prep_t m;
  if (prep_init(&m, pr) != 0) {
    prep_free(&m);
    return NAN;
  }
  int K = pr->K, C = pr->n_categories, nn = m.nn, N = pr->n_taxa;
  double *P = all_branch_matrices(&m);
  int *st = (int *)calloc(nn, sizeof(int));
  long double total = 0.0L;
  for (int p = 0; p < pr->n_patterns; p++) {
    double site = 0.0;
    for (int c = 0; c < C; c++) {
      /* odometer over the internal nodes' states */
      for (int u = 0; u < nn; u++) st[u] = 0;
      double sum = 0.0;
      for (;;) {
        double term = pr->pi[st[m.root]];
        for (int v = 0; v < nn; v++) {
          int u = pr->parent[v];
          if (u < 0) continue;
          const double *Pv = P + ((size_t)v * C + c) * K * K;
          if (v < N) {
            int code = pr->tips[(size_t)v * pr->n_patterns + p];
            double f = 0.0;
            for (int j = 0; j < K; j++)
              if (tip_allows(pr, code, j)) f += Pv[st[u] * K + j];
            term *= f;
          } else {
            term *= Pv[st[u] * K + st[v]];
          }
        }
        sum += term;
        int u = N;
        while (u < nn) {
          st[u]++;
          if (st[u] < K) break;
          st[u] = 0;
          u++;
        }
        if (u == nn) break;
      }
      site += pr->cat_weights[c] * sum;
    }
    double lp = log(site);
    if (site_lnl) site_lnl[p] = lp;
    total += (long double)pr->pattern_weights[p] * (long double)lp;
  }
  free(st);
  free(P);
  prep_free(&m);
  return (double)total;
}

/* ------------------------------------------------------------------ */
/* dlnL/dP for every branch and category:                              */
/*   G_v,c[i][j] = sum_p n_p (d site_p / d p_ij) / site_p              */
/* computed with the pre-order ("outside") partials.  With scaled       */
/* partials the ratio is formed from scaled quantities, the factor      */
/* 1/m_u undoing the parent's own scale.                               */
/* ------------------------------------------------------------------ */
static double branch_adjoints(const prep_t *m, const double *P, double *G,
                              double *site_lnl) {
  const or_problem *pr = m->pr;
  int K = m->K, C = pr->n_categories, nn = m->nn;
  double *L = (double *)malloc(sizeof(double) * nn * C * K);
  double *U = (double *)malloc(sizeof(double) * nn * C * K);
  double *ms = (double *)malloc(sizeof(double) * nn);
  double *O = (double *)malloc(sizeof(double) * C * K);
  double *Sk = (double *)malloc(sizeof(double) * C * K);
  memset(G, 0, sizeof(double) * (size_t)nn * C * K * K);
  long double total = 0.0L;
  for (int p = 0; p < pr->n_patterns; p++) {
    double ls;
    double site = pattern_forward(m, P, p, L, ms, &ls);
    double lp = log(site) + ls;
    if (site_lnl) site_lnl[p] = lp;
    double np = pr->pattern_weights[p];
    total += (long double)np * (long double)lp;
    /* root outside partial: d site / d L_root(c,i), divided by site */
    double *Ur = U + (size_t)m->root * C * K;
    for (int c = 0; c < C; c++)
      for (int i = 0; i < K; i++) Ur[c * K + i] = pr->cat_weights[c] * pr->pi[i] / site;
    /* pre-order: parents before children (reverse post-order) */
    for (int a = nn - 1; a >= 0; a--) {
      int u = m->post[a];
      if (u < pr->n_taxa) continue;
      int nc;
      const int *ch = children_of(m, u, &nc);
      const double *Uu = U + (size_t)u * C * K;
      for (int k = 0; k < nc; k++) {
        int v = ch[k];
        /* O = U_u * prod over siblings of (P_w L_w), / m_u */
        for (int q = 0; q < C * K; q++) O[q] = Uu[q] / ms[u];
        for (int k2 = 0; k2 < nc; k2++) {
          if (k2 == k) continue;
          int w = ch[k2];
          const double *Lw = L + (size_t)w * C * K;
          for (int c = 0; c < C; c++) {
            const double *Pw = P + ((size_t)w * C + c) * K * K;
            for (int i = 0; i < K; i++) {
              double s = 0.0;
              for (int j = 0; j < K; j++) s += Pw[i * K + j] * Lw[c * K + j];
              Sk[c * K + i] = s;
            }
          }
          for (int q = 0; q < C * K; q++) O[q] *= Sk[q];
        }
        const double *Lv = L + (size_t)v * C * K;
        double *Uv = U + (size_t)v * C * K;
        for (int c = 0; c < C; c++) {
          const double *Pv = P + ((size_t)v * C + c) * K * K;
          double *Gv = G + ((size_t)v * C + c) * K * K;
          for (int i = 0; i < K; i++)
            for (int j = 0; j < K; j++) Gv[i * K + j] += np * O[c * K + i] * Lv[c * K + j];
          for (int j = 0; j < K; j++) {
            double s = 0.0;
            for (int i = 0; i < K; i++) s += Pv[i * K + j] * O[c * K + i];
            Uv[c * K + j] = s;
          }
        }
      }
    }
  }
  free(L);
  free(U);
  free(ms);
  free(O);
  free(Sk);
  return (double)total;
}

int or_branch_adjoints(const or_problem *pr, double *G, double *lnl) {
  prep_t m;
  if (prep_init(&m, pr) != 0) {
    prep_free(&m);
    return -1;
  }
  double *P = all_branch_matrices(&m);
  double t = branch_adjoints(&m, P, G, NULL);
  if (lnl) *lnl = t;
  free(P);
  prep_free(&m);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Gradient.  For each branch and category the derivative of the        */
/* product of Eq. convolution is formed explicitly, term by term, and   */
/* contracted with G:                                                  */
/*   d/dh_parent : r rho Q_top P                                       */
/*   d/dh_child  : -r rho P Q_bottom                                   */
/*   d/db_j      : r rho A E_above (Q_below - Q_above) E_below Z        */
/*   d/dr_v      : sum_k A_k (rho dt_k Q_k E_k) Z_k                     */
/*   d/dtheta    : sum_k A_k L(tau_k Q_k, tau_k dQ_k/dtheta) Z_k        */
/* A_k / Z_k: products of the segment exponentials above / below k.    */
/* dQ/dtheta includes the derivative of the normalising constant.      */
/* ------------------------------------------------------------------ */
int or_gradient(const or_problem *pr, double *lnl, double *d_heights,
                double *d_boundaries, double *d_params, double *d_rates) {
  prep_t m;
  if (prep_init(&m, pr) != 0) {
    prep_free(&m);
    return -1;
  }
  int K = pr->K, C = pr->n_categories, nn = m.nn, S = pr->n_matrices;
  int KK = K * K;
  int np = pr->n_params;
  if (np > 0 && !pr->dQ) {
    prep_free(&m);
    return -3;
  }
  double *P = all_branch_matrices(&m);
  double *G = (double *)malloc(sizeof(double) * (size_t)nn * C * KK);
  double t = branch_adjoints(&m, P, G, NULL);
  if (lnl) *lnl = t;
  /* derivative of each normalised Q_s with respect to each parameter */
  double *dQn = NULL;
  if (np > 0) {
    dQn = (double *)malloc(sizeof(double) * (size_t)np * S * KK);
    for (int a = 0; a < np; a++)
      for (int s = 0; s < S; s++) {
        const double *dq = pr->dQ + ((size_t)a * S + s) * KK;
        double *out = dQn + ((size_t)a * S + s) * KK;
        if (pr->normalise) {
          double c = m.cnorm[s];
          double dc = 0.0;
          for (int i = 0; i < K; i++) dc -= pr->pi[i] * dq[i * K + i];
          /* Q = Qraw / c  =>  dQ = dQraw / c - Q dc / c */
          for (int q = 0; q < KK; q++) out[q] = dq[q] / c - m.Q[s * KK + q] * dc / c;
        } else {
          memcpy(out, dq, sizeof(double) * KK);
        }
      }
  }
  if (d_heights) memset(d_heights, 0, sizeof(double) * nn);
  if (d_boundaries && pr->n_epochs > 1) memset(d_boundaries, 0, sizeof(double) * (pr->n_epochs - 1));
  if (d_params && np > 0) memset(d_params, 0, sizeof(double) * np);
  if (d_rates) memset(d_rates, 0, sizeof(double) * nn);

  double *Es = (double *)malloc(sizeof(double) * 64 * KK);
  double *A = (double *)malloc(sizeof(double) * KK);
  double *Z = (double *)malloc(sizeof(double) * KK);
  double *T1 = (double *)malloc(sizeof(double) * KK);
  double *T2 = (double *)malloc(sizeof(double) * KK);
  double *D = (double *)malloc(sizeof(double) * KK);
  double *X = (double *)malloc(sizeof(double) * KK);
  double *Y = (double *)malloc(sizeof(double) * KK);
  int ep[64], hi[64], lo[64];
  double dt[64];
  for (int v = 0; v < nn; v++) {
    int u = pr->parent[v];
    if (u < 0) continue;
    int n = branch_segments(&m, v, ep, dt, hi, lo);
    double rb = branch_rate(pr, v);
    for (int c = 0; c < C; c++) {
      double rr = rb * pr->cat_rates[c];
      const double *Gv = G + ((size_t)v * C + c) * KK;
      const double *Pv = P + ((size_t)v * C + c) * KK;
      for (int k = 0; k < n; k++)
        segment_exp(&m, matrix_of_epoch(pr, ep[k]), rr * dt[k], Es + (size_t)k * KK);
      /* parent height: r rho Q_top P */
      {
        const double *Qt = m.Q + (size_t)matrix_of_epoch(pr, ep[0]) * KK;
        mat_mul(K, Qt, Pv, D);
        if (d_heights) d_heights[u] += rr * frob_dot(K, Gv, D);
      }
      /* child height: -r rho P Q_bottom */
      {
        const double *Qb = m.Q + (size_t)matrix_of_epoch(pr, ep[n - 1]) * KK;
        mat_mul(K, Pv, Qb, D);
        if (d_heights) d_heights[v] -= rr * frob_dot(K, Gv, D);
      }
      /* boundaries crossed: cut between segment k (above) and k+1 (below) */
      for (int k = 0; k + 1 < n; k++) {
        int j = -lo[k] - 1;
        const double *Qa = m.Q + (size_t)matrix_of_epoch(pr, ep[k]) * KK;
        const double *Qbl = m.Q + (size_t)matrix_of_epoch(pr, ep[k + 1]) * KK;
        mat_identity(K, A);
        for (int q = 0; q < k; q++) mat_mul_right(K, A, Es + (size_t)q * KK, T1);
        mat_identity(K, Z);
        for (int q = k + 2; q < n; q++) mat_mul_right(K, Z, Es + (size_t)q * KK, T1);
        for (int q = 0; q < KK; q++) X[q] = Qbl[q] - Qa[q];
        mat_mul(K, A, Es + (size_t)k * KK, T1);       /* A E_above */
        mat_mul(K, T1, X, T2);                        /* (Q_below - Q_above) */
        mat_mul(K, T2, Es + (size_t)(k + 1) * KK, T1); /* E_below */
        mat_mul(K, T1, Z, D);
        if (d_boundaries) d_boundaries[j] += rr * frob_dot(K, Gv, D);
      }
      /* per-segment terms: branch rate and model parameters */
      for (int k = 0; k < n; k++) {
        int s = matrix_of_epoch(pr, ep[k]);
        mat_identity(K, A);
        for (int q = 0; q < k; q++) mat_mul_right(K, A, Es + (size_t)q * KK, T1);
        mat_identity(K, Z);
        for (int q = k + 1; q < n; q++) mat_mul_right(K, Z, Es + (size_t)q * KK, T1);
        if (d_rates) {
          mat_mul(K, m.Q + (size_t)s * KK, Es + (size_t)k * KK, T1);
          for (int q = 0; q < KK; q++) T1[q] *= pr->cat_rates[c] * dt[k];
          mat_mul(K, A, T1, T2);
          mat_mul(K, T2, Z, D);
          d_rates[v] += frob_dot(K, Gv, D);
        }
        if (d_params && np > 0) {
          double tau = rr * dt[k];
          for (int q = 0; q < KK; q++) X[q] = tau * m.Q[(size_t)s * KK + q];
          for (int a = 0; a < np; a++) {
            const double *dq = dQn + ((size_t)a * S + s) * KK;
            int nz = 0;
            for (int q = 0; q < KK; q++)
              if (dq[q] != 0.0) nz = 1;
            if (!nz) continue;
            for (int q = 0; q < KK; q++) Y[q] = tau * dq[q];
            expm_frechet(K, X, Y, T1);
            mat_mul(K, A, T1, T2);
            mat_mul(K, T2, Z, D);
            d_params[a] += frob_dot(K, Gv, D);
          }
        }
      }
    }
  }
  free(Es);
  free(A);
  free(Z);
  free(T1);
  free(T2);
  free(D);
  free(X);
  free(Y);
  free(dQn);
  free(G);
  free(P);
  prep_free(&m);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Expected numbers of i -> j transitions (Markov jumps) given the      */
/* data, summed over the weighted patterns and the rate categories.     */
/* A path's density is a product of jump factors (the off-diagonal     */
/* rates of the moves it makes) and holding factors (the diagonal), so  */
/* for a segment with exponential E = exp(tau Q_s), tau = r rho dt, the */
/* expected count given both end states is q_ij d/dq_ij log E_ab with   */
/* q_ii held fixed (Minin and Suchard 2008).  Over the data:           */
/*   N_ij(segment) = q_ij <G, A_k L(tau Q_s, tau e_i e_j^T) Z_k>       */
/* with G = d lnL / d P (branch_adjoints), A_k / Z_k the products of   */
/* the segment exponentials above / below k and L the Frechet          */
/* derivative of exp.  Since <H, L(X, Y)> = <L(X^T, H), Y> (cyclic      */
/* trace of the integral form), all K^2 directions come from one       */
/* derivative: N_ij = q_ij tau [L(tau Q_s^T, H)]_ij, H = A_k^T G Z_k^T. */
/* Outputs: per branch [2N-1][K][K] (the root's block zero) and per    */
/* epoch [E][K][K]; diagonal entries are zero.                         */
/* ------------------------------------------------------------------ */
int or_expected_counts(const or_problem *pr, double *per_branch, double *per_epoch) {
  prep_t m;
  if (prep_init(&m, pr) != 0) {
    prep_free(&m);
    return -1;
  }
  int K = pr->K, C = pr->n_categories, nn = m.nn, E = pr->n_epochs;
  int KK = K * K;
  double *P = all_branch_matrices(&m);
  double *G = (double *)malloc(sizeof(double) * (size_t)nn * C * KK);
  branch_adjoints(&m, P, G, NULL);
  if (per_branch) memset(per_branch, 0, sizeof(double) * (size_t)nn * KK);
  if (per_epoch) memset(per_epoch, 0, sizeof(double) * (size_t)E * KK);
  double *Es = (double *)malloc(sizeof(double) * 64 * KK);
  double *A = (double *)malloc(sizeof(double) * KK);
  double *Z = (double *)malloc(sizeof(double) * KK);
  double *T1 = (double *)malloc(sizeof(double) * KK);
  double *D = (double *)malloc(sizeof(double) * KK);
  double *X = (double *)malloc(sizeof(double) * KK);
  double *Y = (double *)malloc(sizeof(double) * KK);
  int ep[64], hi[64], lo[64];
  double dt[64];
  for (int v = 0; v < nn; v++) {
    if (pr->parent[v] < 0) continue;
    int n = branch_segments(&m, v, ep, dt, hi, lo);
    double rb = branch_rate(pr, v);
    for (int c = 0; c < C; c++) {
      double rr = rb * pr->cat_rates[c];
      const double *Gv = G + ((size_t)v * C + c) * KK;
      for (int k = 0; k < n; k++)
        segment_exp(&m, matrix_of_epoch(pr, ep[k]), rr * dt[k], Es + (size_t)k * KK);
      for (int k = 0; k < n; k++) {
        int s = matrix_of_epoch(pr, ep[k]);
        const double *Qs = m.Q + (size_t)s * KK;
        double tau = rr * dt[k];
        mat_identity(K, A);
        for (int q = 0; q < k; q++) mat_mul_right(K, A, Es + (size_t)q * KK, T1);
        mat_identity(K, Z);
        for (int q = k + 1; q < n; q++) mat_mul_right(K, Z, Es + (size_t)q * KK, T1);
        /* H = A^T G Z^T */
        for (int i = 0; i < K; i++)
          for (int j = 0; j < K; j++) {
            double acc = 0.0;
            for (int a = 0; a < K; a++) acc += A[a * K + i] * Gv[a * K + j];
            T1[i * K + j] = acc;
          }
        for (int i = 0; i < K; i++)
          for (int j = 0; j < K; j++) {
            double acc = 0.0;
            for (int b = 0; b < K; b++) acc += T1[i * K + b] * Z[j * K + b];
            Y[i * K + j] = acc;
          }
        for (int i = 0; i < K; i++)
          for (int j = 0; j < K; j++) X[i * K + j] = tau * Qs[j * K + i]; /* (tau Q)^T */
        expm_frechet(K, X, Y, D);
        for (int i = 0; i < K; i++)
          for (int j = 0; j < K; j++) {
            if (i == j) continue;
            double nij = Qs[i * K + j] * tau * D[i * K + j];
            if (per_branch) per_branch[(size_t)v * KK + i * K + j] += nij;
            if (per_epoch) per_epoch[(size_t)ep[k] * KK + i * K + j] += nij;
          }
      }
    }
  }
  free(Es);
  free(A);
  free(Z);
  free(T1);
  free(D);
  free(X);
  free(Y);
  free(G);
  free(P);
  prep_free(&m);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Marginal posterior of the state of every internal node u given one   */
/* pattern: Pr(x_u = i | data_p) = sum_c w_c O_u(c,i) L_u(c,i) / site_p */
/* with L the post-order partials (Eq. partial_likelihood) and O the    */
/* outside probabilities: O_root(c,i) = pi_i; for a child v of u,       */
/*   O_v(c,j) = sum_i O_u(c,i) (prod_{siblings w} S_w(c,i)) P_v,c[i][j] */
/* (S_w = P_w L_w).  Every vector may carry its own positive factor:    */
/* the posterior is normalised at the end, so L and O are rescaled by   */
/* their maxima.  out[u - N][p][i].                                    */
/* ------------------------------------------------------------------ */
int or_ancestral(const or_problem *pr, double *out) {
  prep_t m;
  if (prep_init(&m, pr) != 0) {
    prep_free(&m);
    return -1;
  }
  int K = pr->K, C = pr->n_categories, nn = m.nn, N = pr->n_taxa, P = pr->n_patterns;
  double *Pm = all_branch_matrices(&m);
  double *L = (double *)malloc(sizeof(double) * nn * C * K);
  double *O = (double *)malloc(sizeof(double) * nn * C * K);
  double *ms = (double *)malloc(sizeof(double) * nn);
  double *T = (double *)malloc(sizeof(double) * C * K);
  for (int p = 0; p < P; p++) {
    double ls;
    pattern_forward(&m, Pm, p, L, ms, &ls);
    /* outside pass, parents before children (reverse post-order) */
    for (int c = 0; c < C; c++)
      for (int i = 0; i < K; i++) O[((size_t)m.root * C + c) * K + i] = pr->cat_weights[c] * pr->pi[i];
    for (int a = nn - 1; a >= 0; a--) {
      int u = m.post[a];
      if (u < N) continue;
      int nc;
      const int *ch = children_of(&m, u, &nc);
      for (int k = 0; k < nc; k++) {
        int v = ch[k];
        for (int q = 0; q < C * K; q++) T[q] = O[(size_t)u * C * K + q];
        for (int k2 = 0; k2 < nc; k2++) {
          if (k2 == k) continue;
          int w = ch[k2];
          for (int c = 0; c < C; c++) {
            const double *Pw = Pm + ((size_t)w * C + c) * K * K;
            for (int i = 0; i < K; i++) {
              double sw = 0.0;
              for (int j = 0; j < K; j++) sw += Pw[i * K + j] * L[((size_t)w * C + c) * K + j];
              T[c * K + i] *= sw;
            }
          }
        }
        double mx = 0.0;
        for (int c = 0; c < C; c++) {
          const double *Pv = Pm + ((size_t)v * C + c) * K * K;
          for (int j = 0; j < K; j++) {
            double o = 0.0;
            for (int i = 0; i < K; i++) o += T[c * K + i] * Pv[i * K + j];
            O[((size_t)v * C + c) * K + j] = o;
            mx = fmax(mx, o);
          }
        }
        if (mx > 0.0)
          for (int q = 0; q < C * K; q++) O[(size_t)v * C * K + q] /= mx;
      }
    }
    for (int u = N; u < nn; u++) {
      double *o = out + ((size_t)(u - N) * P + p) * K;
      double tot = 0.0;
      for (int i = 0; i < K; i++) {
        double x = 0.0;
        for (int c = 0; c < C; c++) x += O[((size_t)u * C + c) * K + i] * L[((size_t)u * C + c) * K + i];
        o[i] = x;
        tot += x;
      }
      for (int i = 0; i < K; i++) o[i] = tot > 0.0 ? o[i] / tot : 0.0;
    }
  }
  free(Pm);
  free(L);
  free(O);
  free(ms);
  free(T);
  prep_free(&m);
  return 0;
}

/* The same posteriors by enumeration of every joint assignment of the   */
/* internal nodes' states (the brute-force joint of or_brute_force,      */
/* accumulated per node and state).  Small trees only.                   */
int or_ancestral_brute(const or_problem *pr, double *out) {
  prep_t m;
  if (prep_init(&m, pr) != 0) {
    prep_free(&m);
    return -1;
  }
  int K = pr->K, C = pr->n_categories, nn = m.nn, N = pr->n_taxa, Pn = pr->n_patterns;
  double *P = all_branch_matrices(&m);
  int *st = (int *)calloc(nn, sizeof(int));
  for (int p = 0; p < Pn; p++) {
    for (int u = N; u < nn; u++)
      for (int i = 0; i < K; i++) out[((size_t)(u - N) * Pn + p) * K + i] = 0.0;
    double site = 0.0;
    for (int c = 0; c < C; c++) {
      for (int u = 0; u < nn; u++) st[u] = 0;
      for (;;) {
        double term = pr->cat_weights[c] * pr->pi[st[m.root]];
        for (int v = 0; v < nn; v++) {
          int u = pr->parent[v];
          if (u < 0) continue;
          const double *Pv = P + ((size_t)v * C + c) * K * K;
          if (v < N) {
            int code = pr->tips[(size_t)v * Pn + p];
            double f = 0.0;
            for (int j = 0; j < K; j++)
              if (tip_allows(pr, code, j)) f += Pv[st[u] * K + j];
            term *= f;
          } else {
            term *= Pv[st[u] * K + st[v]];
          }
        }
        site += term;
        for (int u = N; u < nn; u++) out[((size_t)(u - N) * Pn + p) * K + st[u]] += term;
        int u = N;
        while (u < nn) {
          st[u]++;
          if (st[u] < K) break;
          st[u] = 0;
          u++;
        }
        if (u == nn) break;
      }
    }
    for (int u = N; u < nn; u++)
      for (int i = 0; i < K; i++) out[((size_t)(u - N) * Pn + p) * K + i] /= site;
  }
  free(st);
  free(P);
  prep_free(&m);
  return 0;
}

/* exported eigen/exp helpers for the tests */
int or_expm(int K, const double *Q, const double *pi, int reversible, double tau,
            double *P) {
  if (reversible) {
    double *lam = (double *)malloc(sizeof(double) * K);
    double *V = (double *)malloc(sizeof(double) * K * K);
    double *Vi = (double *)malloc(sizeof(double) * K * K);
    int rc = or_eig_sym(K, Q, pi, lam, V, Vi);
    or_expm_eig(K, lam, V, Vi, tau, P);
    free(lam);
    free(V);
    free(Vi);
    return rc < 0 ? -1 : 0;
  }
  or_expm_unif(K, Q, tau, P);
  return 0;
}

int or_frechet(int K, const double *X, const double *Y, double *L) {
  expm_frechet(K, X, Y, L);
  return 0;
}
