/*
 * epoch_oracle.h -- interface of the FP64 CPU oracle (test infrastructure
 * only; see epoch_oracle.c).  Not part of the product library.
 */
#ifndef EPOCH_ORACLE_H
#define EPOCH_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* One likelihood problem.  All arrays row-major, host memory, FP64.      */
typedef struct {
  int K;                       /* states                                   */
  int n_epochs;                /* E                                        */
  const double *boundaries;    /* [E-1] heights, strictly increasing       */
  const int *epoch_to_matrix;  /* [E] phi, or NULL = identity              */
  int n_matrices;              /* S                                        */
  const double *Q;             /* [S][K][K] rate matrices (rows sum to 0)  */
  const double *pi;            /* [K] stationary / root frequencies        */
  int normalise;               /* 1: scale each Q_s to sum_i pi_i q_ii=-1  */
  int reversible;              /* 1: eigen path, 0: uniformisation         */
  int n_categories;            /* C                                        */
  const double *cat_rates;     /* [C]                                      */
  const double *cat_weights;   /* [C]                                      */
  int n_taxa;                  /* N; nodes 0..N-1 are the tips             */
  const double *heights;       /* [2N-1]                                   */
  const int *parent;           /* [2N-1], root = -1                        */
  const double *branch_rates;  /* [2N-1] or NULL (= 1)                     */
  int n_patterns;              /* P                                        */
  const int *tips;             /* [N][P] codes: 0..K-1, K missing, K+1+m mask m */
  const double *pattern_weights; /* [P]                                    */
  int n_masks;                 /* ambiguity masks (K <= 64)                */
  const unsigned long long *masks; /* [n_masks] bit j = state j allowed    */
  int n_params;                /* model parameters theta                    */
  const double *dQ;            /* [n_params][S][K][K] d Q_raw / d theta     */
  int scaling;                 /* 1: rescale every internal node           */
} or_problem;

double or_normalise(int K, const double *Qraw, const double *pi, double *Qout);
int or_eig_sym(int K, const double *Q, const double *pi, double *lam, double *V,
               double *Vinv);
void or_expm_eig(int K, const double *lam, const double *V, const double *Vinv,
                 double tau, double *P);
void or_expm_unif(int K, const double *Q, double tau, double *P);
int or_expm(int K, const double *Q, const double *pi, int reversible, double tau,
            double *P);
int or_frechet(int K, const double *X, const double *Y, double *L);
int or_segments(int E, const double *b, double h_lo, double h_hi, int parent,
                int child, int maxseg, int *seg_epoch, double *seg_dt, int *hi_ref,
                int *lo_ref);
int or_branch_matrix(const or_problem *pr, int node, int cat, double *P);
double or_log_likelihood(const or_problem *pr, double *site_lnl);
double or_brute_force(const or_problem *pr, double *site_lnl);
int or_branch_adjoints(const or_problem *pr, double *G, double *lnl);
int or_gradient(const or_problem *pr, double *lnl, double *d_heights,
                double *d_boundaries, double *d_params, double *d_rates);
int or_expected_counts(const or_problem *pr, double *per_branch, double *per_epoch);
int or_ancestral(const or_problem *pr, double *out);
int or_ancestral_brute(const or_problem *pr, double *out);

#ifdef __cplusplus
}
#endif
#endif
