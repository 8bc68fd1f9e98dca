// k_model.cu -- branch segmentation, rate-matrix normalisation and
// eigendecomposition, parameter-derivative transforms and the FP64 branch
// transition matrices (time-ordered products of segment exponentials).
//
// Paper: Methods (Eq. makeprobs and the normalisation sum_i pi_i q_ii = -1),
// "Relaxing time-homogeneity" (branch segmentation, Eq. matrixProduct,
// Eq. convolution) and Appendix A (eigen-decomposition reuse).
#include <math.h>

#include <utility>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

// ---------------------------------------------------------------------------
// Segmentation: one thread per node v (the branch above v).  Segments are
// written parent end first into a fixed stride of E slots: a branch crosses
// at most E-1 boundaries.  A segment belongs to the epoch of its lower end;
// refs name what bounds it (node id >= 0, boundary j as -(j+1)).
// ---------------------------------------------------------------------------
__global__ void k_segments(Dims d, const double *__restrict__ heights,
                           const int *__restrict__ parent,
                           const double *__restrict__ b, const int *__restrict__ phi,
                           int *__restrict__ nseg, int *__restrict__ seg_mat,
                           double *__restrict__ seg_dt, int *__restrict__ seg_hi,
                           int *__restrict__ seg_lo) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.nn) return;
  int u = parent[v];
  if (u < 0) {
    nseg[v] = 0;
    return;
  }
  const int E = d.E;
  double lo = heights[v], hi = heights[u];
  int base = v * E;
  int n = 0;
  if (hi == lo) {
    int e = 0;
    for (int j = 0; j < E - 1; j++) e += (b[j] <= lo);
    seg_mat[base] = phi[e];
    seg_dt[base] = 0.0;
    seg_hi[base] = u;
    seg_lo[base] = v;
    nseg[v] = 1;
    return;
  }
  double top = hi;
  int top_ref = u;
  for (int j = E - 2; j >= 0; j--) {
    double bj = b[j];
    if (bj > lo && bj < hi) {
      // the piece above b_j lies in epoch j+1 (boundaries strictly increase)
      seg_mat[base + n] = phi[j + 1];
      seg_dt[base + n] = top - bj;
      seg_hi[base + n] = top_ref;
      seg_lo[base + n] = -(j + 1);
      n++;
      top = bj;
      top_ref = -(j + 1);
    }
  }
  int e = 0;
  for (int j = 0; j < E - 1; j++) e += (b[j] <= lo);
  seg_mat[base + n] = phi[e];
  seg_dt[base + n] = top - lo;
  seg_hi[base + n] = top_ref;
  seg_lo[base + n] = v;
  nseg[v] = n + 1;
}

// ---------------------------------------------------------------------------
// Block-wide FP64 sum (all threads get the result).
// ---------------------------------------------------------------------------
__device__ double block_sum(double x, double *red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  double t = 0.0;
  int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; i++) t += red[i];
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
// Normalise each Q_s and, for reversible models, diagonalise the symmetric
// S = Pi^{1/2} Q Pi^{-1/2}: Q = V diag(lambda) V^{-1}, V = Pi^{-1/2} U,
// V^{-1} = U^T Pi^{1/2}.  One CTA per matrix.
//
// Each FP64 instruction of a warp costs tens of cycles on this part whatever
// its active lanes, so the rotations are found in FP32 and only polished in
// FP64:
//   1. parallel cyclic Jacobi in FP32 (round-robin pairing: the n/2 rotations
//      of a round act on disjoint index pairs and are applied together as
//      J^T A J) until the off-diagonal part is below 1e-6 of the matrix;
//   2. U = the FP32 rotations in FP64, made orthogonal to FP64 rounding by
//      two Newton-Schulz steps U <- U (3 I - U^T U) / 2;
//   3. A' = U^T S U in FP64 (off-diagonal ~1e-7), then exact FP64 Jacobi
//      sweeps on A' (quadratic convergence: two sweeps to 1e-16), U <- U J.
// ---------------------------------------------------------------------------
// FP64: the exact angle (the annihilated entry is then set to zero).  In
// the polishing sweeps the pivot is tiny against the diagonal gap, so
// t = tan(angle) = r (1 - r^2 + 2 r^4) with r = a_pq / (a_qq - a_pp) and
// c = 1 - t^2 / 2 + 3 t^4 / 8 hold to rounding for |r| < 1e-5 and need no
// square root (each FP64 instruction is expensive here).
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double &c,
                                                double &s) {
  const double gap = aqq - app;
  if (fabs(apq) < 1e-5 * fabs(gap)) {
    const double r = apq / gap, r2 = r * r;
    const double t = r * (1.0 - r2 * (1.0 - 2.0 * r2));
    const double t2 = t * t;
    c = 1.0 - t2 * (0.5 - 0.375 * t2);
    s = t * c;
    return;
  }
  const double theta = gap / (2.0 * apq);
  double t;
  if (fabs(theta) > 1e18)
    t = 0.5 / theta;
  else
    t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
  c = 1.0 / sqrt(t * t + 1.0);
  s = t * c;
}
// FP32: an angle to ~1e-6 is enough (the FP64 stage finishes the job), so
// the fast reciprocal and square-root instructions do.
__device__ __forceinline__ void jacobi_rotation(float app, float aqq, float apq, float &c,
                                                float &s) {
  const float theta = __fdividef(aqq - app, 2.f * apq);
  float t;
  if (fabsf(theta) > 1e18f) {
    t = __fdividef(0.5f, theta);
  } else {
    const float h = theta * theta + 1.f;
    t = copysignf(__fdividef(1.f, fabsf(theta) + h * rsqrtf(h)), theta);
  }
  c = rsqrtf(t * t + 1.f);
  s = t * c;
}

// Cyclic Jacobi sweeps on the K x K symmetric A (row-major, shared memory),
// rotations accumulated into U (U <- U J).  Stops when the squared
// off-diagonal norm is <= tol2 (absolute), after max_sweeps, or when a sweep
// no longer halves it: convergence is quadratic until the rounding floor of
// T, where further sweeps only reshuffle rounding errors (that floor grows
// with K and can lie above tol2).  Returns the last measured value.
template <typename T, int KT>
__device__ __forceinline__ double jacobi_sweeps(T *A, T *U, int Kr, double tol2, int max_sweeps,
                                                double *red, T *cs, T *sn, int *pq) {
  const int K = KT ? KT : Kr;
  const int KK = K * K, tid = threadIdx.x, nt = blockDim.x;
  const int n = K + (K & 1), npair = n / 2;
  double off = 0.0, prev = 0.0;
  for (int sweep = 0;; sweep++) {
    double part = 0.0;
    for (int idx = tid; idx < KK; idx += nt) {
      const int i = idx / K, j = idx % K;
      if (j > i) part += (double)A[idx] * (double)A[idx];
    }
    off = block_sum(part, red);
    if (off <= tol2 || sweep == max_sweeps || (sweep > 0 && off > 0.5 * prev)) break;
    prev = off;
    const int nw = nt >> 5, w = tid >> 5, lane = tid & 31;
    for (int round = 0; round < n - 1; round++) {
      for (int k = tid; k < npair; k += nt) {
        // round-robin position after `round` shifts: element 0 stays, the
        // others move one place per round
        auto pos = [&](int i) {
          const int m = i - 1 - round;  // in (-(n - 1), n - 1)
          return i == 0 ? 0 : 1 + (m < 0 ? m + n - 1 : m);
        };
        const int a = pos(k), b = pos(n - 1 - k);
        const int p = a < b ? a : b, q = a < b ? b : a;
        T c = T(1), s = T(0);
        if (q < K && A[p * K + q] != T(0))
          jacobi_rotation(A[p * K + p], A[q * K + q], A[p * K + q], c, s);
        cs[k] = c;
        sn[k] = s;
        pq[2 * k] = p;
        pq[2 * k + 1] = q;
      }
      __syncthreads();
      if (K < 16) {  // few columns: threads over (pair, column)
        for (int idx = tid; idx < npair * K; idx += nt) {  // rows: B = J^T A
          const int k = idx / K, col = idx % K, p = pq[2 * k], q = pq[2 * k + 1];
          if (q >= K || sn[k] == T(0)) continue;
          const T ap = A[p * K + col], aq = A[q * K + col];
          A[p * K + col] = cs[k] * ap - sn[k] * aq;
          A[q * K + col] = sn[k] * ap + cs[k] * aq;
        }
        __syncthreads();
        for (int idx = tid; idx < npair * K; idx += nt) {  // columns: A' = B J, U' = U J
          const int k = idx / K, row = idx % K, p = pq[2 * k], q = pq[2 * k + 1];
          if (q >= K || sn[k] == T(0)) continue;
          const T ap = A[row * K + p], aq = A[row * K + q];
          A[row * K + p] = cs[k] * ap - sn[k] * aq;
          A[row * K + q] = sn[k] * ap + cs[k] * aq;
          const T up = U[row * K + p], uq = U[row * K + q];
          U[row * K + p] = cs[k] * up - sn[k] * uq;
          U[row * K + q] = sn[k] * up + cs[k] * uq;
        }
        __syncthreads();
      } else {
        // a warp per pair (warp-uniform skip), lanes along the row or column
        for (int k = w; k < npair; k += nw) {  // rows: B = J^T A
          const int p = pq[2 * k], q = pq[2 * k + 1];
          const T ck = cs[k], sk = sn[k];
          if (q >= K || sk == T(0)) continue;
          for (int col = lane; col < K; col += 32) {
            const T ap = A[p * K + col], aq = A[q * K + col];
            A[p * K + col] = ck * ap - sk * aq;
            A[q * K + col] = sk * ap + ck * aq;
          }
        }
        __syncthreads();
        for (int k = w; k < npair; k += nw) {  // columns: A' = B J, U' = U J
          const int p = pq[2 * k], q = pq[2 * k + 1];
          const T ck = cs[k], sk = sn[k];
          if (q >= K || sk == T(0)) continue;
          for (int row = lane; row < K; row += 32) {
            const T ap = A[row * K + p], aq = A[row * K + q];
            A[row * K + p] = ck * ap - sk * aq;
            A[row * K + q] = sk * ap + ck * aq;
            const T up = U[row * K + p], uq = U[row * K + q];
            U[row * K + p] = ck * up - sk * uq;
            U[row * K + q] = sk * up + ck * uq;
          }
        }
        __syncthreads();
      }
      for (int k = tid; k < npair; k += nt) {  // the annihilated pair
        const int p = pq[2 * k], q = pq[2 * k + 1];
        if (q < K && sn[k] != T(0)) {
          A[p * K + q] = T(0);
          A[q * K + p] = T(0);
        }
      }
      __syncthreads();
    }
  }
  return off;
}

// Cyclic Jacobi on a symmetric K x K FP32 matrix (K <= NR) held in registers
// by one thread as an NR x NR array, zero outside K x K (every index is a
// compile-time constant): sweeps over the pairs (p, q), p < q, in row order
// until the squared off-diagonal norm is <= tol2 or no longer halves (at most
// 12 sweeps).  Pairs that reach into the zero padding have a_pq = 0 and are
// skipped, so the padding stays zero.  A and U: row-major K x K in shared memory, U = I on
// entry; A is overwritten by the rotated matrix, U by the rotations.
template <int NR>
__device__ __forceinline__ void rot_registers(float (&a)[NR][NR], float (&u)[NR][NR], int p, int q) {
  const float apq = a[p][q];
  if (apq == 0.f) return;
  float c, s;
  jacobi_rotation(a[p][p], a[q][q], apq, c, s);
#pragma unroll
  for (int k = 0; k < NR; k++) {  // rows p, q
    const float x = a[p][k], y = a[q][k];
    a[p][k] = c * x - s * y;
    a[q][k] = s * x + c * y;
  }
#pragma unroll
  for (int k = 0; k < NR; k++) {  // columns p, q
    const float x = a[k][p], y = a[k][q];
    a[k][p] = c * x - s * y;
    a[k][q] = s * x + c * y;
    const float ux = u[k][p], uy = u[k][q];
    u[k][p] = c * ux - s * uy;
    u[k][q] = s * ux + c * uy;
  }
  a[p][q] = 0.f;
  a[q][p] = 0.f;
}
template <int NR>
__device__ void jacobi_registers(float *A, float *U, int K, float tol2) {
  float a[NR][NR], u[NR][NR];
#pragma unroll
  for (int i = 0; i < NR; i++)
#pragma unroll
    for (int j = 0; j < NR; j++) {
      a[i][j] = (i < K && j < K) ? A[i * K + j] : 0.f;
      u[i][j] = (i == j) ? 1.f : 0.f;
    }
  float prev = 0.f;
  for (int sweep = 0; sweep < 12; sweep++) {
    float off = 0.f;
#pragma unroll
    for (int p = 0; p < NR; p++)
#pragma unroll
      for (int q = p + 1; q < NR; q++) off += a[p][q] * a[p][q];
    // converged, or at the FP32 rounding floor (a sweep no longer halves it)
    if (off <= tol2 || (sweep > 0 && off > 0.5f * prev)) break;
    prev = off;
#pragma unroll
    for (int p = 0; p < NR; p++)
#pragma unroll
      for (int q = p + 1; q < NR; q++) rot_registers<NR>(a, u, p, q);
  }
#pragma unroll
  for (int i = 0; i < NR; i++)
#pragma unroll
    for (int j = 0; j < NR; j++)
      if (i < K && j < K) {
        A[i * K + j] = a[i][j];
        U[i * K + j] = u[i][j];
      }
}

// C = op(X) Y for K x K row-major FP64 matrices in shared memory (op = X^T
// when tx); every thread forms whole entries of C.
template <int KT>
__device__ __forceinline__ void mm_shared(const double *X, const double *Y, double *C, int Kr,
                                          bool tx) {
  const int K = KT ? KT : Kr;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int i = idx / K, j = idx % K;
    double acc = 0.0;
    for (int m = 0; m < K; m++) acc += (tx ? X[m * K + i] : X[i * K + m]) * Y[m * K + j];
    C[idx] = acc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// FP64 refinement of the eigenvectors for large K (Ogita and Aishima 2018,
// "Iterative refinement for symmetric eigenvalue decomposition"), restated:
// with X the current eigenvector estimate of the symmetric S,
//     R = I - X^T X,  T = X^T S X,  lambda_i = t_ii / (1 - r_ii),
//     delta = 2 (||T - diag(lambda)|| + ||S|| ||R||)   (Frobenius bounds),
//     E_ij = (t_ij + lambda_j r_ij) / (lambda_j - lambda_i)  if
//            |lambda_i - lambda_j| > delta, else r_ij / 2  (E_ii = r_ii / 2),
//     X <- X + X E,
// which solves X^T X = I and X^T S X diagonal to first order, so the error
// squares each step.  Its products are spread over many CTAs, where the
// Jacobi sweeps they replace ran on one SM per matrix at the part's FP64
// rate.  A pair closer than delta (an eigenvalue cluster) is only
// orthogonalised; k_eig_finish then rotates such pairs exactly.
// ---------------------------------------------------------------------------
// The refinement's update runs as row blocks of kEigRows rows, one CTA each
// (at most kEigRowBlocks for K <= EPOCH_MAX_STATES).
constexpr int kEigRows = 4, kEigRowBlocks = (EPOCH_MAX_STATES + kEigRows - 1) / kEigRows;
struct EigLayout {  // offsets in doubles within one matrix's block
  int A, X0, X1, T1, T2, T3, E, lam, rs, fro2, cluster, stride;
  __host__ __device__ explicit EigLayout(int K) {
    const int KK = K * K;
    A = 0;
    X0 = KK;
    X1 = 2 * KK;
    T1 = 3 * KK;
    T2 = 4 * KK;
    T3 = 5 * KK;
    E = 6 * KK;
    lam = 7 * KK;
    rs = lam + K;
    fro2 = rs + K;
    cluster = fro2 + 1;  // per row block of the update: 1 when the last step
                         // left a pair closer than delta
    stride = cluster + kEigRowBlocks;
  }
};

// C = op(A) B (+ D) for the K x K matrices of every block; several products
// per launch (blockIdx.z = matrix * n + product).  A 16 x 16 tile of C per
// CTA, its rows of op(A) and columns of B staged in shared memory.  Offsets:
// -1 = no D.  No output may alias an input of the same launch.  comp = 1:
// each dot product is accumulated as an unevaluated sum s + c of FP64 values
// with the exact rounding errors of every product (fma) and every addition
// (Knuth's two-sum) collected in c (Ogita, Rump and Oishi 2005, "Dot2"):
// as accurate as a dot product in twice the working precision, rounded once.
struct EigProd {
  int a, b, c, add, ta, comp;  // comp: compensated dot products
};
struct EigProds {
  EigProd p[2];
  int n;
};
__global__ void __launch_bounds__(256) k_eig_gemm(int K, double *__restrict__ base, int stride,
                                                  EigProds pr) {
  __shared__ double As[16][65];
  __shared__ double Bs[64][17];
  const int s = blockIdx.z / pr.n;
  const EigProd q = pr.p[blockIdx.z % pr.n];
  double *M = base + (size_t)s * stride;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16, tid = threadIdx.x;
  for (int idx = tid; idx < 16 * K; idx += 256) {
    const int r = idx / K, k = idx % K, i = i0 + r;
    As[r][k] = i < K ? (q.ta ? M[q.a + k * K + i] : M[q.a + i * K + k]) : 0.0;
  }
  for (int idx = tid; idx < 16 * K; idx += 256) {
    const int k = idx / 16, cc = idx % 16, j = j0 + cc;
    Bs[k][cc] = j < K ? M[q.b + k * K + j] : 0.0;
  }
  __syncthreads();
  const int r = tid / 16, cc = tid % 16, i = i0 + r, j = j0 + cc;
  if (i < K && j < K) {
    double acc = q.add >= 0 ? M[q.add + i * K + j] : 0.0;
    if (q.comp) {
      double c = 0.0;
      for (int k = 0; k < K; k++) {
        const double a = As[r][k], b = Bs[k][cc];
        const double p = a * b, e = fma(a, b, -p);  // a b = p + e exactly
        const double t = acc + p, z = t - acc;        // acc + p = t + (err) exactly
        c += ((acc - (t - z)) + (p - z)) + e;
        acc = t;
      }
      acc += c;
    } else {
      for (int k = 0; k < K; k++) acc = fma(As[r][k], Bs[k][cc], acc);
    }
    M[q.c + i * K + j] = acc;
  }
}

// One refinement step's E and lambda from T1 = X^T X and T3 = X^T S X; grid
// (row blocks, matrices): every CTA forms lambda and the two norms of delta
// (the same values, in the same order) and then the E entries of its rows,
// whose FP64 divisions dominated when one CTA did all rows.
__global__ void __launch_bounds__(256) k_eig_update(int K, double *__restrict__ base, int stride) {
  __shared__ double red[32];
  const EigLayout L(K);
  double *M = base + (size_t)blockIdx.y * stride;
  const int r0 = blockIdx.x * kEigRows, r1 = min(K, r0 + kEigRows);
  const double *T1 = M + L.T1, *T3 = M + L.T3;
  double *E = M + L.E;
  __shared__ double lam[EPOCH_MAX_STATES];  // every CTA forms them; row block 0 stores them
  const int KK = K * K, tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < K; i += nt) {
    lam[i] = T3[i * K + i] / T1[i * K + i];  // 1 - r_ii = t1_ii
    if (blockIdx.x == 0) M[L.lam + i] = lam[i];
  }
  __syncthreads();
  double po = 0.0, pr = 0.0;
  for (int idx = tid; idx < KK; idx += nt) {
    const int i = idx / K, j = idx % K;
    const double t = T3[idx] - (i == j ? lam[i] : 0.0);
    const double r = (i == j ? 1.0 : 0.0) - T1[idx];
    po += t * t;
    pr += r * r;
  }
  const double off = block_sum(po, red);
  const double rr = block_sum(pr, red);
  const double delta = 2.0 * (sqrt(off) + sqrt(M[L.fro2]) * sqrt(rr));
  int close = 0;
  for (int idx = r0 * K + tid; idx < r1 * K; idx += nt) {
    const int i = idx / K, j = idx % K;
    const double r = (i == j ? 1.0 : 0.0) - T1[idx];
    double e = 0.5 * r;
    if (i != j) {
      if (fabs(lam[i] - lam[j]) > delta)
        e = (T3[idx] + lam[j] * r) / (lam[j] - lam[i]);
      else
        close = 1;
    }
    E[idx] = e;
  }
  close = __syncthreads_or(close);
  if (tid == 0) M[L.cluster + blockIdx.x] = close ? 1.0 : 0.0;
}

// After the refinement: lambda from the last step (its Rayleigh quotients,
// formed with compensated products from an X already accurate to ~1e-14,
// are accurate to rounding) and the updated X give lambda, V = Pi^{-1/2} X
// and V^{-1} = X^T Pi^{1/2}.  When the last step left a pair closer than
// delta (an eigenvalue cluster, only orthogonalised), T = X^T S X is formed
// here and exact FP64 Jacobi sweeps rotate the pair out.  One 512-thread CTA
// per matrix.
__global__ void __launch_bounds__(512) k_eig_finish(int K, const double *__restrict__ base, int stride,
                                                    int xoff, double *__restrict__ lam,
                                                    double *__restrict__ V,
                                                    double *__restrict__ Vinv, int *status) {
  extern __shared__ double sm[];
  const int KK = K * K, tid = threadIdx.x, nt = blockDim.x, s = blockIdx.x;
  const EigLayout L(K);
  const double *M = base + (size_t)s * stride;
  double *A = sm, *U = A + KK, *T = U + KK, *red = T + KK, *cs = red + 32, *sn = cs + 32;
  int *pq = (int *)(sn + 32);
  for (int idx = tid; idx < KK; idx += nt) U[idx] = M[xoff + idx];
  bool cluster = false;
  for (int b = 0; b < (K + kEigRows - 1) / kEigRows; b++) cluster |= M[L.cluster + b] != 0.0;
  if (cluster) {
    for (int idx = tid; idx < KK; idx += nt) T[idx] = M[L.A + idx];
    __syncthreads();
    mm_shared<0>(T, U, A, K, false);  // A = S X
    mm_shared<0>(U, A, T, K, true);   // T = X^T S X
    for (int idx = tid; idx < KK; idx += nt) {
      const int i = idx / K, j = idx % K;
      A[idx] = 0.5 * (T[idx] + T[j * K + i]);
    }
    __syncthreads();
    const double fro2 = M[L.fro2];
    const double off = jacobi_sweeps<double, 0>(A, U, K, 1e-32 * fro2, 30, red, cs, sn, pq);
    if (off > 1e-24 * fro2 && tid == 0) atomicOr(status, ST_EIG_NOCONV);
    for (int i = tid; i < K; i += nt) lam[(size_t)s * K + i] = A[i * K + i];
  } else {
    for (int i = tid; i < K; i += nt) lam[(size_t)s * K + i] = M[L.lam + i];
  }
  __syncthreads();
  const double *rs = M + L.rs;
  for (int idx = tid; idx < KK; idx += nt) {
    const int i = idx / K, j = idx % K;
    V[(size_t)s * KK + idx] = U[idx] / rs[i];
    Vinv[(size_t)s * KK + idx] = U[j * K + i] * rs[j];
  }
}

// KT: K known at compile time (0 = take d.K).  RJ: FP32 rotations in one
// thread's registers for K <= RJ (4 or 8; one warp per matrix), or 0: shared-
// memory sweeps by a 512-thread CTA.
// refine != NULL (large K): stop after the FP32 rotations and hand S, the
// rotations U (in FP64), sqrt(pi) and ||S||_F^2 to the refinement kernels
// below, in the matrix's block of `refine` (layout: EigLayout).
template <int KT, int RJ>
__global__ void __launch_bounds__(RJ ? 32 : 512) k_model_setup(Dims d, int normalise, const double *__restrict__ Qraw,
                              const double *__restrict__ pi, double *__restrict__ Qn,
                              double *__restrict__ cnorm, double *__restrict__ lam,
                              double *__restrict__ V, double *__restrict__ Vinv,
                              int *__restrict__ status, double *__restrict__ refine) {
  extern __shared__ double sm[];
  const int K = KT ? KT : d.K, KK = K * K;
  const int s = blockIdx.x;
  double *A = sm;            // K*K  S, then U^T S U
  double *U = A + KK;        // K*K  eigenvectors
  double *T1 = U + KK;       // K*K  work
  double *T2 = T1 + KK;      // K*K  work
  double *rs = T2 + KK;      // K    sqrt(pi)
  double *red = rs + K;      // 32
  double *cs = red + 32;     // 32 rotation cosines
  double *sn = cs + 32;      // 32 rotation sines
  int *pq = (int *)(sn + 32);                // 64 pair indices
  float *A32 = (float *)(pq + 64);           // K*K
  float *U32 = A32 + KK;                     // K*K
  float *cs32 = U32 + KK, *sn32 = cs32 + 32;  // 32 + 32
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int i = tid; i < KK; i += nt) A[i] = Qraw[(size_t)s * KK + i];
  for (int i = tid; i < K; i += nt) rs[i] = sqrt(pi[i]);
  __syncthreads();
  double part = 0.0;
  for (int i = tid; i < K; i += nt) part -= pi[i] * A[i * K + i];
  double c = block_sum(part, red);
  double scale = normalise ? c : 1.0;
  if (!(scale > 0.0)) scale = 1.0;  // rejected on the host already
  const double inv_scale = 1.0 / scale;
  for (int i = tid; i < KK; i += nt) {
    A[i] *= inv_scale;
    Qn[(size_t)s * KK + i] = A[i];
  }
  if (tid == 0) cnorm[s] = scale;
  if (!d.reversible) return;
  __syncthreads();
  // symmetric form S = (Pi^1/2 Q Pi^-1/2 + its transpose) / 2
  for (int idx = tid; idx < KK; idx += nt) {
    const int i = idx / K, j = idx % K;
    T1[idx] = rs[i] * A[idx] / rs[j];
  }
  __syncthreads();
  part = 0.0;
  for (int idx = tid; idx < KK; idx += nt) {
    const int i = idx / K, j = idx % K;
    A[idx] = 0.5 * (T1[i * K + j] + T1[j * K + i]);
    A32[idx] = (float)A[idx];
    U32[idx] = (i == j) ? 1.f : 0.f;
    part += A[idx] * A[idx];
  }
  const double fro2 = block_sum(part, red);
  // 1. FP32 rotations (K <= RJ: one thread, the matrix in registers)
  if constexpr (RJ > 0) {
    __syncthreads();
    if (tid == 0) jacobi_registers<RJ>(A32, U32, K, (float)(1e-12 * fro2));
    __syncthreads();
  } else {
    jacobi_sweeps<float, KT>(A32, U32, K, 1e-12 * fro2, 40, red, cs32, sn32, pq);
  }
  if (refine) {  // the FP64 stage runs as the refinement kernels
    const EigLayout L(K);
    double *blk = refine + (size_t)s * L.stride;
    for (int idx = tid; idx < KK; idx += nt) {
      blk[L.A + idx] = A[idx];
      blk[L.X0 + idx] = (double)U32[idx];
    }
    for (int i = tid; i < K; i += nt) blk[L.rs + i] = rs[i];
    if (tid == 0) blk[L.fro2] = fro2;
    return;
  }
  // 2. orthogonal U in FP64
  for (int idx = tid; idx < KK; idx += nt) U[idx] = (double)U32[idx];
  __syncthreads();
  for (int it = 0; it < 2; it++) {
    mm_shared<KT>(U, U, T1, K, true);  // T1 = U^T U
    for (int idx = tid; idx < KK; idx += nt) {
      const int i = idx / K, j = idx % K;
      T1[idx] = ((i == j) ? 1.5 : 0.0) - 0.5 * T1[idx];
    }
    __syncthreads();
    mm_shared<KT>(U, T1, T2, K, false);  // T2 = U (3 I - U^T U) / 2
    for (int idx = tid; idx < KK; idx += nt) U[idx] = T2[idx];
    __syncthreads();
  }
  // 3. A' = U^T S U, symmetrised, then exact FP64 sweeps
  mm_shared<KT>(A, U, T1, K, false);   // T1 = S U
  mm_shared<KT>(U, T1, T2, K, true);   // T2 = U^T S U
  for (int idx = tid; idx < KK; idx += nt) {
    const int i = idx / K, j = idx % K;
    A[idx] = 0.5 * (T2[i * K + j] + T2[j * K + i]);
  }
  __syncthreads();
  const double off = jacobi_sweeps<double, KT>(A, U, K, 1e-32 * fro2, 30, red, cs, sn, pq);
  if (off > 1e-24 * fro2 && tid == 0) atomicOr(status, ST_EIG_NOCONV);
  for (int i = tid; i < K; i += nt) lam[(size_t)s * K + i] = A[i * K + i];
  for (int idx = tid; idx < KK; idx += nt) {
    const int i = idx / K, j = idx % K;
    V[(size_t)s * KK + idx] = U[idx] / rs[i];
    Vinv[(size_t)s * KK + idx] = U[j * K + i] * rs[j];
  }
}

// ---------------------------------------------------------------------------
// Parameter derivatives in the eigenbasis: D_{a,s} = V_s^{-1} dQ_eff V_s with
// dQ_eff = (dQraw - Q_s dc) / c the derivative of the normalised matrix
// (c = -sum_i pi_i qraw_ii, dc its derivative).  One CTA per (a, s), FP64.
// ---------------------------------------------------------------------------
__global__ void k_param_transform(Dims d, int normalise, const double *__restrict__ dQraw,
                                  const double *__restrict__ pi,
                                  const double *__restrict__ Qn,
                                  const double *__restrict__ cnorm,
                                  const double *__restrict__ V,
                                  const double *__restrict__ Vinv,
                                  double *__restrict__ D, float *__restrict__ D32,
                                  int *__restrict__ Dnz) {
  extern __shared__ double sm[];
  const int K = d.K, KK = d.KK;
  const int a = blockIdx.x, s = blockIdx.y;
  double *X = sm, *T = sm + KK, *red = sm + 2 * KK;
  const double *dq = dQraw + ((size_t)a * d.S + s) * KK;
  const int tid = threadIdx.x, nt = blockDim.x;
  double part = 0.0;
  int nz = 0;
  for (int i = tid; i < KK; i += nt) nz |= (dq[i] != 0.0);
  for (int i = tid; i < K; i += nt) part -= pi[i] * dq[i * K + i];
  double dc = block_sum(part, red);
  nz = __syncthreads_or(nz);
  double c = cnorm[s];
  for (int i = tid; i < KK; i += nt)
    X[i] = normalise ? (dq[i] - Qn[(size_t)s * KK + i] * dc) / c : dq[i];
  __syncthreads();
  const double *Vs = V + (size_t)s * KK, *Vi = Vinv + (size_t)s * KK;
  for (int idx = tid; idx < KK; idx += nt) {  // T = X V
    int i = idx / K, j = idx % K;
    double acc = 0.0;
    for (int k = 0; k < K; k++) acc += X[i * K + k] * Vs[k * K + j];
    T[idx] = acc;
  }
  __syncthreads();
  double *out = D + ((size_t)a * d.S + s) * KK;
  float *out32 = D32 + ((size_t)a * d.S + s) * KK;
  for (int idx = tid; idx < KK; idx += nt) {  // D = V^-1 T
    int i = idx / K, j = idx % K;
    double acc = 0.0;
    for (int k = 0; k < K; k++) acc += Vi[i * K + k] * T[k * K + j];
    out[idx] = acc;
    out32[idx] = (float)acc;
  }
  if (tid == 0) Dnz[a * d.S + s] = nz;
}

// ---------------------------------------------------------------------------
// Branch transition matrices, FP64.  One CTA per (branch v, category c):
// M = I; for each segment from the parent end, M <- M * exp(r rho dt Q_s)
// (Eq. convolution).  Reversible: exp via the eigensystem,
// E = V diag(exp(tau lambda)) V^{-1}.  General Q: uniformisation,
// M <- sum_m Pois(m; mu tau) M B^m, B = I + Q/mu, in pieces of mu*tau <= 30.
// Writes P64[v][c] and, for the FP32 paths, the transposed table
// PT32[v][c][j][i] = P[i][j] with rows K (missing: row sums) and
// K+1+m (ambiguity mask m) appended.
// ---------------------------------------------------------------------------
__global__ void k_branch_matrices(Dims d, const int *__restrict__ nseg,
                                  const int *__restrict__ seg_mat,
                                  const double *__restrict__ seg_dt,
                                  const double *__restrict__ brate,
                                  const double *__restrict__ catr,
                                  const double *__restrict__ lam,
                                  const double *__restrict__ V,
                                  const double *__restrict__ Vinv,
                                  const double *__restrict__ Qn,
                                  const double *__restrict__ pi,
                                  const unsigned long long *__restrict__ masks,
                                  double *__restrict__ P64, float *__restrict__ PT32) {
  extern __shared__ double sm[];
  const int K = d.K, KK = d.KK;
  const int v = blockIdx.x, c = blockIdx.y;
  const int ns = nseg[v];
  if (ns == 0) return;  // root
  double *M = sm, *W = sm + KK, *Y = sm + 2 * KK, *B = sm + 3 * KK, *ev = sm + 4 * KK;
  double *rs = ev + K, *irs = rs + K;  // sqrt(pi_i) and its inverse
  const int tid = threadIdx.x, nt = blockDim.x;
  const double r = brate[v] * catr[c];
  for (int idx = tid; idx < KK; idx += nt) M[idx] = (idx / K == idx % K) ? 1.0 : 0.0;
  if (d.reversible)
    for (int i = tid; i < K; i += nt) {
      rs[i] = sqrt(pi[i]);
      irs[i] = 1.0 / rs[i];
    }
  __syncthreads();
  bool M_is_identity = true;
  for (int k = 0; k < ns; k++) {
    const int s = seg_mat[v * d.E + k];
    const double tau = r * seg_dt[v * d.E + k];
    if (tau == 0.0) continue;  // exp(0) = I exactly (zero-length branch)
    if (d.reversible) {
      // With D = diag(sqrt(pi)) the eigenvectors V = D^-1 U, V^-1 = U^T D
      // (U orthonormal, the symmetrised matrix's), so
      //   W = V diag(ev) V^-1 = D^-1 (U diag(ev) U^T) D
      // and the middle factor is symmetric: only its upper triangle is
      // formed (half the FP64 multiply-adds of the plain product).
      const double *Vs = V + (size_t)s * KK;
      for (int i = tid; i < K; i += nt) ev[i] = exp(tau * lam[(size_t)s * K + i]);
      __syncthreads();
      // U diag(ev) and U staged in shared memory (Y and B are free here)
      for (int idx = tid; idx < KK; idx += nt) {
        const double u = Vs[idx] * rs[idx / K];
        Y[idx] = u * ev[idx % K];
        B[idx] = u;
      }
      __syncthreads();
      // entry t of the upper triangle, row-major: row i holds K - i entries
      // starting at i K - i (i - 1) / 2.  Transition probabilities are >= 0,
      // so the rounding-level negatives of the eigen form are cut at 0
      // (keeps every partial likelihood >= 0).
      const int ntri = K * (K + 1) / 2;
      for (int t = tid; t < ntri; t += nt) {
        const float b2 = 2.f * K + 1.f;
        int i = (int)((b2 - sqrtf(b2 * b2 - 8.f * (float)t)) * 0.5f);
        i = i < 0 ? 0 : (i > K - 1 ? K - 1 : i);
        while (i > 0 && i * K - i * (i - 1) / 2 > t) i--;
        while (i + 1 < K && (i + 1) * K - (i + 1) * i / 2 <= t) i++;
        const int j = i + (t - (i * K - i * (i - 1) / 2));
        double acc = 0.0;
        for (int m = 0; m < K; m++) acc += Y[i * K + m] * B[j * K + m];
        W[i * K + j] = fmax(acc * rs[j] * irs[i], 0.0);
        if (j != i) W[j * K + i] = fmax(acc * rs[i] * irs[j], 0.0);
      }
      __syncthreads();
      if (k == 0 || M_is_identity) {
        for (int idx = tid; idx < KK; idx += nt) M[idx] = W[idx];
      } else {
        for (int idx = tid; idx < KK; idx += nt) {
          int i = idx / K, j = idx % K;
          double acc = 0.0;
          for (int m = 0; m < K; m++) acc += M[i * K + m] * W[m * K + j];
          Y[idx] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < KK; idx += nt) M[idx] = Y[idx];
      }
      M_is_identity = false;
      __syncthreads();
    } else {
      const double *Qs = Qn + (size_t)s * KK;
      double mu = 0.0;
      for (int i = 0; i < K; i++) mu = fmax(mu, fabs(Qs[i * K + i]));
      if (mu == 0.0 || tau == 0.0) continue;
      for (int idx = tid; idx < KK; idx += nt)
        B[idx] = Qs[idx] / mu + ((idx / K == idx % K) ? 1.0 : 0.0);
      const double mt = mu * tau;
      const int npc = (int)ceil(mt / 30.0);
      const double x = mt / npc;
      const int mmax = (int)ceil(x + 12.0 * sqrt(x) + 30.0);
      for (int piece = 0; piece < npc; piece++) {
        double w = exp(-x);
        __syncthreads();
        for (int idx = tid; idx < KK; idx += nt) {
          Y[idx] = M[idx];       // Y = M B^0
          W[idx] = w * M[idx];   // accumulator
        }
        __syncthreads();
        for (int m = 1; m <= mmax; m++) {
          w = w * x / (double)m;
          // Y <- Y B  (in place through M as scratch is unsafe: use ev-free temp)
          for (int idx = tid; idx < KK; idx += nt) {
            int i = idx / K, j = idx % K;
            double acc = 0.0;
            for (int q = 0; q < K; q++) acc += Y[i * K + q] * B[q * K + j];
            M[idx] = acc;
          }
          __syncthreads();
          for (int idx = tid; idx < KK; idx += nt) {
            Y[idx] = M[idx];
            W[idx] += w * M[idx];
          }
          __syncthreads();
        }
        for (int idx = tid; idx < KK; idx += nt) M[idx] = W[idx];
        __syncthreads();
      }
      M_is_identity = false;
    }
  }
  __syncthreads();
  double *out = P64 + ((size_t)v * d.C + c) * KK;
  for (int idx = tid; idx < KK; idx += nt) out[idx] = M[idx];
  if (PT32) {
    float *pt = PT32 + ((size_t)v * d.C + c) * d.NR * d.Kp;
    for (int idx = tid; idx < d.NR * d.Kp; idx += nt) {
      int row = idx / d.Kp, i = idx % d.Kp;
      double val = 0.0;
      if (i < K) {
        if (row < K) {
          val = M[i * K + row];
        } else {
          unsigned long long mk = (row == K) ? ~0ull : masks[row - K - 1];
          for (int j = 0; j < K; j++)
            if ((mk >> j) & 1ull) val += M[i * K + j];
        }
      }
      pt[idx] = (float)val;
    }
  }
}


// ---------------------------------------------------------------------------
// The same matrices for the FP32 paths of reversible models, in double-float
// arithmetic: a value is the unevaluated sum hi + lo of two floats (Dekker,
// 1971), products are formed exactly with an FMA and sums by Knuth's
// two-sum, which carries about 48 significant bits on the FP32 pipes.  FP32
// alone would not do: the eigen form adds terms up to 1 / sqrt(pi_i pi_j)
// whose sum can be far smaller; and every FP64 instruction, conversions
// included, runs at a small fraction of the FP32 rate on this part, so the
// FP64 inputs are split into float pairs once per matrix (k_df_prep) and the
// per-branch kernel does no FP64 arithmetic but the K exponentials of each
// segment and the P64 output.  The result (about 1e-13 of the terms' size)
// is written as P64 and as the FP32 table PT32, like k_branch_matrices.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 df_split(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
// (sh, sl) += a b; the intrinsics keep the compiler from fusing the
// error-free steps
__device__ __forceinline__ void df_mac(float2 a, float2 b, float &sh, float &sl) {
  const float ph = __fmul_rn(a.x, b.x);
  float pe = __fmaf_rn(a.x, b.x, -ph);  // a.x b.x - ph exactly
  pe = __fmaf_rn(a.x, b.y, pe);
  pe = __fmaf_rn(a.y, b.x, pe);
  const float s = __fadd_rn(sh, ph);
  const float z = __fsub_rn(s, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(ph, z));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, pe));
}
// (h, l) renormalised so that |l| <= ulp(h) / 2
__device__ __forceinline__ float2 df_norm(float h, float l) {
  const float s = __fadd_rn(h, l);
  return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float ph = __fmul_rn(a.x, b.x);
  float pe = __fmaf_rn(a.x, b.x, -ph);
  pe = __fmaf_rn(a.x, b.y, pe);
  pe = __fmaf_rn(a.y, b.x, pe);
  return df_norm(ph, pe);
}

// Per matrix s: U = D V (D = diag(sqrt(pi)), U orthonormal) and the
// diagonals of D and D^-1, as float pairs: out[s] = [U (K K) | D (K) | D^-1 (K)];
// and the eigensystem rounded to FP32 for the FP32 chain rule, laid out
// like the FP64 one: e32 = [V (S K K) | V^-1 (S K K) | lambda (S K)].
__global__ void k_df_prep(Dims d, const double *__restrict__ lam, const double *__restrict__ V,
                          const double *__restrict__ Vinv, const double *__restrict__ pi,
                          float2 *__restrict__ out, float *__restrict__ e32) {
  const int K = d.K, KK = d.KK, s = blockIdx.x;
  float2 *o = out + (size_t)s * (KK + 2 * K);
  float *fV = e32 + (size_t)s * KK, *fVi = e32 + (size_t)(d.S + s) * KK,
        *fl = e32 + (size_t)2 * d.S * KK + (size_t)s * K;
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
    const double vv = V[(size_t)s * KK + idx];
    o[idx] = df_split(vv * sqrt(pi[idx / K]));
    fV[idx] = (float)vv;
    fVi[idx] = (float)Vinv[(size_t)s * KK + idx];
  }
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double r = sqrt(pi[i]);
    o[KK + i] = df_split(r);
    o[KK + K + i] = df_split(1.0 / r);
    fl[i] = (float)lam[(size_t)s * K + i];
  }
}

__global__ void k_branch_matrices_df(Dims d, const int *__restrict__ nseg,
                                     const int *__restrict__ seg_mat,
                                     const double *__restrict__ seg_dt,
                                     const double *__restrict__ brate,
                                     const double *__restrict__ catr,
                                     const double *__restrict__ lam,
                                     const float2 *__restrict__ dfU,
                                     const unsigned long long *__restrict__ masks,
                                     double *__restrict__ P64, float *__restrict__ PT32) {
  extern __shared__ float2 smf[];
  const int K = d.K, KK = d.KK;
  const int v = blockIdx.x, c = blockIdx.y;
  const int ns = nseg[v];
  if (ns == 0) return;  // root
  float2 *M = smf, *W = M + KK, *Y = W + KK, *B = Y + KK, *ev = B + KK, *rs = ev + K,
         *irs = rs + K;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double r = brate[v] * catr[c];
  for (int idx = tid; idx < KK; idx += nt)
    M[idx] = make_float2((idx / K == idx % K) ? 1.f : 0.f, 0.f);
  bool M_is_identity = true;
  for (int k = 0; k < ns; k++) {
    const int s = seg_mat[v * d.E + k];
    const double tau = r * seg_dt[v * d.E + k];
    if (tau == 0.0) continue;  // exp(0) = I exactly (zero-length branch)
    const float2 *U = dfU + (size_t)s * (KK + 2 * K);
    for (int i = tid; i < K; i += nt) {
      ev[i] = df_split(exp(tau * lam[(size_t)s * K + i]));
      rs[i] = U[KK + i];
      irs[i] = U[KK + K + i];
    }
    __syncthreads();
    for (int idx = tid; idx < KK; idx += nt) {  // B = U, Y = U diag(ev)
      const float2 u = U[idx];
      B[idx] = u;
      Y[idx] = df_mul(u, ev[idx % K]);
    }
    __syncthreads();
    // W = D^-1 (U diag(ev) U^T) D from the upper triangle of the symmetric
    // middle factor (entry t: row i holds K - i entries from i K - i (i-1)/2);
    // negatives at rounding level are cut at 0
    const int ntri = K * (K + 1) / 2;
    for (int t = tid; t < ntri; t += nt) {
      const float b2 = 2.f * K + 1.f;
      int i = (int)((b2 - sqrtf(b2 * b2 - 8.f * (float)t)) * 0.5f);
      i = i < 0 ? 0 : (i > K - 1 ? K - 1 : i);
      while (i > 0 && i * K - i * (i - 1) / 2 > t) i--;
      while (i + 1 < K && (i + 1) * K - (i + 1) * i / 2 <= t) i++;
      const int j = i + (t - (i * K - i * (i - 1) / 2));
      float sh = 0.f, sl = 0.f;
      for (int m = 0; m < K; m++) df_mac(Y[i * K + m], B[j * K + m], sh, sl);
      const float2 a = df_norm(sh, sl);
      const float2 z = make_float2(0.f, 0.f);
      const float2 wij = df_mul(df_mul(a, rs[j]), irs[i]);
      W[i * K + j] = wij.x > 0.f ? wij : z;
      if (j != i) {
        const float2 wji = df_mul(df_mul(a, rs[i]), irs[j]);
        W[j * K + i] = wji.x > 0.f ? wji : z;
      }
    }
    __syncthreads();
    if (M_is_identity) {
      for (int idx = tid; idx < KK; idx += nt) M[idx] = W[idx];
    } else {  // M <- M W through Y (free again)
      for (int idx = tid; idx < KK; idx += nt) {
        const int i = idx / K, j = idx % K;
        float sh = 0.f, sl = 0.f;
        for (int m = 0; m < K; m++) df_mac(M[i * K + m], W[m * K + j], sh, sl);
        Y[idx] = df_norm(sh, sl);
      }
      __syncthreads();
      for (int idx = tid; idx < KK; idx += nt) M[idx] = Y[idx];
    }
    M_is_identity = false;
    __syncthreads();
  }
  double *out = P64 + ((size_t)v * d.C + c) * KK;
  for (int idx = tid; idx < KK; idx += nt) out[idx] = (double)M[idx].x + (double)M[idx].y;
  float *pt = PT32 + ((size_t)v * d.C + c) * d.NR * d.Kp;
  for (int idx = tid; idx < d.NR * d.Kp; idx += nt) {
    const int row = idx / d.Kp, i = idx % d.Kp;
    float val = 0.f;
    if (i < K) {
      if (row < K) {
        val = __fadd_rn(M[i * K + row].x, M[i * K + row].y);
      } else {  // row sums over a mask: in FP32, as the FP32 path adds them
        const unsigned long long mk = (row == K) ? ~0ull : masks[row - K - 1];
        float sh = 0.f, sl = 0.f;
        for (int j = 0; j < K; j++)
          if ((mk >> j) & 1ull) df_mac(M[i * K + j], make_float2(1.f, 0.f), sh, sl);
        val = __fadd_rn(sh, sl);
      }
    }
    pt[idx] = val;
  }
}

}  // namespace

cudaError_t launch_segments(epoch_ctx *c) {
  const Dims &d = c->d;
  k_segments<<<ceil_div(d.nn, 128), 128, 0, c->stream>>>(
      d, c->d_heights, c->d_parent, c->d_boundaries, c->d_phi, c->d_nseg, c->d_seg_mat,
      c->d_seg_dt, c->d_seg_hi, c->d_seg_lo);
  c->launches++;
  return cudaGetLastError();
}

static size_t setup_smem(const Dims &d) {
  return sizeof(double) * (4 * d.KK + d.K + 32 + 64) + sizeof(int) * 64 +
         sizeof(float) * (2 * d.KK + 64);
}

// Heights that arrived from device memory: every height finite and no parent
// below its child, else ST_HEIGHTS (reported by the next synchronising call).
__global__ void k_check_heights(Dims d, const double *__restrict__ h, const int *__restrict__ parent,
                                int *status) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.nn) return;
  const int u = parent[v];
  const bool ok = isfinite(h[v]) && (u < 0 || h[u] >= h[v]);
  if (!ok) atomicOr(status, ST_HEIGHTS);
}

cudaError_t launch_check_heights(epoch_ctx *c) {
  k_check_heights<<<ceil_div(c->d.nn, 256), 256, 0, c->stream>>>(c->d, c->d_heights, c->d_parent,
                                                                 c->d_status);
  c->launches++;
  return cudaGetLastError();
}

// Large K (reversible): the FP32 rotations in k_model_setup, then
// kEigSteps refinement steps of four launches (X^T X and S X; X^T (S X); E;
// X + X E), the last with compensated products, and k_eig_finish.
constexpr int kEigSteps = 5;
bool eig_refined(const Dims &d) { return d.K > 8 && d.reversible; }
size_t eig_scratch_doubles(int K, int S) { return (size_t)S * EigLayout(K).stride; }

// FP32 paths, reversible models: the float forms of the eigensystem that
// the branch matrices and the chain rule read (k_df_prep).
static cudaError_t launch_df_prep(epoch_ctx *c) {
  const Dims &d = c->d;
  if (c->precision == EPOCH_FP64 || !d.reversible) return cudaGetLastError();
  // the K = 4 kernels read neither form (unless its chain rule falls back to
  // the generic kernel)
  if (fast_k4(c) && k4_chain_smem(d) <= 160 * 1024) return cudaGetLastError();
  k_df_prep<<<d.S, 256, 0, c->stream>>>(d, c->d_lam, c->d_V, c->d_Vinv, c->d_pi, c->d_dfU,
                                        c->d_eig32);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_model_setup(epoch_ctx *c) {
  const Dims &d = c->d;
  size_t smem = setup_smem(d);
  // small K: one warp per matrix, rotations in registers; large K: 16 warps
  const int threads = d.K <= 8 ? 32 : 512;
  auto kern = d.K == 4 ? k_model_setup<4, 4> : (d.K <= 8 ? k_model_setup<0, 8> : k_model_setup<0, 0>);
  const bool refine = eig_refined(d) && c->d_eig;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<d.S, threads, smem, c->stream>>>(d, c->normalise, c->d_Qraw, c->d_pi, c->d_Q, c->d_cnorm,
                                          c->d_lam, c->d_V, c->d_Vinv, c->d_status,
                                          refine ? c->d_eig : nullptr);
  c->launches++;
  if (!refine) return launch_df_prep(c);
  const int K = d.K;
  const EigLayout L(K);
  const int tiles = (K + 15) / 16;
  auto gemm = [&](EigProds pr) {
    k_eig_gemm<<<dim3(tiles, tiles, d.S * pr.n), 256, 0, c->stream>>>(K, c->d_eig, L.stride, pr);
    c->launches++;
  };
  int x = L.X0, xn = L.X1;
  for (int it = 0; it < kEigSteps; it++) {
    const int comp = it == kEigSteps - 1;  // the last step at the FP64 rounding floor
    gemm(EigProds{{{x, x, L.T1, -1, 1, comp}, {L.A, x, L.T2, -1, 0, comp}}, 2});  // X^T X, S X
    gemm(EigProds{{{x, L.T2, L.T3, -1, 1, comp}, {}}, 1});                        // X^T S X
    k_eig_update<<<dim3((K + kEigRows - 1) / kEigRows, d.S), 256, 0, c->stream>>>(K, c->d_eig,
                                                                                 L.stride);
    c->launches++;
    gemm(EigProds{{{x, L.E, xn, x, 0, 0}, {}}, 1});  // X + X E
    std::swap(x, xn);
  }
  const size_t fsmem = sizeof(double) * (3 * (size_t)K * K + 96) + sizeof(int) * 64;
  cudaFuncSetAttribute(k_eig_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
  k_eig_finish<<<d.S, 512, fsmem, c->stream>>>(K, c->d_eig, L.stride, x, c->d_lam, c->d_V,
                                               c->d_Vinv, c->d_status);
  c->launches++;
  return launch_df_prep(c);
}

cudaError_t launch_param_transform(epoch_ctx *c) {
  const Dims &d = c->d;
  if (d.np == 0 || !d.reversible) return cudaSuccess;
  size_t smem = sizeof(double) * (2 * d.KK + 32);
  cudaFuncSetAttribute(k_param_transform, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  dim3 grid(d.np, d.S);
  k_param_transform<<<grid, 256, smem, c->stream>>>(d, c->normalise, c->d_dQraw, c->d_pi,
                                                    c->d_Q, c->d_cnorm, c->d_V, c->d_Vinv,
                                                    c->d_Dth, c->d_Dth32, c->d_Dnz);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_branch_matrices(epoch_ctx *c) {
  const Dims &d = c->d;
  if (c->precision != EPOCH_FP64 && d.reversible) {
    const size_t smem = sizeof(float2) * (4 * (size_t)d.KK + 3 * d.K);
    cudaFuncSetAttribute(k_branch_matrices_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    const int threads = d.KK >= 1024 ? 512 : (d.KK >= 256 ? 128 : 32);
    k_branch_matrices_df<<<dim3(d.nn, d.C), threads, smem, c->stream>>>(
        d, c->d_nseg, c->d_seg_mat, c->d_seg_dt, c->d_brate, c->d_catr, c->d_lam, c->d_dfU,
        c->d_masks, c->d_P64, c->d_PT32);
    c->launches++;
    return cudaGetLastError();
  }
  size_t smem = sizeof(double) * (4 * d.KK + 3 * d.K);
  cudaFuncSetAttribute(k_branch_matrices, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  int threads = d.KK >= 1024 ? 256 : (d.KK >= 256 ? 128 : 32);
  dim3 grid(d.nn, d.C);
  k_branch_matrices<<<grid, threads, smem, c->stream>>>(
      d, c->d_nseg, c->d_seg_mat, c->d_seg_dt, c->d_brate, c->d_catr, c->d_lam, c->d_V,
      c->d_Vinv, c->d_Q, c->d_pi, c->d_masks, c->d_P64,
      c->precision == EPOCH_FP64 ? nullptr : c->d_PT32);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace epoch
