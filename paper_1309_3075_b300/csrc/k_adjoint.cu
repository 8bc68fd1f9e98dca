// k_adjoint.cu -- gradient of lnL: pre-order ("outside") partials, the
// per-branch adjoint G_{v,c} = d lnL / d P_{v,c}, and the chain rule through
// the time-ordered segment products of Eq. convolution.
//
// The paper gives no gradient.  With post-order partials scaled per node
// (L_u = (S_v o S_w) 2^{-e_u}, S_x = P_x L_x), define the normalised outside
// partials U: U_root(c,i) = w_c pi_i / site, and for a child v of u with
// sibling w
//   X_v = U_u o S_w 2^{-e_u},      U_v = P_v^T X_v,
//   G_{v,c}[i][j] = sum_p n_p X_v(c,p,i) L_v(c,p,j),
// which equals sum_p n_p (d site_p / d P_v[i][j]) / site_p exactly (the
// scale factors cancel).  For a branch with segments E_1 (parent end) ..
// E_n, H_k = A_k^T G Z_k^T (A_k, Z_k the products above / below k) and
//   d lnL / d dt_k = r rho <H_k, Q_k E_k>,
//   d lnL / d theta = sum_k <Hhat_k o Phi_k, V^-1 dQ/dtheta V>,
// Hhat_k = V^T H_k V^-T, Phi_ij = (e^{tau l_i} - e^{tau l_j}) / (l_i - l_j)
// (tau e^{tau l_i} on the diagonal; Daleckii-Krein).  Heights, boundaries
// and branch rates then follow from how each dt_k depends on them.
#include <math.h>

#include "branch_table.cuh"

namespace epoch {
namespace {

// ---- generic pre-order (plain path and SIMT path for K > 4) ---------------

// X for both children of each node of the level: one thread per
// (child slot, category, pattern, state).
template <typename T>
__global__ void k_pre_x(Dims d, BranchTable<T> bt, const int *__restrict__ lvl_nodes, int lvl_off,
                        const int *__restrict__ child, int root, const T *__restrict__ part,
                        const T *__restrict__ pre, const int16_t *__restrict__ scale,
                        const uint8_t *__restrict__ tips, const double *__restrict__ pi,
                        const double *__restrict__ catw, const double *__restrict__ site_inv,
                        T *__restrict__ xbuf) {
  const int bi = blockIdx.y, x = blockIdx.z;
  const int u = lvl_nodes[lvl_off + bi];
  const int slot = u - d.N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)d.C * d.P * d.Kp) return;
  const int i = (int)(idx % d.Kp);
  const long long cp = idx / d.Kp;
  const int p = (int)(cp % d.P), c = (int)(cp / d.P);
  T out = 0;
  if (i < d.K) {
    const int sib = child[2 * slot + 1 - x];
    T uu;
    if (u == root)
      uu = (T)(catw[c] * pi[i] * site_inv[p]);
    else
      uu = pre[(((size_t)slot * d.C + c) * d.P + p) * d.Kp + i];
    const T s = child_factor<T>(d, bt, part, tips, sib, c, p, i);
    out = scale_by(uu * s, (int)scale[(size_t)slot * d.Pp + p]);
  }
  xbuf[((((size_t)bi * 2 + x) * d.C + c) * d.P + p) * d.Kp + i] = out;
}

// U_v = P_v^T X_v for internal children.
template <typename T>
__global__ void k_pre_u(Dims d, BranchTable<T> bt, const int *__restrict__ lvl_nodes, int lvl_off,
                        const int *__restrict__ child, const T *__restrict__ xbuf,
                        T *__restrict__ pre) {
  const int bi = blockIdx.y, x = blockIdx.z;
  const int u = lvl_nodes[lvl_off + bi];
  const int slot = u - d.N;
  const int v = child[2 * slot + x];
  if (v < d.N) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)d.C * d.P * d.Kp) return;
  const int j = (int)(idx % d.Kp);
  const long long cp = idx / d.Kp;
  const int p = (int)(cp % d.P), c = (int)(cp / d.P);
  T acc = 0;
  if (j < d.K) {
    const T *X = xbuf + ((((size_t)bi * 2 + x) * d.C + c) * d.P + p) * d.Kp;
    for (int i = 0; i < d.K; i++) acc += bt.mat(d, v, c, i, j) * X[i];
  }
  pre[(((size_t)(v - d.N) * d.C + c) * d.P + p) * d.Kp + j] = acc;
}

// Partial sums of G over a chunk of kTile patterns: one CTA per
// (chunk, node of level, child slot); threads over (c, i, j).
template <typename T>
__global__ void k_G_part(Dims d, const int *__restrict__ lvl_nodes, int lvl_off,
                         const int *__restrict__ child, const T *__restrict__ xbuf,
                         const T *__restrict__ part, const uint8_t *__restrict__ tips,
                         const unsigned long long *__restrict__ masks,
                         const double *__restrict__ pw, int nchunk, T *__restrict__ Gpart) {
  const int chunk = blockIdx.x, bi = blockIdx.y, x = blockIdx.z;
  const int u = lvl_nodes[lvl_off + bi];
  const int slot = u - d.N;
  const int v = child[2 * slot + x];
  const int p0 = chunk * kTile, p1 = min(d.P, p0 + kTile);
  T *out = Gpart + (((size_t)slot * nchunk + chunk) * 2 + x) * d.C * d.KK;
  for (int item = threadIdx.x; item < d.C * d.KK; item += blockDim.x) {
    const int c = item / d.KK, ij = item % d.KK, i = ij / d.K, j = ij % d.K;
    T acc = 0;
    const T *X = xbuf + (((size_t)bi * 2 + x) * d.C + c) * d.P * d.Kp;
    if (v < d.N) {
      for (int p = p0; p < p1; p++)
        if (code_allows(d, masks, tips[(size_t)v * d.Pp + p], j))
          acc += (T)pw[p] * X[(size_t)p * d.Kp + i];
    } else {
      const T *L = part + ((size_t)(v - d.N) * d.C + c) * d.P * d.Kp;
      for (int p = p0; p < p1; p++)
        acc += (T)pw[p] * X[(size_t)p * d.Kp + i] * L[(size_t)p * d.Kp + j];
    }
    out[item] = acc;
  }
}

// G[v][c][i][j] = sum over pattern blocks of Gpart in a fixed order (FP64 on
// the FP64 path; compensated FP32, as accurate, on the FP32 paths).  One thread per (child node v, c, i, j).
template <typename T>
__global__ void k_G_reduce(Dims d, const int *__restrict__ parent, const int *__restrict__ child,
                           const T *__restrict__ Gpart, int nchunk, double *__restrict__ G) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)d.nn * d.C * d.KK) return;
  const int ij = (int)(idx % d.KK);
  const int c = (int)((idx / d.KK) % d.C);
  const int v = (int)(idx / ((long long)d.KK * d.C));
  const int u = parent[v];
  if (u < 0) {
    G[idx] = 0.0;
    return;
  }
  const int slot = u - d.N;
  const int x = (child[2 * slot] == v) ? 0 : 1;
  if constexpr (sizeof(T) == sizeof(float)) {  // compensated FP32 (CSum)
    CSum acc;
    for (int k = 0; k < nchunk; k++)
      acc.add(Gpart[((((size_t)slot * nchunk + k) * 2 + x) * d.C + c) * d.KK + ij]);
    G[idx] = acc.value();
  } else {
    double acc = 0.0;
    for (int k = 0; k < nchunk; k++)
      acc += (double)Gpart[((((size_t)slot * nchunk + k) * 2 + x) * d.C + c) * d.KK + ij];
    G[idx] = acc;
  }
}

// ---- chain rule per (branch, category) --------------------------------------
// Matrices in shared memory in precision T (FP64 on the plain path, FP32 on
// the FP32 paths, where G itself comes from FP32 partials).
template <typename T>
__device__ void mm(const Dims &d, const T *A, const T *B, T *C, bool ta, bool tb) {
  // C = op(A) op(B)
  const int K = d.K;
  if (sizeof(T) == sizeof(float) && blockDim.x == 256 && K > 16 && K <= 64) {
    // 16 x 16 threads, a 4 x 4 block of C each (rows bi.., columns bj..)
    const int bi = (threadIdx.x >> 4) * 4, bj = (threadIdx.x & 15) * 4;
    T acc[4][4] = {};
    for (int m = 0; m < K; m++) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const int i = bi + r, j = bj + r;
        a[r] = i < K ? (ta ? A[m * K + i] : A[i * K + m]) : (T)0;
        b[r] = j < K ? (tb ? B[j * K + m] : B[m * K + j]) : (T)0;
      }
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[r][q] += a[r] * b[q];
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (bi + r < K && bj + q < K) C[(bi + r) * K + bj + q] = acc[r][q];
    return;
  }
  for (int idx = threadIdx.x; idx < d.KK; idx += blockDim.x) {
    const int i = idx / K, j = idx % K;
    T acc = 0;
    for (int m = 0; m < K; m++) {
      const T a = ta ? A[m * K + i] : A[i * K + m];
      const T b = tb ? B[j * K + m] : B[m * K + j];
      acc += a * b;
    }
    C[idx] = acc;
  }
}

template <typename T>
__device__ T bsum(T x, T *red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  T t = 0;
  for (int i = 0; i < (int)((blockDim.x + 31) >> 5); i++) t += red[i];
  __syncthreads();
  return t;
}

__device__ __forceinline__ double t_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float t_expm1(float x) { return expm1f(x); }
// e^{tau lambda} in the precision of the path (FP32: single-precision exp
// of the rounded exponent; each dependent FP64 instruction costs tens of
// cycles on this part, and these exponentials sit on the chain rule's
// critical path)
__device__ __forceinline__ double t_exp(double x) { return exp(x); }
__device__ __forceinline__ float t_exp(float x) { return expf(x); }

// Segment exponential E = exp(tau Q_s) into Eo (eigen path or
// uniformisation); scratch W, Y, B.
// The eigensystem (lam, V, V^-1) in the path's precision T: the FP64 one, or
// its FP32 copy (k_df_prep), so that the FP32 kernels convert nothing.
template <typename T>
__device__ void seg_exp(const Dims &d, int s, double tau, const T *lam, const T *V,
                        const T *Vinv, const double *Qn, T *Eo, T *W, T *Y, T *Bm, T *ev) {
  const int K = d.K, KK = d.KK;
  if (d.reversible) {
    for (int i = threadIdx.x; i < K; i += blockDim.x) ev[i] = t_exp((T)tau * lam[(size_t)s * K + i]);
    __syncthreads();
    const T *Vs = V + (size_t)s * KK, *Vi = Vinv + (size_t)s * KK;
    if (sizeof(T) == sizeof(float)) {
      // E = (V diag(ev)) V^-1 through shared memory (the tiled product for
      // large K; one batch of global loads for small K)
      for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
        W[idx] = Vs[idx] * ev[idx % K];
        Y[idx] = Vi[idx];
      }
      __syncthreads();
      mm<T>(d, W, Y, Eo, false, false);
      __syncthreads();
      return;
    }
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
      const int i = idx / K, j = idx % K;
      T acc = 0;
      for (int m = 0; m < K; m++) acc += Vs[i * K + m] * ev[m] * Vi[m * K + j];
      Eo[idx] = acc;
    }
    __syncthreads();
    return;
  }
  const double *Qs = Qn + (size_t)s * KK;
  double mu = 0.0;
  for (int i = 0; i < K; i++) mu = fmax(mu, fabs(Qs[i * K + i]));
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x)
    Eo[idx] = (idx / K == idx % K) ? (T)1 : (T)0;
  __syncthreads();
  if (mu == 0.0 || tau == 0.0) return;
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x)
    Bm[idx] = (T)(Qs[idx] / mu + ((idx / K == idx % K) ? 1.0 : 0.0));
  const double mt = mu * tau;
  const int npc = (int)ceil(mt / 30.0);
  const double x = mt / npc;
  const int mmax = (int)ceil(x + 12.0 * sqrt(x) + 30.0);
  for (int piece = 0; piece < npc; piece++) {
    double w = exp(-x);
    __syncthreads();
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
      Y[idx] = Eo[idx];
      W[idx] = (T)w * Eo[idx];
    }
    __syncthreads();
    for (int m = 1; m <= mmax; m++) {
      w = w * x / (double)m;
      mm<T>(d, Y, Bm, Eo, false, false);
      __syncthreads();
      for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
        Y[idx] = Eo[idx];
        W[idx] += (T)w * Eo[idx];
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) Eo[idx] = W[idx];
    __syncthreads();
  }
}

template <typename T>
__global__ void k_grad_branch(Dims d, const double *__restrict__ G, const int *__restrict__ nseg,
                              const int *__restrict__ seg_mat, const double *__restrict__ seg_dt,
                              const double *__restrict__ brate, const double *__restrict__ catr,
                              const T *__restrict__ lam, const T *__restrict__ V,
                              const T *__restrict__ Vinv, const double *__restrict__ Qn,
                              const T *__restrict__ Dth, const int *__restrict__ Dnz,
                              T *__restrict__ gseg) {
  extern __shared__ unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  const int v = blockIdx.x, c = blockIdx.y;
  const int ns = nseg[v];
  if (ns == 0) return;
  const int K = d.K, KK = d.KK;
  // seven K x K work matrices (an FP64 K = 64 set must fit in 227 KB; on the
  // FP32 path they leave room for two CTAs per SM at K = 61); G comes from
  // global memory into a free work matrix where a product needs it
  T *A = sm, *Z = A + KK, *H = Z + KK, *E = H + KK, *W = E + KK, *Y = W + KK, *Bm = Y + KK,
    *ev = Bm + KK, *red = ev + K;
  const double r = brate[v] * catr[c];
  const int stride = 1 + d.np;
  const double *Gd = G + ((size_t)v * d.C + c) * KK;
  auto g_into = [&](T *dst) {
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) dst[idx] = (T)Gd[idx];
  };
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) A[idx] = (idx / K == idx % K) ? 1 : 0;
  __syncthreads();
  for (int k = 0; k < ns; k++) {
    const int s = seg_mat[v * d.E + k];
    const double tau = r * seg_dt[v * d.E + k];
    // Z = E_{k+1} ... E_{n-1}  (recomputed; branches rarely have many
    // segments).  A (k = 0) and Z (k = ns - 1) are the identity at the ends:
    // products with them are copies.
    const bool A_id = (k == 0), Z_id = (k + 1 == ns);
    for (int q = k + 1; q < ns; q++) {
      seg_exp<T>(d, seg_mat[v * d.E + q], r * seg_dt[v * d.E + q], lam, V, Vinv, Qn, E, W, Y, Bm,
                 ev);
      if (q == k + 1) {
        for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) Z[idx] = E[idx];
      } else {
        mm<T>(d, Z, E, W, false, false);
        __syncthreads();
        for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) Z[idx] = W[idx];
      }
      __syncthreads();
    }
    // H = A^T G Z^T (W and Y are free here)
    if (A_id && Z_id) {
      g_into(H);
    } else if (A_id) {
      g_into(W);
      __syncthreads();
      mm<T>(d, W, Z, H, false, true);
    } else if (Z_id) {
      g_into(W);
      __syncthreads();
      mm<T>(d, A, W, H, true, false);
    } else {
      g_into(Y);
      __syncthreads();
      mm<T>(d, A, Y, W, true, false);
      __syncthreads();
      mm<T>(d, W, Z, H, false, true);
    }
    __syncthreads();
    // this segment's exponential: the eigen form needs it only to carry A
    // to the next segment
    if (!d.reversible || k + 1 < ns) seg_exp<T>(d, s, tau, lam, V, Vinv, Qn, E, W, Y, Bm, ev);
    T dk;
    if (d.reversible) {
      // Hhat = V^T H V^-T  into W, with V^-1 and then V of this segment's
      // matrix staged in Bm (free on the eigen path) for the shared-memory
      // products
      const T *Vs = V + (size_t)s * KK, *Vi = Vinv + (size_t)s * KK;
      for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) Bm[idx] = Vi[idx];
      __syncthreads();
      mm<T>(d, H, Bm, Y, false, true);  // Y = H V^-T
      __syncthreads();
      for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) Bm[idx] = Vs[idx];
      __syncthreads();
      mm<T>(d, Bm, Y, W, true, false);  // W = V^T Y
      for (int i = threadIdx.x; i < K; i += blockDim.x)
        ev[i] = t_exp((T)tau * lam[(size_t)s * K + i]);
      __syncthreads();
      T part = 0;
      for (int i = threadIdx.x; i < K; i += blockDim.x)
        part += W[i * K + i] * lam[(size_t)s * K + i] * ev[i];
      dk = bsum<T>(part, red);
      // model parameters: <Hhat o Phi, D_a,s>
      if (d.np > 0) {
        for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {  // W <- Hhat o Phi
          const int i = idx / K, j = idx % K;
          const T li = lam[(size_t)s * K + i], lj = lam[(size_t)s * K + j];
          const T tt = (T)tau;
          const T xx = tt * (li - lj);
          T phi;
          if (xx == (T)0)
            phi = tt * ev[j];
          else
            phi = ev[j] * tt * (t_expm1(xx) / xx);
          W[idx] *= phi;
        }
        __syncthreads();
        if (KK <= 256) {
          // few entries: a thread per parameter, no block reductions
          for (int a = threadIdx.x; a < d.np; a += blockDim.x) {
            T pa = 0;
            if (Dnz[a * d.S + s]) {
              const T *Da = Dth + ((size_t)a * d.S + s) * KK;
              for (int idx = 0; idx < KK; idx++) pa += W[idx] * Da[idx];
            }
            gseg[(((size_t)v * d.E + k) * d.C + c) * stride + 1 + a] = pa;
          }
        } else {
          for (int a = 0; a < d.np; a++) {
            if (!Dnz[a * d.S + s]) {
              if (threadIdx.x == 0) gseg[(((size_t)v * d.E + k) * d.C + c) * stride + 1 + a] = 0;
              continue;
            }
            const T *Da = Dth + ((size_t)a * d.S + s) * KK;
            T pa = 0;
            for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) pa += W[idx] * Da[idx];
            const T ga = bsum<T>(pa, red);
            if (threadIdx.x == 0) gseg[(((size_t)v * d.E + k) * d.C + c) * stride + 1 + a] = ga;
          }
        }
      }
    } else {
      // <H, Q E>
      const double *Qs = Qn + (size_t)s * KK;
      T part = 0;
      for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
        const int i = idx / K, j = idx % K;
        T qe = 0;
        for (int m = 0; m < K; m++) qe += (T)Qs[i * K + m] * E[m * K + j];
        part += H[idx] * qe;
      }
      dk = bsum<T>(part, red);
      for (int a = 0; a < d.np; a++)
        if (threadIdx.x == 0) gseg[(((size_t)v * d.E + k) * d.C + c) * stride + 1 + a] = 0;
    }
    if (threadIdx.x == 0) gseg[(((size_t)v * d.E + k) * d.C + c) * stride] = dk;
    // A <- A E_k
    __syncthreads();
    if (k + 1 < ns) {
      if (A_id) {
        for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) A[idx] = E[idx];
      } else {
        mm<T>(d, A, E, W, false, false);
        __syncthreads();
        for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) A[idx] = W[idx];
      }
      __syncthreads();
    }
  }
}

// Expected transition counts of every segment (FP64, reversible models), one
// CTA per (branch v, category c).  For segment k (parent end first), with A /
// Z the products of the segment exponentials above / below it,
//   H = A^T G Z^T,  Hhat = V^T H V^-T,  M = V^-T (Hhat o Phi) V^T,
//   N_ij = q_ij M_ij  (i != j; 0 on the diagonal),
// i.e. q_ij <H, dE/dq_ij> with dE/dq_ij = V ((V^-1 e_i e_j^T V) o Phi) V^-1
// (Daleckii-Krein, Phi as in the parameter terms of k_grad_branch).
// out[v][k][c][K][K].
__global__ void k_jump_counts(Dims d, const double *__restrict__ G, const int *__restrict__ nseg,
                              const int *__restrict__ seg_mat, const double *__restrict__ seg_dt,
                              const double *__restrict__ brate, const double *__restrict__ catr,
                              const double *__restrict__ lam, const double *__restrict__ V,
                              const double *__restrict__ Vinv, const double *__restrict__ Qn,
                              double *__restrict__ out) {
  extern __shared__ unsigned char smraw[];
  double *sm = reinterpret_cast<double *>(smraw);
  const int v = blockIdx.x, c = blockIdx.y;
  const int ns = nseg[v];
  if (ns == 0) return;
  const int K = d.K, KK = d.KK;
  double *A = sm, *Z = A + KK, *H = Z + KK, *E = H + KK, *W = E + KK, *Y = W + KK, *ev = Y + KK;
  const double r = brate[v] * catr[c];
  const double *Gm = G + ((size_t)v * d.C + c) * KK;
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) A[idx] = (idx / K == idx % K) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < ns; k++) {
    const int s = seg_mat[v * d.E + k];
    const double tau = r * seg_dt[v * d.E + k];
    // Z = E_{k+1} ... E_{ns-1}
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) Z[idx] = (idx / K == idx % K) ? 1.0 : 0.0;
    __syncthreads();
    for (int q = k + 1; q < ns; q++) {
      seg_exp<double>(d, seg_mat[v * d.E + q], r * seg_dt[v * d.E + q], lam, V, Vinv, Qn, E, W, Y,
                      W, ev);
      mm<double>(d, Z, E, W, false, false);
      __syncthreads();
      for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) Z[idx] = W[idx];
      __syncthreads();
    }
    mm<double>(d, A, Gm, W, true, false);  // W = A^T G
    __syncthreads();
    mm<double>(d, W, Z, H, false, true);   // H = A^T G Z^T
    __syncthreads();
    const double *Vs = V + (size_t)s * KK, *Vi = Vinv + (size_t)s * KK;
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {  // Y = H V^-T
      const int i = idx / K, j = idx % K;
      double acc = 0.0;
      for (int m = 0; m < K; m++) acc += H[i * K + m] * Vi[j * K + m];
      Y[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {  // W = V^T Y = Hhat
      const int i = idx / K, j = idx % K;
      double acc = 0.0;
      for (int m = 0; m < K; m++) acc += Vs[m * K + i] * Y[m * K + j];
      W[idx] = acc;
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) ev[i] = exp(tau * lam[(size_t)s * K + i]);
    __syncthreads();
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {  // W <- Hhat o Phi
      const int i = idx / K, j = idx % K;
      const double xx = tau * (lam[(size_t)s * K + i] - lam[(size_t)s * K + j]);
      W[idx] *= (xx == 0.0) ? tau * ev[j] : ev[j] * tau * (expm1(xx) / xx);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {  // Y = W V^T
      const int i = idx / K, j = idx % K;
      double acc = 0.0;
      for (int m = 0; m < K; m++) acc += W[i * K + m] * Vs[j * K + m];
      Y[idx] = acc;
    }
    __syncthreads();
    const double *Qs = Qn + (size_t)s * KK;
    double *o = out + (((size_t)v * d.E + k) * d.C + c) * KK;
    for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {  // M = V^-T Y; N = Q o M
      const int i = idx / K, j = idx % K;
      double acc = 0.0;
      for (int m = 0; m < K; m++) acc += Vi[m * K + i] * Y[m * K + j];
      o[idx] = (i != j) ? Qs[idx] * acc : 0.0;
    }
    __syncthreads();
    if (k + 1 < ns) {  // A <- A E_k
      seg_exp<double>(d, s, tau, lam, V, Vinv, Qn, E, W, Y, W, ev);
      mm<double>(d, A, E, W, false, false);
      __syncthreads();
      for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) A[idx] = W[idx];
      __syncthreads();
    }
  }
}

// Sums of the segment counts in a fixed order: threads [0, nn*KK) per branch
// (over segments and categories), then [nn*KK, (nn+E)*KK) per epoch (over
// every segment lying in the epoch: above boundary j it is epoch j+1, the
// bottom segment is in the epoch of its child's height).
__global__ void k_jump_reduce(Dims d, const int *__restrict__ parent, const int *__restrict__ nseg,
                              const int *__restrict__ seg_lo, const double *__restrict__ heights,
                              const double *__restrict__ b, const double *__restrict__ jumps,
                              double *__restrict__ per_branch, double *__restrict__ per_epoch) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nb = (long long)d.nn * d.KK;
  auto seg_sum = [&](int v, int k, int ij) {
    double acc = 0.0;
    for (int c = 0; c < d.C; c++) acc += jumps[(((size_t)v * d.E + k) * d.C + c) * d.KK + ij];
    return acc;
  };
  if (idx < nb) {
    const int v = (int)(idx / d.KK), ij = (int)(idx % d.KK);
    double acc = 0.0;
    if (parent[v] >= 0)
      for (int k = 0; k < nseg[v]; k++) acc += seg_sum(v, k, ij);
    per_branch[idx] = acc;
    return;
  }
  idx -= nb;
  if (idx >= (long long)d.E * d.KK) return;
  const int e = (int)(idx / d.KK), ij = (int)(idx % d.KK);
  double acc = 0.0;
  for (int v = 0; v < d.nn; v++) {
    if (parent[v] < 0) continue;
    int eb = 0;
    for (int j = 0; j < d.E - 1; j++) eb += (b[j] <= heights[v]);
    for (int k = 0; k < nseg[v]; k++) {
      const int lo = seg_lo[v * d.E + k];
      if ((lo < 0 ? -lo : eb) == e) acc += seg_sum(v, k, ij);
    }
  }
  per_epoch[idx] = acc;
}

// Final reductions into FP64 outputs (fixed order, deterministic):
//   blocks [0, nb_nodes): node heights and branch rates (thread per node);
//   next E-1 blocks: boundary j;  next np blocks: parameter a.
// out = [d_heights (nn) | d_boundaries (E-1) | d_params (np) | d_rates (nn)].
template <typename T>
__global__ void k_grad_reduce(Dims d, const int *__restrict__ parent, const int *__restrict__ child,
                              const int *__restrict__ nseg, const double *__restrict__ seg_dt,
                              const int *__restrict__ seg_hi, const int *__restrict__ seg_lo,
                              const double *__restrict__ brate, const double *__restrict__ catr,
                              const T *__restrict__ gseg, int nb_nodes, double *__restrict__ out) {
  pdl_wait();  // the segment terms
  pdl_trigger();
  __shared__ double red[32];
  const int stride = 1 + d.np;
  // d lnL / d dt of segment (v, k) summed over categories
  auto gdt = [&](int v, int k) {
    double acc = 0.0;
    for (int c = 0; c < d.C; c++)
      acc += brate[v] * catr[c] * (double)gseg[(((size_t)v * d.E + k) * d.C + c) * stride];
    return acc;
  };
  if ((int)blockIdx.x < nb_nodes) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= d.nn) return;
    double dh = 0.0;
    if (u >= d.N) {
      for (int x = 0; x < 2; x++) dh += gdt(child[2 * (u - d.N) + x], 0);
    }
    double dr = 0.0;
    if (parent[u] >= 0) {
      dh -= gdt(u, nseg[u] - 1);
      for (int k = 0; k < nseg[u]; k++) {
        double acc = 0.0;
        for (int c = 0; c < d.C; c++)
          acc += catr[c] * (double)gseg[(((size_t)u * d.E + k) * d.C + c) * stride];
        dr += acc * seg_dt[u * d.E + k];
      }
    }
    out[u] = dh;
    out[d.nn + (d.E - 1) + d.np + u] = dr;
    return;
  }
  const int b = blockIdx.x - nb_nodes;
  double part = 0.0;
  if (b < d.E - 1) {
    const int ref = -(b + 1);
    for (int v = threadIdx.x; v < d.nn; v += blockDim.x) {
      for (int k = 0; k < nseg[v]; k++) {
        if (seg_hi[v * d.E + k] == ref) part += gdt(v, k);
        if (seg_lo[v * d.E + k] == ref) part -= gdt(v, k);
      }
    }
  } else {
    const int a = b - (d.E - 1);
    for (int v = threadIdx.x; v < d.nn; v += blockDim.x)
      for (int k = 0; k < nseg[v]; k++)
        for (int c = 0; c < d.C; c++)
          part += (double)gseg[(((size_t)v * d.E + k) * d.C + c) * stride + 1 + a];
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
    if (b < d.E - 1)
      out[d.nn + b] = t;
    else
      out[d.nn + (d.E - 1) + (b - (d.E - 1))] = t;
  }
}

// G over one chunk of kTile patterns for (level node, child x, category c),
// register-tiled: the KB x KB block of (i, j) (KB = K rounded up to 8, 16, 32
// or 64) is split over a (KB/RT) x (KB/RT) thread grid, each thread owning an
// RT x RT tile (RT = 4; 8 x 8 tiles at KB = 64 measured slower).  The 256
// threads form
// NG = 256 / (KB/RT)^2 groups that take interleaved patterns and are summed in
// a fixed order at the end.  Patterns go through shared memory SUB = 2048 / KB
// at a time (X rows, and n_p L_v rows or the tip code's indicator); the next
// batch is loaded into registers while the current one is multiplied.  Same
// output layout as k_G_part.
template <int KB>
__global__ void __launch_bounds__(256) k_G_tiled(Dims d, const int *__restrict__ lvl_nodes,
                                                 int lvl_off, const int *__restrict__ child,
                                                 const float *__restrict__ xbuf,
                                                 const float *__restrict__ part,
                                                 const uint8_t *__restrict__ tips,
                                                 const unsigned long long *__restrict__ masks,
                                                 const double *__restrict__ pw, int nchunk,
                                                 float *__restrict__ Gpart) {
  constexpr int RT = 4, TW = KB / RT, NG = 256 / (TW * TW), SUB = 2048 / KB;
  constexpr int V4 = SUB * KB / 4 / 256;  // float4 of X (and of L) per thread per batch: 2
  __shared__ __align__(16) float Xs[SUB * KB];
  __shared__ __align__(16) float Ls[SUB * KB];
  const int chunk = blockIdx.x, bi = blockIdx.y, x = blockIdx.z / d.C, c = blockIdx.z % d.C;
  const int u = lvl_nodes[lvl_off + bi];
  const int slot = u - d.N;
  const int v = child[2 * slot + x];
  const int p0 = chunk * kTile, p1 = min(d.P, p0 + kTile);
  const float *X = xbuf + (((size_t)bi * 2 + x) * d.C + c) * d.P * d.Kp;
  const float *L = v >= d.N ? part + ((size_t)(v - d.N) * d.C + c) * d.P * d.Kp : nullptr;
  const int grp = threadIdx.x / (TW * TW), t = threadIdx.x % (TW * TW);
  const int ti = t / TW, tj = t % TW;
  float4 xr[V4], lr[V4];
  // batch q0 into registers: float4 e = threadIdx.x + 256 m is pattern e / (KB/4),
  // states 4 (e % (KB/4)) ..
  auto fetch = [&](int q0) {
#pragma unroll
    for (int m = 0; m < V4; m++) {
      const int e = threadIdx.x + 256 * m, pr = e / (KB / 4), k = 4 * (e % (KB / 4)), p = q0 + pr;
      float4 xv = make_float4(0.f, 0.f, 0.f, 0.f), lv = xv;
      if (p < p1 && k < d.Kp) {  // entries K..Kp-1 are stored zeros
        xv = *reinterpret_cast<const float4 *>(X + (size_t)p * d.Kp + k);
        const float n = (float)pw[p];
        if (L) {
          lv = *reinterpret_cast<const float4 *>(L + (size_t)p * d.Kp + k);
          lv = make_float4(n * lv.x, n * lv.y, n * lv.z, n * lv.w);
        } else {
          const int code = tips[(size_t)v * d.Pp + p];
          lv = make_float4(code_allows(d, masks, code, k) && k < d.K ? n : 0.f,
                           code_allows(d, masks, code, k + 1) && k + 1 < d.K ? n : 0.f,
                           code_allows(d, masks, code, k + 2) && k + 2 < d.K ? n : 0.f,
                           code_allows(d, masks, code, k + 3) && k + 3 < d.K ? n : 0.f);
        }
      }
      xr[m] = xv;
      lr[m] = lv;
    }
  };
  float acc[RT][RT] = {};
  fetch(p0);
  for (int q0 = p0; q0 < p1; q0 += SUB) {
#pragma unroll
    for (int m = 0; m < V4; m++) {
      const int e = threadIdx.x + 256 * m;
      reinterpret_cast<float4 *>(Xs)[e] = xr[m];
      reinterpret_cast<float4 *>(Ls)[e] = lr[m];
    }
    __syncthreads();
    if (q0 + SUB < p1) fetch(q0 + SUB);  // in flight during the products
#pragma unroll 2
    for (int pr = grp; pr < SUB; pr += NG) {
      float av[RT], bv[RT];
#pragma unroll
      for (int h = 0; h < RT / 4; h++) {
        const float4 a = *reinterpret_cast<const float4 *>(&Xs[pr * KB + RT * ti + 4 * h]);
        const float4 b = *reinterpret_cast<const float4 *>(&Ls[pr * KB + RT * tj + 4 * h]);
        av[4 * h] = a.x, av[4 * h + 1] = a.y, av[4 * h + 2] = a.z, av[4 * h + 3] = a.w;
        bv[4 * h] = b.x, bv[4 * h + 1] = b.y, bv[4 * h + 2] = b.z, bv[4 * h + 3] = b.w;
      }
#pragma unroll
      for (int r = 0; r < RT; r++)
#pragma unroll
        for (int q = 0; q < RT; q++) acc[r][q] += av[r] * bv[q];
    }
    __syncthreads();
  }
  float *out = Gpart + (((size_t)slot * nchunk + chunk) * 2 + x) * d.C * d.KK + (size_t)c * d.KK;
  if (NG == 1) {
#pragma unroll
    for (int r = 0; r < RT; r++)
#pragma unroll
      for (int q = 0; q < RT; q++) {
        const int i = RT * ti + r, j = RT * tj + q;
        if (i < d.K && j < d.K) out[i * d.K + j] = acc[r][q];
      }
    return;
  }
  // group sums in a fixed order through the 4096 floats of Xs | Ls (flat
  // index f, split at SUB * KB): all groups at once when NG * KB^2 fits,
  // else one group after another
  auto red_at = [&](int f) -> float & { return f < SUB * KB ? Xs[f] : Ls[f - SUB * KB]; };
  if (NG * KB * KB <= 2 * SUB * KB) {
#pragma unroll
    for (int r = 0; r < RT; r++)
#pragma unroll
      for (int q = 0; q < RT; q++) red_at(grp * KB * KB + (RT * ti + r) * KB + RT * tj + q) = acc[r][q];
    __syncthreads();
    for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) {
      const int i = e / KB, j = e % KB;
      float sum = 0.f;
      for (int g = 0; g < NG; g++) sum += red_at(g * KB * KB + e);
      if (i < d.K && j < d.K) out[i * d.K + j] = sum;
    }
  } else {
    for (int g = 0; g < NG; g++) {
      if (grp == g) {
#pragma unroll
        for (int r = 0; r < RT; r++)
#pragma unroll
          for (int q = 0; q < RT; q++) {
            float &cell = red_at((RT * ti + r) * KB + RT * tj + q);
            cell = g ? cell + acc[r][q] : acc[r][q];
          }
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) {
      const int i = e / KB, j = e % KB;
      if (i < d.K && j < d.K) out[i * d.K + j] = red_at(e);
    }
  }
}

template <int KB>
void launch_G_tiled(epoch_ctx *c, int l, int w, int nchunk) {
  const Dims &d = c->d;
  dim3 gg(nchunk, w, 2 * d.C);
  k_G_tiled<KB><<<gg, 256, 0, c->stream>>>(d, c->d_level_nodes, c->h_level_off[l], c->d_child,
                                           (const float *)c->d_xbuf, (const float *)c->d_part,
                                           c->d_tips, c->d_masks, c->d_pw, nchunk,
                                           (float *)c->d_Gpart);
}

template <typename T>
void launch_pre_generic(epoch_ctx *c, BranchTable<T> bt, int root) {
  const Dims &d = c->d;
  const int L = (int)c->h_level_off.size() - 1;
  const long long items = (long long)d.C * d.P * d.Kp;
  const int nchunk = ceil_div(d.P, kTile);
  for (int l = L - 1; l >= 0; l--) {
    const int w = c->h_level_off[l + 1] - c->h_level_off[l];
    dim3 g(ceil_div(items, 256), w, 2);
    if (sizeof(T) == sizeof(float) && tc_path(c)) {
      launch_tc_pre_x(c, l, root);  // S by tile products, then X
      c->launches--;                // counted below
    } else {
      k_pre_x<T><<<g, 256, 0, c->stream>>>(d, bt, c->d_level_nodes, c->h_level_off[l],
                                           c->d_child, root, (const T *)c->d_part,
                                           (const T *)c->d_pre, c->d_scale, c->d_tips, c->d_pi,
                                           c->d_catw, c->d_site_inv, (T *)c->d_xbuf);
    }
    if (sizeof(T) == sizeof(float) && tc_path(c)) {
      launch_tc_pre_u(c, l);  // U = P^T X on the tensor cores
      c->launches--;          // counted below
    } else {
      k_pre_u<T><<<g, 256, 0, c->stream>>>(d, bt, c->d_level_nodes, c->h_level_off[l],
                                           c->d_child, (const T *)c->d_xbuf, (T *)c->d_pre);
    }
    if (sizeof(T) == sizeof(float) && d.K > 32) {
      launch_G_tiled<64>(c, l, w, nchunk);
    } else if (sizeof(T) == sizeof(float) && d.K > 16) {
      launch_G_tiled<32>(c, l, w, nchunk);
    } else if (sizeof(T) == sizeof(float) && d.K > 8) {
      launch_G_tiled<16>(c, l, w, nchunk);
    } else if (sizeof(T) == sizeof(float)) {
      launch_G_tiled<8>(c, l, w, nchunk);
    } else {
      dim3 gg(nchunk, w, 2);
      k_G_part<T><<<gg, 256, 0, c->stream>>>(d, c->d_level_nodes, c->h_level_off[l], c->d_child,
                                             (const T *)c->d_xbuf, (const T *)c->d_part,
                                             c->d_tips, c->d_masks, c->d_pw, nchunk,
                                             (T *)c->d_Gpart);
    }
    c->launches += 3;
  }
}

}  // namespace

cudaError_t launch_expected_counts(epoch_ctx *c, double *d_per_branch, double *d_per_epoch) {
  const Dims &d = c->d;
  const int threads = d.KK >= 1024 ? 256 : (d.KK >= 256 ? 128 : 32);
  const size_t smem = sizeof(double) * (6 * d.KK + d.K);
  cudaFuncSetAttribute(k_jump_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_jump_counts<<<dim3(d.nn, d.C), threads, smem, c->stream>>>(
      d, c->d_G, c->d_nseg, c->d_seg_mat, c->d_seg_dt, c->d_brate, c->d_catr, c->d_lam, c->d_V,
      c->d_Vinv, c->d_Q, c->d_jumps);
  const long long n = (long long)(d.nn + d.E) * d.KK;
  k_jump_reduce<<<ceil_div(n, 256), 256, 0, c->stream>>>(d, c->d_parent, c->d_nseg, c->d_seg_lo,
                                                         c->d_heights, c->d_boundaries,
                                                         c->d_jumps, d_per_branch, d_per_epoch);
  c->launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_adjoint(epoch_ctx *c) {
  const Dims &d = c->d;
  int root = -1;
  for (int v = 0; v < d.nn; v++)
    if (c->h_parent[v] < 0) root = v;
  const long long nG = (long long)d.nn * d.C * d.KK;
  if (small_path(c)) {  // one launch for all levels; G terms per pattern
    cudaError_t e = launch_small_pre(c);
    if (e != cudaSuccess) return e;
    if (c->precision == EPOCH_FP64)
      k_G_reduce<double><<<ceil_div(nG, 256), 256, 0, c->stream>>>(
          d, c->d_parent, c->d_child, (const double *)c->d_Gpart, d.P, c->d_G);
    else
      k_G_reduce<float><<<ceil_div(nG, 256), 256, 0, c->stream>>>(
          d, c->d_parent, c->d_child, (const float *)c->d_Gpart, d.P, c->d_G);
    c->launches++;
    return cudaGetLastError();
  }
  const int nchunk = ceil_div(d.P, kTile);
  if (c->precision == EPOCH_FP64) {
    launch_pre_generic<double>(c, BranchTable<double>{c->d_P64, c->d_masks}, root);
    k_G_reduce<double><<<ceil_div(nG, 256), 256, 0, c->stream>>>(
        d, c->d_parent, c->d_child, (const double *)c->d_Gpart, nchunk, c->d_G);
  } else {
    if (fast_k4(c)) return launch_preorder_k4(c);  // adjoint pass and G reduction
    launch_pre_generic<float>(c, BranchTable<float>{c->d_PT32, c->d_masks}, root);
    k_G_reduce<float><<<ceil_div(nG, 256), 256, 0, c->stream>>>(
        d, c->d_parent, c->d_child, (const float *)c->d_Gpart, nchunk, c->d_G);
  }
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_chain_rule(epoch_ctx *c) {
  {
    cudaError_t je = join_side(c, 0);  // the parameter transform
    if (je != cudaSuccess) return je;
  }
  const Dims &d = c->d;
  dim3 grid(d.nn, d.C);
  const int threads = d.KK >= 1024 ? 256 : (d.KK >= 256 ? 128 : 32);
  const int nb_nodes = ceil_div(d.nn, 256);
  const int nblocks = nb_nodes + (d.E - 1) + d.np;
  if (c->precision == EPOCH_FP64) {
    size_t smem = sizeof(double) * (7 * d.KK + d.K + 32);
    cudaFuncSetAttribute(k_grad_branch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_grad_branch<double><<<grid, threads, smem, c->stream>>>(
        d, c->d_G, c->d_nseg, c->d_seg_mat, c->d_seg_dt, c->d_brate, c->d_catr, c->d_lam, c->d_V,
        c->d_Vinv, c->d_Q, c->d_Dth, c->d_Dnz, (double *)c->d_gseg);
    k_grad_reduce<double><<<nblocks, 256, 0, c->stream>>>(
        d, c->d_parent, c->d_child, c->d_nseg, c->d_seg_dt, c->d_seg_hi, c->d_seg_lo, c->d_brate,
        c->d_catr, (const double *)c->d_gseg, nb_nodes, c->d_grad);
  } else {
    if (fast_k4(c) && d.reversible && k4_chain_smem(d) <= 160 * 1024) {
      cudaError_t e = launch_chain_k4(c);
      if (e != cudaSuccess) return e;
      c->launches--;  // counted below with the reduction
    } else {
      size_t smem = sizeof(float) * (7 * d.KK + d.K + 32);
      cudaFuncSetAttribute(k_grad_branch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      // the eigensystem in FP32 (k_df_prep; unused by non-reversible models)
      const size_t SKK = (size_t)d.S * d.KK;
      const float *e32 = c->d_eig32;
      k_grad_branch<float><<<grid, threads, smem, c->stream>>>(
          d, c->d_G, c->d_nseg, c->d_seg_mat, c->d_seg_dt, c->d_brate, c->d_catr,
          e32 + 2 * SKK, e32, e32 + SKK, c->d_Q, c->d_Dth32, c->d_Dnz, (float *)c->d_gseg);
    }
    launch_pdl(k_grad_reduce<float>, dim3(nblocks), dim3(256), 0, c->stream, d,
               (const int *)c->d_parent, (const int *)c->d_child, (const int *)c->d_nseg,
               (const double *)c->d_seg_dt, (const int *)c->d_seg_hi, (const int *)c->d_seg_lo,
               (const double *)c->d_brate, (const double *)c->d_catr, (const float *)c->d_gseg,
               nb_nodes, c->d_grad);
  }
  c->launches += 2;
  return cudaGetLastError();
}

}  // namespace epoch
