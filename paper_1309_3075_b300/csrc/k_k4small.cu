// k_k4small.cu -- per-branch kernels of the FP32 K = 4 path with a reversible
// model: 4 x 4 matrices in registers, no shared memory.
//
//  k4_branch: cuts the branch at the epoch boundaries ("Relaxing
//    time-homogeneity"), forms P = prod_k V diag(exp(r rho dt_k lambda)) V^-1
//    in FP64 in time order, parent end first (Eq. convolution), and writes
//    the FP64 matrix and the transposed FP32 table with the missing-data and
//    ambiguity rows.  One thread per row of P; the first thread of each
//    branch also records the segments for the gradient.
//  k4_chain: the chain rule through the product for one (branch,
//    category): d lnL / d dt_k = <H_k, Q_k E_k> and the model-parameter terms
//    <Hhat_k o Phi_k, V^-1 dQ V>, H_k = A_k^T G Z_k^T (see k_adjoint.cu).
#include <math.h>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

// Thread = (branch v, category c, row i): the four threads of a quad share
// the branch's segments; each carries row i of the running product.  Per
// segment, row <- ((row V) o exp(tau lambda)) V^-1; lane i of the quad takes
// the exponential of eigenvalue i and the quad exchanges them by shuffles.
__global__ void __launch_bounds__(128) k4_branch(Dims d, const double *__restrict__ heights,
                                                 const int *__restrict__ parent,
                                                 const double *__restrict__ b,
                                                 const int *__restrict__ phi,
                                                 const double *__restrict__ brate,
                                                 const double *__restrict__ catr,
                                                 const double *__restrict__ lam,
                                                 const double *__restrict__ V,
                                                 const double *__restrict__ Vinv,
                                                 const unsigned long long *__restrict__ masks,
                                                 int *__restrict__ nseg, int *__restrict__ seg_mat,
                                                 double *__restrict__ seg_dt, int *__restrict__ seg_hi,
                                                 int *__restrict__ seg_lo, double *__restrict__ P64,
                                                 float *__restrict__ PT32) {
  pdl_wait();  // the eigensystems
  pdl_trigger();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = idx & 3, vc = idx >> 2;
  const int v = vc / d.C, c = vc % d.C;
  if (v >= d.nn) return;  // whole quads leave together
  const unsigned qmask = 0xfu << (threadIdx.x & 28);
  const bool writer = (c == 0 && i == 0);
  const int u = parent[v];
  if (u < 0) {
    if (writer) nseg[v] = 0;
    return;
  }
  const int E = d.E;
  const double lo = heights[v], hi = heights[u];
  const double r = brate[v] * catr[c];
  double row[4] = {i == 0 ? 1.0 : 0.0, i == 1 ? 1.0 : 0.0, i == 2 ? 1.0 : 0.0, i == 3 ? 1.0 : 0.0};
  int n = 0;
  // segments from the parent end: (matrix, dt, hi ref, lo ref)
  auto apply = [&](int s, double dt, int href, int lref) {
    if (writer) {
      seg_mat[v * E + n] = s;
      seg_dt[v * E + n] = dt;
      seg_hi[v * E + n] = href;
      seg_lo[v * E + n] = lref;
    }
    n++;
    const double tau = r * dt;
    if (tau == 0.0) return;  // exact identity
    const double mine = exp(tau * lam[s * 4 + i]);
    double ev[4];
#pragma unroll
    for (int m = 0; m < 4; m++) ev[m] = __shfl_sync(qmask, mine, m, 4);
    const double *Vs = V + s * 16, *Vi = Vinv + s * 16;
    double y[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 4; k++) acc += row[k] * Vs[k * 4 + m];
      y[m] = acc * ev[m];
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 4; m++) acc += y[m] * Vi[m * 4 + j];
      row[j] = acc;
    }
  };
  if (hi == lo) {
    int e = 0;
    for (int j = 0; j < E - 1; j++) e += (b[j] <= lo);
    apply(phi[e], 0.0, u, v);
  } else {
    double top = hi;
    int top_ref = u;
    for (int j = E - 2; j >= 0; j--) {
      const double bj = b[j];
      if (bj > lo && bj < hi) {
        apply(phi[j + 1], top - bj, top_ref, -(j + 1));
        top = bj;
        top_ref = -(j + 1);
      }
    }
    int e = 0;
    for (int j = 0; j < E - 1; j++) e += (b[j] <= lo);
    apply(phi[e], top - lo, top_ref, v);
  }
  if (writer) nseg[v] = n;
#pragma unroll
  for (int j = 0; j < 4; j++) row[j] = fmax(row[j], 0.0);  // probabilities: cut rounding negatives
  double *out = P64 + (((size_t)v * d.C + c) * 4 + i) * 4;
#pragma unroll
  for (int j = 0; j < 4; j++) out[j] = row[j];
  float *pt = PT32 + ((size_t)v * d.C + c) * d.NR * 4;
#pragma unroll
  for (int j = 0; j < 4; j++) pt[j * 4 + i] = (float)row[j];
  for (int code = 4; code < d.NR; code++) {
    const unsigned long long mk = (code == 4) ? ~0ull : masks[code - 5];
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; j++)
      if ((mk >> j) & 1ull) s += row[j];
    pt[code * 4 + i] = (float)s;
  }
}

__device__ __forceinline__ void mm4(const float *A, const float *B, float *C) {
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float acc = 0.f;
#pragma unroll
      for (int m = 0; m < 4; m++) acc += A[i * 4 + m] * B[m * 4 + j];
      C[i * 4 + j] = acc;
    }
}

// Thread = (branch v, category c, quarter q): the four threads of a quad
// form the same 4 x 4 products (registers) and split the model parameters
// (q, q + 4, ...).  The eigensystems and V^-1 dQ V of every matrix sit in
// shared memory as FP32.
__global__ void __launch_bounds__(128) k4_chain(Dims d, const double *__restrict__ G,
                                                const int *__restrict__ nseg,
                                                const int *__restrict__ seg_mat,
                                                const double *__restrict__ seg_dt,
                                                const double *__restrict__ brate,
                                                const double *__restrict__ catr,
                                                const double *__restrict__ lam,
                                                const double *__restrict__ V,
                                                const double *__restrict__ Vinv,
                                                const float *__restrict__ Dth,
                                                const int *__restrict__ Dnz,
                                                float *__restrict__ gseg) {
  extern __shared__ float sm[];
  float *sV = sm, *sVi = sV + d.S * 16, *slam = sVi + d.S * 16, *sD = slam + d.S * 4;
  int *sNz = reinterpret_cast<int *>(sD + (size_t)d.np * d.S * 16);
  for (int i = threadIdx.x; i < d.S * 16; i += blockDim.x) {
    sV[i] = (float)V[i];
    sVi[i] = (float)Vinv[i];
  }
  for (int i = threadIdx.x; i < d.S * 4; i += blockDim.x) slam[i] = (float)lam[i];
  for (int i = threadIdx.x; i < d.np * d.S * 16; i += blockDim.x) sD[i] = Dth[i];
  for (int i = threadIdx.x; i < d.np * d.S; i += blockDim.x) sNz[i] = Dnz[i];
  pdl_wait();  // G
  pdl_trigger();
  __syncthreads();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int qq = idx & 3, vc = idx >> 2;
  const int v = vc / d.C, c = vc % d.C;
  if (v >= d.nn) return;
  const int ns = nseg[v];
  if (ns == 0) return;
  const int E = d.E, stride = 1 + d.np;
  const double r = brate[v] * catr[c];
  float Gm[16], A[16];
#pragma unroll
  for (int q = 0; q < 16; q++) {
    Gm[q] = (float)G[((size_t)v * d.C + c) * 16 + q];
    A[q] = (q % 5 == 0) ? 1.f : 0.f;
  }
  for (int k = 0; k < ns; k++) {
    const int s = seg_mat[v * E + k];
    const float tau = (float)(r * seg_dt[v * E + k]);
    const float *Vs = sV + s * 16, *Vi = sVi + s * 16;
    float li[4], ev[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      li[i] = slam[s * 4 + i];
      ev[i] = expf(tau * li[i]);
    }
    // Z = E_{k+1} ... E_{n-1}
    float Z[16];
#pragma unroll
    for (int q = 0; q < 16; q++) Z[q] = (q % 5 == 0) ? 1.f : 0.f;
    for (int qn = k + 1; qn < ns; qn++) {
      const int s2 = seg_mat[v * E + qn];
      const float t2 = (float)(r * seg_dt[v * E + qn]);
      const float *V2 = sV + s2 * 16, *Vi2 = sVi + s2 * 16;
      float e2[4], Ek[16], T[16];
#pragma unroll
      for (int i = 0; i < 4; i++) e2[i] = expf(t2 * slam[s2 * 4 + i]);
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < 4; m++) acc += V2[i * 4 + m] * e2[m] * Vi2[m * 4 + j];
          Ek[i * 4 + j] = acc;
        }
      mm4(Z, Ek, T);
#pragma unroll
      for (int q = 0; q < 16; q++) Z[q] = T[q];
    }
    // H = A^T G Z^T
    float H[16];
    if (ns == 1) {
#pragma unroll
      for (int q = 0; q < 16; q++) H[q] = Gm[q];
    } else {
      float W[16];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < 4; m++) acc += A[m * 4 + i] * Gm[m * 4 + j];
          W[i * 4 + j] = acc;
        }
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < 4; m++) acc += W[i * 4 + m] * Z[j * 4 + m];
          H[i * 4 + j] = acc;
        }
    }
    // Hhat = V^T H V^-T
    float Y[16], Hh[16];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < 4; m++) acc += H[i * 4 + m] * Vi[j * 4 + m];
        Y[i * 4 + j] = acc;
      }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < 4; m++) acc += Vs[m * 4 + i] * Y[m * 4 + j];
        Hh[i * 4 + j] = acc;
      }
    float *out = gseg + (((size_t)v * E + k) * d.C + c) * stride;
    if (qq == 0) {
      float dk = 0.f;
#pragma unroll
      for (int i = 0; i < 4; i++) dk += Hh[i * 5] * li[i] * ev[i];
      out[0] = dk;
    }
    if (d.np > qq) {
      float W[16];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const float x = tau * (li[i] - li[j]);
          const float ph = (x == 0.f) ? tau * ev[j] : ev[j] * tau * (expm1f(x) / x);
          W[i * 4 + j] = Hh[i * 4 + j] * ph;
        }
      for (int a = qq; a < d.np; a += 4) {
        float ga = 0.f;
        if (sNz[a * d.S + s]) {
          const float *Da = sD + ((size_t)a * d.S + s) * 16;
#pragma unroll
          for (int q = 0; q < 16; q++) ga += W[q] * Da[q];
        }
        out[1 + a] = ga;
      }
    }
    // A <- A E_k
    if (k + 1 < ns) {
      float Ek[16], T[16];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < 4; m++) acc += Vs[i * 4 + m] * ev[m] * Vi[m * 4 + j];
          Ek[i * 4 + j] = acc;
        }
      mm4(A, Ek, T);
#pragma unroll
      for (int q = 0; q < 16; q++) A[q] = T[q];
    }
  }
}

}  // namespace

size_t k4_chain_smem(const Dims &d) {
  return sizeof(float) * ((size_t)d.S * 36 + (size_t)d.np * d.S * 16) +
         sizeof(int) * (size_t)d.np * d.S;
}

cudaError_t launch_branch_k4(epoch_ctx *c) {
  const Dims &d = c->d;
  const int n = d.nn * d.C * 4;
  cudaError_t e = launch_pdl(k4_branch, dim3(ceil_div(n, 64)), dim3(64), 0, c->stream, d,
                             (const double *)c->d_heights, (const int *)c->d_parent,
                             (const double *)c->d_boundaries, (const int *)c->d_phi,
                             (const double *)c->d_brate, (const double *)c->d_catr,
                             (const double *)c->d_lam, (const double *)c->d_V,
                             (const double *)c->d_Vinv, (const unsigned long long *)c->d_masks,
                             c->d_nseg, c->d_seg_mat, c->d_seg_dt, c->d_seg_hi, c->d_seg_lo,
                             c->d_P64, c->d_PT32);
  c->launches++;
  return e;
}

cudaError_t launch_chain_k4(epoch_ctx *c) {
  const Dims &d = c->d;
  const int n = d.nn * d.C * 4;
  const size_t smem = k4_chain_smem(d);
  cudaFuncSetAttribute(k4_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaError_t e = launch_pdl(k4_chain, dim3(ceil_div(n, 128)), dim3(128), smem, c->stream, d,
                             (const double *)c->d_G, (const int *)c->d_nseg,
                             (const int *)c->d_seg_mat, (const double *)c->d_seg_dt,
                             (const double *)c->d_brate, (const double *)c->d_catr,
                             (const double *)c->d_lam, (const double *)c->d_V,
                             (const double *)c->d_Vinv, (const float *)c->d_Dth32,
                             (const int *)c->d_Dnz, (float *)c->d_gseg);
  c->launches++;
  return e;
}

}  // namespace epoch
