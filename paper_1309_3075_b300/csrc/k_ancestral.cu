// k_ancestral.cu -- marginal posterior of every internal node's state, per
// pattern, from the two passes of a gradient evaluation.  With L_u the
// post-order partials (Eq. partial_likelihood, scaled) and U_u the
// normalised outside partials of the adjoint pass (U_root(c,i) = w_c pi_i /
// site), Pr(x_u = i | data_p) = sum_c U_u(c,p,i) L_u(c,p,i): both vectors
// carry the same scale factors that the site value divides out, so the sum
// over (c, i) is 1.  It is divided out all the same, to absorb rounding.
// Not in the paper (an adjacent use of the adjoint pass).
#include "epoch_internal.cuh"

namespace epoch {
namespace {

// One thread per (internal node, pattern).  On the FP32 K = 4 path the
// cherries' partials are not stored: their L is the code-pair table entry.
template <typename T>
__global__ void k_ancestral(Dims d, const T *__restrict__ part, const T *__restrict__ pre,
                            int root, const double *__restrict__ pi,
                            const double *__restrict__ catw, const int *__restrict__ child,
                            const uint8_t *__restrict__ tips, const float *__restrict__ pairL,
                            double *__restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)(d.N - 1) * d.P) return;
  const int slot = (int)(idx / d.P), p = (int)(idx % d.P);
  const int u = slot + d.N;
  int pair = -1;
  if (pairL) {
    const int a = child[2 * slot], b = child[2 * slot + 1];
    if (a < d.N && b < d.N && u != root)
      pair = tips[(size_t)a * d.Pp + p] * d.NR + tips[(size_t)b * d.Pp + p];
  }
  double tot = 0.0;
  for (int pass = 0; pass < 2; pass++) {
    for (int i = 0; i < d.K; i++) {
      double x = 0.0;
      for (int c = 0; c < d.C; c++) {
        const size_t row = (((size_t)slot * d.C + c) * d.P + p) * d.Kp;
        const double l = pair >= 0
                             ? (double)pairL[((((size_t)u * d.C + c) * d.NR * d.NR) + pair) * 4 + i]
                             : (double)part[row + i];
        const double uu = (u == root) ? catw[c] * pi[i] : (double)pre[row + i];
        x += uu * l;
      }
      if (pass == 0)
        tot += x;
      else
        out[idx * d.K + i] = tot > 0.0 ? x / tot : 0.0;
    }
  }
}

}  // namespace

cudaError_t launch_ancestral(epoch_ctx *c, double *d_out) {
  const Dims &d = c->d;
  const long long n = (long long)(d.N - 1) * d.P;
  int root = -1;
  for (int v = 0; v < d.nn; v++)
    if (c->h_parent[v] < 0) root = v;
  const float *pairL = fast_k4(c) ? reinterpret_cast<const float *>(c->d_pairL) : nullptr;
  if (c->precision == EPOCH_FP64)
    k_ancestral<double><<<ceil_div(n, 256), 256, 0, c->stream>>>(
        d, (const double *)c->d_part, (const double *)c->d_pre, root, c->d_pi, c->d_catw,
        c->d_child, c->d_tips, nullptr, d_out);
  else
    k_ancestral<float><<<ceil_div(n, 256), 256, 0, c->stream>>>(
        d, (const float *)c->d_part, (const float *)c->d_pre, root, c->d_pi, c->d_catw,
        c->d_child, c->d_tips, pairL, d_out);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace epoch
