// branch_table.cuh -- device views of the branch matrices and the per-state
// helpers shared by the generic (any K) pruning and adjoint kernels.
#pragma once

#include <math.h>

#include "epoch_internal.cuh"

namespace epoch {

template <typename T>
struct BranchTable;

// FP64: row-major P64[v][c][i][j]; a tip row sums the columns its code allows.
template <>
struct BranchTable<double> {
  const double *P;
  const unsigned long long *masks;
  __device__ double mat(const Dims &d, int v, int c, int i, int j) const {
    return P[((size_t)v * d.C + c) * d.KK + i * d.K + j];
  }
  __device__ double tip(const Dims &d, int v, int c, int i, int code) const {
    const double *row = P + ((size_t)v * d.C + c) * d.KK + i * d.K;
    if (code < d.K) return row[code];
    unsigned long long mk = (code == d.K) ? ~0ull : masks[code - d.K - 1];
    double s = 0.0;
    for (int j = 0; j < d.K; j++)
      if ((mk >> j) & 1ull) s += row[j];
    return s;
  }
};

// FP32: transposed table PT32[v][c][row][Kp], row j < K = column j of P,
// rows K.. = missing / mask sums.
template <>
struct BranchTable<float> {
  const float *PT;
  const unsigned long long *masks;
  __device__ float mat(const Dims &d, int v, int c, int i, int j) const {
    return PT[(((size_t)v * d.C + c) * d.NR + j) * d.Kp + i];
  }
  __device__ float tip(const Dims &d, int v, int c, int i, int code) const {
    return PT[(((size_t)v * d.C + c) * d.NR + code) * d.Kp + i];
  }
};

// Whether tip code `code` allows state j (observed, missing, or a mask).
__device__ __forceinline__ bool code_allows(const Dims &d, const unsigned long long *masks,
                                            int code, int j) {
  if (code < d.K) return code == j;
  if (code == d.K) return true;
  return (masks[code - d.K - 1] >> j) & 1ull;
}

// S_x(c,p,i) = sum_j P_x[i][j] L_x(c,p,j) for child x (tip: from its code).
template <typename T>
__device__ __forceinline__ T child_factor(const Dims &d, const BranchTable<T> &bt,
                                          const T *__restrict__ part,
                                          const uint8_t *__restrict__ tips, int x, int c,
                                          int p, int i) {
  if (x < d.N) return bt.tip(d, x, c, i, tips[(size_t)x * d.Pp + p]);
  const T *L = part + (((size_t)(x - d.N) * d.C + c) * d.P + p) * d.Kp;
  T s = 0;
  for (int j = 0; j < d.K; j++) s += bt.mat(d, x, c, i, j) * L[j];
  return s;
}

// Exact power-of-two rescaling: x * 2^-e, and the binary exponent e of a
// finite m > 0 (m = f 2^e with f in [0.5, 1), as frexp gives it).
__device__ __forceinline__ double scale_by(double x, int e) { return ldexp(x, -e); }
__device__ __forceinline__ float scale_by(float x, int e) { return ldexpf(x, -e); }
__device__ __forceinline__ int exp_of(double m) { return ilogb(m) + 1; }
__device__ __forceinline__ int exp_of(float m) { return ilogbf(m) + 1; }

}  // namespace epoch
