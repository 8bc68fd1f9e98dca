// k_small.cu -- the whole tree in one launch per pass when the patterns are
// few: a discrete trait (one pattern, as in the paper's seasonal
// phylogeography), or a handful of replicate traits.  With one launch per
// post-order level the evaluation would be bound by launch latency (tens of
// levels, two passes, a few kernels each); here one CTA per pattern walks
// every level with a block barrier in between.
//
// A node's values over (category, state) sit in one aligned group of g lanes
// of a warp (g = C * Kp rounded up to a power of two, at most 32), lane
// c * Kp + i holding state i of category c.  The rescaling maximum (Eq.
// partial_likelihood followed by the per-pattern power-of-two scaling), the
// adjoint product U_v = P_v^T X_v and the branch adjoint G_v = n_p X_v (x) L_v
// then need only shuffles inside the group.  Results and layouts are those of
// the per-level kernels (k_partials.cu, k_adjoint.cu): partials, exponents and
// outside partials in the same buffers, G terms per (branch, pattern) reduced
// by k_G_reduce in a fixed order, so the chain rule is shared.
#include <math.h>

#include "branch_table.cuh"

namespace epoch {
namespace {

constexpr int kSmallThreads = 1024;

// Shared-memory image of one pattern's tree: topology (level order), tip
// codes, exponents and the partials of every internal node, so that a level
// waits on global memory only for its branch-matrix rows; and, when they fit
// too, those rows as well (layout sized by small_smem_bytes).
template <typename T>
struct SmallSmem {
  T *mat;       // [N-1][C][K][K] P of the branch above each internal node (tables)
  T *tiprow;    // [N][C][K] the P row set a tip's code selects (tables)
  T *part;      // [N-1][C*Kp] post-order partials of this pattern
  T *pre;       // [N-1][C*Kp] outside partials (pre-order kernel only)
  int *nodes;   // [N-1] internal nodes, level-ascending
  int *child;   // [N-1][2]
  int *escale;  // [N-1] exponents of this pattern
  int *off;     // [L+1] level offsets into nodes (L <= N-1)
  uint8_t *code;  // [N] tip codes of this pattern
  bool tabs;
  __device__ SmallSmem(unsigned char *raw, const Dims &d, bool with_pre, bool tables)
      : tabs(tables) {
    const size_t nv = (size_t)(d.N - 1) * d.C * d.Kp;
    mat = reinterpret_cast<T *>(raw);
    tiprow = mat + (tables ? (size_t)(d.N - 1) * d.C * d.KK : 0);
    part = tiprow + (tables ? (size_t)d.N * d.C * d.K : 0);
    pre = part + nv;
    nodes = reinterpret_cast<int *>(pre + (with_pre ? nv : 0));
    child = nodes + (d.N - 1);
    escale = child + 2 * (d.N - 1);
    off = escale + (d.N - 1);
    code = reinterpret_cast<uint8_t *>(off + d.N);
  }
};

// Load topology and tip codes into shared memory (every thread).
template <typename T>
__device__ void stage_topology(const Dims &d, SmallSmem<T> &sm, const int *__restrict__ lvl_nodes,
                               const int *__restrict__ lvl_off, int L,
                               const int *__restrict__ child, const uint8_t *__restrict__ tips,
                               int p) {
  for (int l = threadIdx.x; l <= L; l += blockDim.x) sm.off[l] = lvl_off[l];
  for (int k = threadIdx.x; k < d.N - 1; k += blockDim.x) {
    sm.nodes[k] = lvl_nodes[k];
    sm.child[2 * k] = child[2 * k];
    sm.child[2 * k + 1] = child[2 * k + 1];
  }
  for (int v = threadIdx.x; v < d.N; v += blockDim.x) sm.code[v] = tips[(size_t)v * d.Pp + p];
}

// The branch matrices every level will read, in one batch of loads (after
// stage_topology and a barrier: the tip rows depend on the codes).
template <typename T>
__device__ void stage_tables(const Dims &d, SmallSmem<T> &sm, const BranchTable<T> &bt) {
  if (!sm.tabs) return;
  const int CKK = d.C * d.KK, CK = d.C * d.K;
  for (int e = threadIdx.x; e < (d.N - 1) * CKK; e += blockDim.x) {
    const int slot = e / CKK, r = e % CKK, c = r / d.KK, ij = r % d.KK;
    sm.mat[e] = bt.mat(d, slot + d.N, c, ij / d.K, ij % d.K);
  }
  for (int e = threadIdx.x; e < d.N * CK; e += blockDim.x) {
    const int x = e / CK, r = e % CK;
    sm.tiprow[e] = bt.tip(d, x, r / d.K, r % d.K, sm.code[x]);
  }
}
// P_x[i][j] for an internal node x (from the tables when they are staged)
template <typename T>
__device__ __forceinline__ T mat_sm(const Dims &d, const BranchTable<T> &bt,
                                    const SmallSmem<T> &sm, int x, int c, int i, int j) {
  if (sm.tabs) return sm.mat[(((size_t)(x - d.N) * d.C + c) * d.K + i) * d.K + j];
  return bt.mat(d, x, c, i, j);
}

// S_x(c, i) = sum_j P_x[i][j] L_x(c, j) with L_x from shared memory (tip:
// the table row of its code).
template <typename T>
__device__ __forceinline__ T child_factor_sm(const Dims &d, const BranchTable<T> &bt,
                                             const SmallSmem<T> &sm, int x, int c, int i) {
  if (x < d.N)
    return sm.tabs ? sm.tiprow[((size_t)x * d.C + c) * d.K + i] : bt.tip(d, x, c, i, sm.code[x]);
  const T *L = sm.part + ((size_t)(x - d.N) * d.C + c) * d.Kp;
  T s = 0;
  for (int j = 0; j < d.K; j++) s += mat_sm(d, bt, sm, x, c, i, j) * L[j];
  return s;
}

// Post-order pruning with rescaling over all levels, then the root sum of
// the CTA's pattern: site_p = sum_c w_c sum_i pi_i L_root(c,p,i) (scaled) and
// lnL_p = log site_p + ln2 * sum_u e_u(p).
template <typename T>
__global__ void __launch_bounds__(kSmallThreads)
    k_small_post(Dims d, BranchTable<T> bt, const int *__restrict__ lvl_nodes,
                 const int *__restrict__ lvl_off, int L, const int *__restrict__ child,
                 T *__restrict__ part, int16_t *__restrict__ scale,
                 const uint8_t *__restrict__ tips, int gsz, const double *__restrict__ pi,
                 const double *__restrict__ catw, double *__restrict__ site_lnl,
                 double *__restrict__ site_inv, int *__restrict__ status, int tables) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_esum;
  __shared__ double s_site;
  const int p = blockIdx.x;
  SmallSmem<T> sm(smraw, d, false, tables != 0);
  stage_topology<T>(d, sm, lvl_nodes, lvl_off, L, child, tips, p);
  if (threadIdx.x == 0) s_esum = 0;
  __syncthreads();
  stage_tables<T>(d, sm, bt);
  __syncthreads();
  const int lane_g = threadIdx.x & (gsz - 1), grp = threadIdx.x / gsz;
  const int ngrp = blockDim.x / gsz;
  const int c = lane_g / d.Kp, i = lane_g % d.Kp;
  const bool holds = c < d.C;           // lane maps to a stored entry
  const bool act = holds && i < d.K;    // ... and to a real state
  int esum = 0;                         // lane 0 of a group: its nodes' exponents
  for (int l = 0; l < L; l++) {
    const int o0 = sm.off[l], o1 = sm.off[l + 1];
    // the trip count is the same for every thread: whole warps take part in
    // the shuffles, groups past the level's end carry zeros
    for (int base = o0; base < o1; base += ngrp) {
      const int k = base + grp;
      const bool node = k < o1;
      int slot = 0;
      T val = 0;
      if (node) {
        slot = sm.nodes[k] - d.N;
        if (act)
          val = child_factor_sm<T>(d, bt, sm, sm.child[2 * slot], c, i) *
                child_factor_sm<T>(d, bt, sm, sm.child[2 * slot + 1], c, i);
      }
      T m = val;
      for (int o = gsz >> 1; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o, gsz));
      if (node) {
        int e = 0;
        if (!isfinite(m)) {
          if (lane_g == 0) atomicOr(status, ST_NONFINITE);
        } else if (m > 0) {
          e = exp_of(m);
          val = scale_by(val, e);
        }
        if (holds) {
          sm.part[((size_t)slot * d.C + c) * d.Kp + i] = val;
          part[(((size_t)slot * d.C + c) * d.P + p) * d.Kp + i] = val;
        }
        if (lane_g == 0) {
          scale[(size_t)slot * d.Pp + p] = (int16_t)e;
          esum += e;
        }
      }
    }
    __syncthreads();  // this level's partials are read by the next
  }
  if (esum) atomicAdd(&s_esum, esum);  // integer sum: exact in any order
  // the root is the single node of the last level
  const int rslot = sm.nodes[sm.off[L - 1]] - d.N;
  if (threadIdx.x < 32) {
    // one warp: lane t sums entries t, t+32, .. of (c, i); then a fixed tree
    double acc = 0.0;
    for (int t = threadIdx.x; t < d.C * d.K; t += 32) {
      const int cc = t / d.K, ii = t % d.K;
      acc += catw[cc] * pi[ii] * (double)sm.part[((size_t)rslot * d.C + cc) * d.Kp + ii];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) s_site = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double site = s_site;
    site_lnl[p] = log(site) + 0.69314718055994530942 * (double)s_esum;
    site_inv[p] = site > 0.0 ? 1.0 / site : 0.0;
  }
}

// lnL = sum_p n_p lnL_p over the (few) patterns, in a fixed order.
__global__ void k_small_lnl(int P, const double *__restrict__ pw,
                            const double *__restrict__ site_lnl, double *__restrict__ out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) t += pw[p] != 0.0 ? pw[p] * site_lnl[p] : 0.0;
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
    out[0] = s;
  }
}

// Pre-order adjoint over all levels, top down, for the CTA's pattern: for
// each child v of u (sibling w)
//   X_v = U_u o S_w 2^{-e_u}   (U_root = w_c pi_i / site_p),
//   U_v = P_v^T X_v            (internal v: kept in shared memory and stored),
//   Gs[slot(u)][p][x][c][i][j] = n_p X_v(c,i) L_v(c,p,j)
// (L_v of a tip is the indicator of its code).
template <typename T>
__global__ void __launch_bounds__(kSmallThreads)
    k_small_pre(Dims d, BranchTable<T> bt, const int *__restrict__ lvl_nodes,
                const int *__restrict__ lvl_off, int L, const int *__restrict__ child, int root,
                const T *__restrict__ part, T *__restrict__ pre, const int16_t *__restrict__ scale,
                const uint8_t *__restrict__ tips, const unsigned long long *__restrict__ masks,
                const double *__restrict__ pi, const double *__restrict__ catw,
                const double *__restrict__ site_inv, const double *__restrict__ pw, int gsz,
                T *__restrict__ Gs, int tables) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int p = blockIdx.x;
  SmallSmem<T> sm(smraw, d, true, tables != 0);
  stage_topology<T>(d, sm, lvl_nodes, lvl_off, L, child, tips, p);
  __syncthreads();
  stage_tables<T>(d, sm, bt);
  const int CKp = d.C * d.Kp;
  for (int e = threadIdx.x; e < (d.N - 1) * CKp; e += blockDim.x) {
    const int slot = e / CKp, r = e % CKp;  // r = c * Kp + i
    sm.part[e] = part[(((size_t)slot * d.C + r / d.Kp) * d.P + p) * d.Kp + r % d.Kp];
  }
  for (int k = threadIdx.x; k < d.N - 1; k += blockDim.x) sm.escale[k] = scale[(size_t)k * d.Pp + p];
  __syncthreads();
  const int lane_g = threadIdx.x & (gsz - 1), grp = threadIdx.x / gsz;
  const int ngrp = blockDim.x / gsz;
  const int c = lane_g / d.Kp, i = lane_g % d.Kp;
  const bool holds = c < d.C;
  const bool act = holds && i < d.K;
  const T n = (T)pw[p];
  const T uroot = act ? (T)(catw[c] * pi[i] * site_inv[p]) : (T)0;
  for (int l = L - 1; l >= 0; l--) {
    const int o0 = sm.off[l], items = 2 * (sm.off[l + 1] - o0);
    for (int base = 0; base < items; base += ngrp) {
      const int it = base + grp;
      const bool node = it < items;
      const int x = it & 1;
      int slot = 0, v = 0;
      T X = 0;
      if (node) {
        const int u = sm.nodes[o0 + (it >> 1)];
        slot = u - d.N;
        v = sm.child[2 * slot + x];
        if (act) {
          const int w = sm.child[2 * slot + 1 - x];
          const T uu = (u == root) ? uroot : sm.pre[((size_t)slot * d.C + c) * d.Kp + i];
          X = scale_by(uu * child_factor_sm<T>(d, bt, sm, w, c, i), sm.escale[slot]);
        }
      }
      // U_v(c, i) = sum_k P_v[k][i] X_v(c, k); X_v(c, k) is in lane c*Kp + k
      const bool inner = node && v >= d.N;
      T U = 0;
      for (int k = 0; k < d.K; k++) {
        const T xk = __shfl_sync(0xffffffffu, X, c * d.Kp + k, gsz);
        if (inner && act) U += mat_sm(d, bt, sm, v, c, k, i) * xk;
      }
      if (inner && holds) {  // read by the next level; kept for the ancestral states
        sm.pre[((size_t)(v - d.N) * d.C + c) * d.Kp + i] = U;
        pre[(((size_t)(v - d.N) * d.C + c) * d.P + p) * d.Kp + i] = U;
      }
      if (node && act) {
        T *g = Gs + ((((size_t)slot * d.P + p) * 2 + x) * d.C + c) * d.KK + (size_t)i * d.K;
        if (v >= d.N) {
          const T *Lv = sm.part + ((size_t)(v - d.N) * d.C + c) * d.Kp;
          for (int j = 0; j < d.K; j++) g[j] = n * X * Lv[j];
        } else {
          const int code = sm.code[v];
          for (int j = 0; j < d.K; j++) g[j] = code_allows(d, masks, code, j) ? n * X : (T)0;
        }
      }
    }
    __syncthreads();  // this level's U are read by the next
  }
}

int group_size(const Dims &d) {
  int g = 1;
  while (g < d.C * d.Kp) g <<= 1;
  return g;
}

int root_node(const epoch_ctx *c) {
  for (int v = 0; v < c->d.nn; v++)
    if (c->h_parent[v] < 0) return v;
  return -1;
}

}  // namespace

cudaError_t launch_small_post(epoch_ctx *c) {
  const Dims &d = c->d;
  const int L = (int)c->h_level_off.size() - 1;
  const int g = group_size(d);
  const size_t es = c->precision == EPOCH_FP64 ? sizeof(double) : sizeof(float);
  // stage the branch matrices too when the pre-order kernel's image fits
  const int tabs = small_smem_bytes(d, d.N, es, true, true) <= kSmallMaxSmem ? 1 : 0;
  const size_t smem = small_smem_bytes(d, d.N, es, false, tabs != 0);
  if (c->precision == EPOCH_FP64) {
    cudaFuncSetAttribute(k_small_post<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_small_post<double><<<d.P, kSmallThreads, smem, c->stream>>>(
        d, BranchTable<double>{c->d_P64, c->d_masks}, c->d_level_nodes, c->d_level_off, L,
        c->d_child, (double *)c->d_part, c->d_scale, c->d_tips, g, c->d_pi, c->d_catw,
        c->d_site_lnl, c->d_site_inv, c->d_status, tabs);
  } else {
    cudaFuncSetAttribute(k_small_post<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_small_post<float><<<d.P, kSmallThreads, smem, c->stream>>>(
        d, BranchTable<float>{c->d_PT32, c->d_masks}, c->d_level_nodes, c->d_level_off, L,
        c->d_child, (float *)c->d_part, c->d_scale, c->d_tips, g, c->d_pi, c->d_catw,
        c->d_site_lnl, c->d_site_inv, c->d_status, tabs);
  }
  k_small_lnl<<<1, 256, 0, c->stream>>>(d.P, c->d_pw, c->d_site_lnl, c->d_lnl);
  c->launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_small_pre(epoch_ctx *c) {
  const Dims &d = c->d;
  const int L = (int)c->h_level_off.size() - 1;
  const int g = group_size(d), root = root_node(c);
  const size_t es = c->precision == EPOCH_FP64 ? sizeof(double) : sizeof(float);
  const int tabs = small_smem_bytes(d, d.N, es, true, true) <= kSmallMaxSmem ? 1 : 0;
  const size_t smem = small_smem_bytes(d, d.N, es, true, tabs != 0);
  if (c->precision == EPOCH_FP64) {
    cudaFuncSetAttribute(k_small_pre<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_small_pre<double><<<d.P, kSmallThreads, smem, c->stream>>>(
        d, BranchTable<double>{c->d_P64, c->d_masks}, c->d_level_nodes, c->d_level_off, L,
        c->d_child, root, (const double *)c->d_part, (double *)c->d_pre, c->d_scale, c->d_tips,
        c->d_masks, c->d_pi, c->d_catw, c->d_site_inv, c->d_pw, g, (double *)c->d_Gpart, tabs);
  } else {
    cudaFuncSetAttribute(k_small_pre<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_small_pre<float><<<d.P, kSmallThreads, smem, c->stream>>>(
        d, BranchTable<float>{c->d_PT32, c->d_masks}, c->d_level_nodes, c->d_level_off, L,
        c->d_child, root, (const float *)c->d_part, (float *)c->d_pre, c->d_scale, c->d_tips,
        c->d_masks, c->d_pi, c->d_catw, c->d_site_inv, c->d_pw, g, (float *)c->d_Gpart, tabs);
  }
  c->launches++;
  return cudaGetLastError();
}

}  // namespace epoch
