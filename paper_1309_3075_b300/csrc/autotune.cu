// autotune.cu -- EPOCH_FP32_AUTO: the choice between the two FP32 paths
// (SIMT contractions, EPOCH_FP32; tcgen05 tile products, EPOCH_FP32_TC) made
// by timing both on the device, once per shape.
//
// The paper's method applies to any finite state space (Introduction), and
// where the dense contraction of a partials update starts to pay on the
// tensor cores depends on K (tile width 16, 32 or 64 after padding), on the
// categories and on the pattern count.  Rather than a fixed K threshold, the
// first context created with EPOCH_FP32_AUTO for a (K, C, pattern-count
// bucket) builds a synthetic problem of that shape (a random binary tree of
// up to 64 taxa, a random reversible Q per epoch with uniform pi and one
// parameter derivative, random tip codes), evaluates lnL + gradient on each
// path through this library's own entry points (graph replays timed with
// CUDA events after warm-up) and caches the fastest for the process.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

struct Probe {
  int precision;
  double ms_simt, ms_tc, ms_bf;
};
std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, Probe> g_cache;  // (device, K, C, pattern bucket)

// A small deterministic generator (xorshift64*): the probe's inputs need no
// statistical quality, only to be the same on every run.
struct Rng {
  uint64_t s;
  double u() {
    s ^= s >> 12;
    s ^= s << 25;
    s ^= s >> 27;
    return (double)((s * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0);
  }
};

// Time one lnL + gradient evaluation (ms) on a fresh context of the given
// precision, or a negative value if the path could not run.
double time_path(int prec, int K, int C, int P, int N, int E, const std::vector<double> &b,
                 const std::vector<double> &Q, const std::vector<double> &dQ,
                 const std::vector<double> &pi, const std::vector<double> &heights,
                 const std::vector<int> &parent, const std::vector<int> &codes,
                 const std::vector<double> &w, cudaStream_t stream) {
  epoch_ctx *c = nullptr;
  if (epoch_create(&c, K, E, E > 1 ? b.data() : nullptr, nullptr, E, N, P, C, prec, stream) !=
      EPOCH_OK)
    return -1.0;
  std::vector<double> rates(C), cw(C, 1.0 / C);
  for (int k = 0; k < C; k++) rates[k] = (k + 0.5) * 2.0 / C;
  double ms = -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = epoch_set_rate_matrices(c, Q.data(), pi.data(), 1, 1) == EPOCH_OK &&
            epoch_set_rate_derivatives(c, 1, dQ.data()) == EPOCH_OK &&
            epoch_set_categories(c, rates.data(), cw.data()) == EPOCH_OK &&
            epoch_set_tree(c, N, heights.data(), parent.data(), nullptr) == EPOCH_OK &&
            epoch_set_tip_data(c, codes.data(), w.data()) == EPOCH_OK &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (ok) {
    for (int r = 0; r < 3 && ok; r++) ok = epoch_evaluate_async(c, 1) == EPOCH_OK;
    const int reps = 5;
    ok = ok && cudaEventRecord(e0, c->stream) == cudaSuccess;
    for (int r = 0; r < reps && ok; r++) ok = epoch_evaluate_async(c, 1) == EPOCH_OK;
    ok = ok && cudaEventRecord(e1, c->stream) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess;
    double lnl = 0.0;
    ok = ok && epoch_read_results(c, &lnl, nullptr, nullptr, nullptr, nullptr) == EPOCH_OK;
    float f = 0.f;
    if (ok && cudaEventElapsedTime(&f, e0, e1) == cudaSuccess) ms = f / reps;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  epoch_destroy(c);
  return ms;
}

}  // namespace

// The path EPOCH_FP32_AUTO resolves to for this shape (EPOCH_FP32,
// EPOCH_FP32_TC or EPOCH_FP32_TC_BF16), with the probe's times; probes once
// per (device, K, C, pattern bucket).  Shapes the tensor-core paths do not
// take resolve to EPOCH_FP32 without a probe.
int resolve_auto(int K, int E, int C, int P, int max_taxa, cudaStream_t stream, double *ms_simt,
                 double *ms_tc, double *ms_bf) {
  *ms_simt = *ms_tc = *ms_bf = -1.0;
  if (K <= 8 || K > 64 || C > 4) return EPOCH_FP32;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EPOCH_FP32;
  int bucket = 0;
  while ((128 << bucket) < P && bucket < 12) bucket++;
  const auto key = std::make_tuple(dev, K, C, bucket);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *ms_simt = it->second.ms_simt;
      *ms_tc = it->second.ms_tc;
      *ms_bf = it->second.ms_bf;
      return it->second.precision;
    }
  }
  const int N = std::max(2, std::min(max_taxa, 64));
  const int Pp = std::min(P, 128 << bucket);
  E = std::max(1, std::min(E, 4));
  Rng rng{0x9E3779B97F4A7C15ull ^ ((uint64_t)K << 32) ^ (uint64_t)(C * 131 + bucket)};
  // tree: join random pairs of lineages at increasing heights (root 1)
  const int nn = 2 * N - 1;
  std::vector<double> heights(nn, 0.0);
  std::vector<int> parent(nn, -1), live;
  for (int v = 0; v < N; v++) live.push_back(v);
  double h = 0.0;
  for (int u = N; u < nn; u++) {
    h += 0.5 + rng.u();
    const int i = (int)(rng.u() * live.size()) % (int)live.size();
    const int a = live[i];
    live.erase(live.begin() + i);
    const int j = (int)(rng.u() * live.size()) % (int)live.size();
    const int bb = live[j];
    live.erase(live.begin() + j);
    parent[a] = parent[bb] = u;
    heights[u] = h;
    live.push_back(u);
  }
  for (int u = N; u < nn; u++) heights[u] /= h;
  std::vector<double> b;
  for (int k = 1; k < E; k++) b.push_back((double)k / E);
  // reversible Q per epoch with uniform pi: symmetric exchange rates
  const int KK = K * K;
  std::vector<double> pi(K, 1.0 / K), Q((size_t)E * KK, 0.0), dQ((size_t)E * KK, 0.0);
  for (int e = 0; e < E; e++) {
    double *q = &Q[(size_t)e * KK];
    for (int i = 0; i < K; i++)
      for (int j = i + 1; j < K; j++) q[i * K + j] = q[j * K + i] = (0.2 + rng.u()) / K;
    for (int i = 0; i < K; i++) {
      double s = 0.0;
      for (int j = 0; j < K; j++) s += (i == j) ? 0.0 : q[i * K + j];
      q[i * K + i] = -s;
    }
  }
  dQ[1] = dQ[K] = 1.0 / K;  // d/d theta of the (0, 1) exchange rate of epoch 0
  dQ[0] = dQ[K + 1] = -1.0 / K;
  std::vector<int> codes((size_t)N * Pp);
  for (auto &x : codes) x = (int)(rng.u() * K) % K;
  std::vector<double> w(Pp, 1.0);
  const double ms_s = time_path(EPOCH_FP32, K, C, Pp, N, E, b, Q, dQ, pi, heights, parent, codes, w, stream);
  const double ms_t = time_path(EPOCH_FP32_TC, K, C, Pp, N, E, b, Q, dQ, pi, heights, parent, codes, w, stream);
  const double ms_b = time_path(EPOCH_FP32_TC_BF16, K, C, Pp, N, E, b, Q, dQ, pi, heights, parent, codes, w, stream);
  cudaGetLastError();
  Probe pr{EPOCH_FP32, ms_s, ms_t, ms_b};
  double best = ms_s > 0.0 ? ms_s : 1e300;
  if (ms_t > 0.0 && ms_t < best) {
    best = ms_t;
    pr.precision = EPOCH_FP32_TC;
  }
  if (ms_b > 0.0 && ms_b < best) pr.precision = EPOCH_FP32_TC_BF16;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = pr;
  }
  *ms_simt = ms_s;
  *ms_tc = ms_t;
  *ms_bf = ms_b;
  return pr.precision;
}

}  // namespace epoch
