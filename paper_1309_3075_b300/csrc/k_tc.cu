// k_tc.cu -- tensor-core contractions of the larger state spaces (codon
// K = 61, amino acids K = 20, traits; 8 < K <= 64): tcgen05.mma with the
// accumulator in tensor memory.
//
// A partial vector of one (category, pattern) is a row of KW floats (K
// padded with zeros; KW = 64 for 32 < K <= 64, 32 for 16 < K <= 32, 16 for
// 8 < K <= 16), so a branch applied to 128 patterns is one tile product
//     D[128 x KW] = A[128 x KW] * B^T,   B[n][k] = P[n][k] (S = P L)
//                                        or  B[n][k] = P[k][n] (U = P^T X),
// run on the tensor cores in one of two operand formats, both accumulated
// in FP32 in tensor memory (M = 128, N = KW):
//  * TF32 x 3 (EPOCH_FP32_TC): tcgen05.mma kind::tf32, K = 8 per
//    instruction.  x = hi + lo (hi = x rounded to TF32, lo = the rest
//    rounded to TF32): A B ~ Ahi Bhi + Ahi Blo + Alo Bhi; the dropped Alo Blo
//    is below 2^-22 of the product.
//  * BF16 x 3 (EPOCH_FP32_TC_BF16): kind::f16 with BF16 A and B, K = 16 per
//    instruction.  x = x1 + x2 + x3, each the rest so far rounded to BF16 (8
//    significant bits each, 24 in all): A B ~ A1 B1 + A1 B2 + A2 B1 + A1 B3
//    + A2 B2 + A3 B1; the dropped terms are below 2^-23 of the product.
//
// Operands sit in shared memory in the no-swizzle K-major canonical layout:
// 8-row x 16-byte core matrices (4 TF32 or 8 BF16 along K), element (r, k)
// at byte
//     TF32: (r / 8) * 32 KW + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4,
//     BF16: (r / 8) * 16 KW + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// i.e. leading-dimension (K) byte offset 128 between core matrices and
// stride-dimension byte offset 32 KW (TF32) or 16 KW (BF16) between 8-row
// groups.  The B operands of every (branch, category) are laid out once per
// evaluation (k_tc_prep).
#include <stdint.h>

#include <type_traits>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

constexpr int kRows = 128;            // tile rows (patterns)
constexpr int kTcThr = 128;           // one thread per row; warp w owns TMEM lanes 32w..

// Sizes for the tile width KW and operand format (BF: BF16 x 3, else TF32 x
// 3), in bytes unless named in floats.
template <int KW, bool BF>
struct Tw {
  static constexpr int ES = BF ? 2 : 4;           // bytes per operand element
  static constexpr int NP = BF ? 3 : 2;           // planes of the split
  static constexpr int A = kRows * KW * ES;       // one 128 x KW operand plane
  static constexpr int B = KW * KW * ES;          // one KW x KW operand plane
  static constexpr int stage = NP * A + NP * B;   // A planes, then B planes
  static constexpr int c4 = KW / 4;               // float4 per FP32 row
  static constexpr int pad = KW + 4;              // row-buffer stride in floats (bank spread)
  static constexpr int buf = kRows * pad;         // one FP32 row buffer, in floats
  static constexpr int kstep = BF ? 16 : 8;       // K per instruction
  static constexpr int sbo = BF ? 16 * KW : 32 * KW;  // 8-row group stride
  // B operands of one (branch, category) in tcB: [post planes | pre planes]
  static constexpr int vc_floats = 4 * KW * KW;   // per (v, c) stride, either format
};

template <int KW, bool BF>
__device__ __forceinline__ int core_off(int r, int k) {  // in bytes
  return BF ? (r >> 3) * (16 * KW) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2
            : (r >> 3) * (32 * KW) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// x rounded to BF16 (nearest even): the bits, and the value as FP32
__device__ __forceinline__ uint16_t to_bf16(float x, float &back) {
  uint16_t h;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
  back = __uint_as_float((uint32_t)h << 16);
  return h;
}
// The three BF16 parts of x (x1 + x2 + x3 ~ x to 2^-24).
__device__ __forceinline__ void split3(float x, uint16_t &a, uint16_t &b, uint16_t &c) {
  float v;
  a = to_bf16(x, v);
  const float r1 = x - v;
  b = to_bf16(r1, v);
  c = to_bf16(r1 - v, v);
}
// x * 2^-e for the binary exponent e of a value in (0, 2] (e in [-148, 1]),
// exactly: one multiply by 2^-e when -e <= 126, else 2^126 then 2^(-e-126).
struct Pow2 {
  float a, b;
};
__device__ __forceinline__ Pow2 pow2_neg(int e) {
  if (e >= -126) return {__int_as_float((127 - e) << 23), 1.f};
  return {__int_as_float(253 << 23), __int_as_float((1 - e) << 23)};
}
__device__ __forceinline__ float sc(float x, Pow2 f) { return (x * f.a) * f.b; }
__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
template <int KW, bool BF>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;              // leading (K) byte offset
  d |= (uint64_t)(Tw<KW, BF>::sbo >> 4) << 32;  // stride (8-row group) byte offset
  d |= (uint64_t)1 << 46;                       // descriptor version; no swizzle, base offset 0
  return d;
}
// D = F32, A = B = TF32 (kind::tf32) or BF16 (kind::f16), both K-major,
// N = KW, M = 128
template <int KW, bool BF>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((BF ? 1u : 2u) << 7) | ((BF ? 1u : 2u) << 10) |
         (((uint32_t)KW >> 3) << 17) | ((128u >> 4) << 24);
}

template <int KW, bool BF>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
  if constexpr (BF)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc<KW, BF>()), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc<KW, BF>()), "r"(acc));
}

// B operands: for every (v, c): [post planes | pre planes], each KW x KW in
// core order; post = P_v (rows = parent state), pre = P_v^T.  TF32: planes
// hi, lo; BF16: the three parts.
template <int KW, bool BF>
__global__ void k_tc_prep(Dims d, const double *__restrict__ P64, const int *__restrict__ parent,
                          float *__restrict__ tcB) {
  using W = Tw<KW, BF>;
  const int v = blockIdx.x / d.C, c = blockIdx.x % d.C;
  if (parent[v] < 0) return;
  const double *P = P64 + ((size_t)v * d.C + c) * d.KK;
  unsigned char *out = reinterpret_cast<unsigned char *>(tcB + ((size_t)v * d.C + c) * W::vc_floats);
  for (int idx = threadIdx.x; idx < KW * KW; idx += blockDim.x) {
    const int r = idx / KW, k = idx % KW;
    const bool in = r < d.K && k < d.K;
    const float vp = in ? (float)P[r * d.K + k] : 0.f;   // post: B[r][k] = P[r][k]
    const float vq = in ? (float)P[k * d.K + r] : 0.f;   // pre:  B[r][k] = P[k][r]
    const int o = core_off<KW, BF>(r, k);
    if constexpr (BF) {
      uint16_t a, b, cc;
      split3(vp, a, b, cc);
      *reinterpret_cast<uint16_t *>(out + o) = a;
      *reinterpret_cast<uint16_t *>(out + W::B + o) = b;
      *reinterpret_cast<uint16_t *>(out + 2 * W::B + o) = cc;
      split3(vq, a, b, cc);
      *reinterpret_cast<uint16_t *>(out + 3 * W::B + o) = a;
      *reinterpret_cast<uint16_t *>(out + 4 * W::B + o) = b;
      *reinterpret_cast<uint16_t *>(out + 5 * W::B + o) = cc;
    } else {
      const float hp = to_tf32(vp), hq = to_tf32(vq);
      *reinterpret_cast<float *>(out + o) = hp;
      *reinterpret_cast<float *>(out + W::B + o) = to_tf32(vp - hp);
      *reinterpret_cast<float *>(out + 2 * W::B + o) = hq;
      *reinterpret_cast<float *>(out + 3 * W::B + o) = to_tf32(vq - hq);
    }
  }
}

// Shared memory: one stage (A planes, B planes), and at least the two FP32
// epilogue row buffers that reuse it, plus room to align the start to 1024
// bytes.
template <int KW, bool BF>
__host__ __device__ constexpr size_t tc_smem() {
  using W = Tw<KW, BF>;
  return (size_t)(W::stage > 8 * W::buf ? W::stage : 8 * W::buf) + 1024;
}

// An A tile in registers.  A warp's load instruction covers 8 rows x 4
// consecutive float4 (64 contiguous bytes of each row: whole sectors); a
// quarter-warp's store covers 8 consecutive rows of one core-matrix column,
// 128 contiguous bytes (no bank conflicts).  With nG = KW / 16 column groups
// of 4 float4, warp w takes group w % nG and every (4 / nG)-th block of 8
// rows from w / nG: thread (w, l) holds, for q < KW / 4, row
// 8 (q (4 / nG) + w / nG) + (l & 7), float4 4 (w % nG) + (l >> 3).
template <int KW>
struct ATile {
  float4 x[KW / 4];
};
template <int KW>
__device__ __forceinline__ void a_pos(int q, int &r, int &col) {
  constexpr int nG = KW / 16, RB = 4 / nG;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  r = 8 * (q * RB + w / nG) + (l & 7);
  col = 4 * (4 * (w % nG) + (l >> 3));
}
// Rows >= rows read as zero.
template <int KW>
__device__ __forceinline__ void tc_load_A(const float *A, int lda, int rows, ATile<KW> &t) {
#pragma unroll
  for (int q = 0; q < KW / 4; q++) {
    int r, col;
    a_pos<KW>(q, r, col);
    t.x[q] = r < rows ? *reinterpret_cast<const float4 *>(A + (size_t)r * lda + col)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}
// The split of an A tile into the stage's A planes, core order (TF32: hi,
// lo; BF16: the three parts).  st: the stage's first byte.
template <int KW, bool BF>
__device__ __forceinline__ void tc_store_A(const ATile<KW> &t, unsigned char *st) {
  using W = Tw<KW, BF>;
#pragma unroll
  for (int q = 0; q < KW / 4; q++) {
    int r, col;
    a_pos<KW>(q, r, col);
    const float4 x = t.x[q];
    const int o = core_off<KW, BF>(r, col);
    if constexpr (BF) {
      uint16_t a[4], b[4], c[4];
      split3(x.x, a[0], b[0], c[0]);
      split3(x.y, a[1], b[1], c[1]);
      split3(x.z, a[2], b[2], c[2]);
      split3(x.w, a[3], b[3], c[3]);
      auto pack = [](const uint16_t (&h)[4]) {
        return make_uint2((uint32_t)h[0] | ((uint32_t)h[1] << 16),
                          (uint32_t)h[2] | ((uint32_t)h[3] << 16));
      };
      *reinterpret_cast<uint2 *>(st + o) = pack(a);
      *reinterpret_cast<uint2 *>(st + W::A + o) = pack(b);
      *reinterpret_cast<uint2 *>(st + 2 * W::A + o) = pack(c);
    } else {
      const float4 h = make_float4(to_tf32(x.x), to_tf32(x.y), to_tf32(x.z), to_tf32(x.w));
      const float4 l = make_float4(to_tf32(x.x - h.x), to_tf32(x.y - h.y), to_tf32(x.z - h.z),
                                   to_tf32(x.w - h.w));
      *reinterpret_cast<float4 *>(st + o) = h;
      *reinterpret_cast<float4 *>(st + W::A + o) = l;
    }
  }
}
// The B planes (laid out by k_tc_prep) into the stage's B area by cp.async,
// as one commit group.
template <int KW, bool BF>
__device__ __forceinline__ void tc_async_B(const float *Bq, unsigned char *st) {
  using W = Tw<KW, BF>;
  const uint32_t dst = su32(st + W::NP * W::A);
  const size_t src = __cvta_generic_to_global(Bq);
#pragma unroll 4
  for (int i = threadIdx.x; i < W::NP * W::B / 16; i += kTcThr)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * i),
                 "l"(src + 16 * (size_t)i)
                 : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// Issue (thread 0) D[col..col+KW-1] = A B^T from stage st with the split
// products (TF32: 3, BF16: 6 per K step), then signal mbar when they have
// completed.  Staged operands must be fenced and the CTA synchronised before
// the call.
template <int KW, bool BF>
__device__ __forceinline__ void tc_mma(uint32_t dtmem, const unsigned char *st, uint64_t *mbar) {
  using W = Tw<KW, BF>;
  if (threadIdx.x != 0) return;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t a0 = su32(st), b0 = a0 + W::NP * W::A;
  for (int ks = 0; ks < KW / W::kstep; ks++) {  // one K step = 2 core matrices = 256 bytes
    const uint32_t o = ks * 256;
    auto mm = [&](int i, int j, uint32_t acc) {
      mma_issue<KW, BF>(dtmem, smem_desc<KW, BF>(a0 + i * W::A + o),
                        smem_desc<KW, BF>(b0 + j * W::B + o), acc);
    };
    mm(0, 0, ks > 0);
    mm(0, 1, 1);
    mm(1, 0, 1);
    if constexpr (BF) {
      mm(0, 2, 1);
      mm(1, 1, 1);
      mm(2, 0, 1);
    }
  }
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(mbar)));
}
__device__ __forceinline__ void tc_sync_staged() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
}
// Waits on an MMA-completion barrier are bounded in time, not in polls: a
// kernel slowed by a profiler's replay must not reach the limit.
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Thread 0 polls mbar for the given phase until it completes or kWaitNs has
// passed on %globaltimer.
__device__ __forceinline__ bool mbar_poll(uint64_t *mbar, uint32_t phase) {
  const uint64_t t0 = gtimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(mbar)), "r"(phase)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > kWaitNs) return false;
  }
}
// Wait for the MMAs signalled on mbar.  One thread polls and publishes the
// outcome in *s_ok, so that every thread of the CTA takes the same branch
// (the tcgen05 loads and the barriers after it are CTA- or warp-collective).
// On success the phase flips.  On failure it does not: the MMA is still in
// flight, and the caller must call tc_drain on the same phase before the CTA
// releases its tensor memory or exits.  Callers separate two calls by a
// __syncthreads, so *s_ok is never rewritten while a thread still reads it.
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t &phase, int *s_ok) {
  if (threadIdx.x == 0) *s_ok = mbar_poll(mbar, phase) ? 1 : 0;
  __syncthreads();
  const bool ok = *s_ok != 0;
  if (ok) phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return ok;
}
// After a timed-out wait: wait once more, again bounded, for the MMA that is
// still in flight, so that its shared-memory operands, its barrier and its
// tensor-memory columns stay valid while it runs.  CTA-collective.
__device__ __forceinline__ void tc_drain(uint64_t *mbar, uint32_t phase) {
  if (threadIdx.x == 0) (void)mbar_poll(mbar, phase);
  __syncthreads();
}
// 64 columns of the thread's TMEM lane (warp w reads lanes 32w..32w+31),
// one load and one wait.
__device__ __forceinline__ void tc_ld64(uint32_t taddr, int col, float *out) {
  uint32_t v[64];
  const uint32_t a = taddr + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16) + col;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
      "%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,"
      "%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
        "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
        "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]),
        "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]),
        "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]),
        "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
        "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]),
        "=r"(v[63])
      : "r"(a));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 64; j++) out[j] = __uint_as_float(v[j]);
}

// 32 columns of the thread's TMEM lane, one load and one wait.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, int col, float *out) {
  uint32_t v[32];
  const uint32_t a = taddr + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16) + col;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
        "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
        "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(a));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; j++) out[j] = __uint_as_float(v[j]);
}
// 16 columns of the thread's TMEM lane, one load and one wait.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, int col, float *out) {
  uint32_t v[16];
  const uint32_t a = taddr + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16) + col;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(a));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; j++) out[j] = __uint_as_float(v[j]);
}
// KW columns of the thread's TMEM lane.
template <int KW>
__device__ __forceinline__ void tc_ld(uint32_t taddr, int col, float *out) {
  if constexpr (KW == 64)
    tc_ld64(taddr, col, out);
  else if constexpr (KW == 32)
    tc_ld32(taddr, col, out);
  else
    tc_ld16(taddr, col, out);
}

// Epilogue row buffers in the (then free) stage memory: 128 rows of KW
// floats, padded to KW + 4 so that the eight rows a quarter-warp writes at
// one column fall in distinct banks.
// Thread r's row of KW values into buffer row r (float4 stores).
template <int KW>
__device__ __forceinline__ void row_put(float *buf, const float (&v)[KW]) {
  float *dst = buf + threadIdx.x * Tw<KW, false>::pad;
#pragma unroll
  for (int q = 0; q < KW / 4; q++)
    *reinterpret_cast<float4 *>(dst + 4 * q) =
        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
// A buffer of `rows` rows to global rows (ld floats apart) with whole-warp
// contiguous float4 stores; each row scaled by 2^-e[row] when e is given.
template <int KW>
__device__ __forceinline__ void rows_store(const float *buf, float *dst, int ld, int rows,
                                           const int *e) {
  constexpr int C4 = Tw<KW, false>::c4;
#pragma unroll 4
  for (int q = 0; q < C4; q++) {
    const int idx = threadIdx.x + kTcThr * q, row = idx / C4, c4 = idx % C4;
    if (row < rows) {
      float4 v = *reinterpret_cast<const float4 *>(buf + row * Tw<KW, false>::pad + 4 * c4);
      if (e) {
        const Pow2 f = pow2_neg(e[row]);
        v = make_float4(sc(v.x, f), sc(v.y, f), sc(v.z, f), sc(v.w, f));
      }
      *reinterpret_cast<float4 *>(dst + (size_t)row * ld + 4 * c4) = v;
    }
  }
}
// Global rows (ld floats apart) into a buffer with contiguous loads; rows >=
// `rows` become zero.
template <int KW>
__device__ __forceinline__ void rows_load(const float *src, int ld, int rows, float *buf) {
  constexpr int C4 = Tw<KW, false>::c4;
#pragma unroll 4
  for (int q = 0; q < C4; q++) {
    const int idx = threadIdx.x + kTcThr * q, row = idx / C4, c4 = idx % C4;
    const float4 v = row < rows ? *reinterpret_cast<const float4 *>(src + (size_t)row * ld + 4 * c4)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4 *>(buf + row * Tw<KW, false>::pad + 4 * c4) = v;
  }
}
// KW floats of a table row (a tip's S: the row of its code).
template <int KW>
__device__ __forceinline__ void row_get(const float *src, float (&v)[KW]) {
#pragma unroll
  for (int q = 0; q < KW / 4; q++) {
    const float4 t = reinterpret_cast<const float4 *>(src)[q];
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
}

// Tile products D_j[128 x KW] = A_j B_j^T into TMEM columns col_j, j < n,
// for one tile of 128 rows (A rows lda floats apart; rows >= `rows` read as
// zero), through one shared-memory stage so that two CTAs fit on an SM:
// item j+1's A is loaded into registers during item j's MMA, its B (by
// cp.async) once that MMA has completed.  item(j, A, B, col) names the
// operands.  Every thread takes part.  (Two stages with one CTA per SM were
// measured slower on the wide levels.)  At most one MMA is in flight at any
// time.  Returns false when an MMA did not complete within the wait bound;
// that MMA has then been drained (a second bounded wait) and no cp.async is
// pending, so the caller may release tensor memory.  The result is the same
// in every thread of the CTA.
template <int KW, bool BF, class Item>
__device__ bool tc_pipeline(int n, int lda, int rows, Item item, unsigned char *st, uint32_t taddr,
                            uint64_t *mbar, uint32_t *ph, int *s_ok) {
  if (n <= 0) return true;
  ATile<KW> ra;
  const float *A, *B;
  uint32_t col;
  item(0, A, B, col);
  tc_async_B<KW, BF>(B, st);
  tc_load_A<KW>(A, lda, rows, ra);
  for (int j = 0; j < n; j++) {
    if (j >= 1) {  // the stage is free once MMA j-1 has completed
      const int b = (j - 1) & 1;
      if (!tc_wait(&mbar[b], ph[b], s_ok)) {
        tc_drain(&mbar[b], ph[b]);
        return false;
      }
      tc_async_B<KW, BF>(B, st);
    }
    tc_store_A<KW, BF>(ra, st);
    const uint32_t colj = col;
    if (j + 1 < n) {
      item(j + 1, A, B, col);
      tc_load_A<KW>(A, lda, rows, ra);  // in flight during this item's MMA
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    tc_sync_staged();
    tc_mma<KW, BF>(taddr + colj, st, &mbar[j & 1]);
  }
  const int b = (n - 1) & 1;
  if (!tc_wait(&mbar[b], ph[b], s_ok)) {
    tc_drain(&mbar[b], ph[b]);
    return false;
  }
  return true;
}

// CTA prologue / epilogue: TMEM columns and the two MMA-completion barriers.
__device__ uint32_t tc_begin(uint32_t *s_tmem, uint64_t *mbar, uint32_t ncols) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(s_tmem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar[1])), "r"(1));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *s_tmem;
}
__device__ void tc_end(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ float *tc_smem(float *tsm) {
  return reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(tsm) + 1023) & ~(uintptr_t)1023);
}
// Pre-order: U_v = P_v^T X_v for the non-tip children of one level's nodes.
// grid = (tiles of 128 patterns, level nodes * 2 children, categories); one
// tile product per CTA (one shared-memory stage).
template <int KW, bool BF>
__global__ void __launch_bounds__(kTcThr) k_tc_pre_u(Dims d, const int *__restrict__ lvl_nodes,
                                                    int lvl_off, const int *__restrict__ child,
                                                    const float *__restrict__ xbuf,
                                                    const float *__restrict__ tcB,
                                                    float *__restrict__ pre, int *status) {
  extern __shared__ __align__(1024) float tsm[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int s_ok;
  const int bi = blockIdx.y >> 1, x = blockIdx.y & 1, c = blockIdx.z;
  const int u = lvl_nodes[lvl_off + bi];
  const int v = child[2 * (u - d.N) + x];
  if (v < d.N) return;  // tips carry no outside partial (uniform over the CTA)
  float *sm = tc_smem(tsm);
  const uint32_t ncols = KW < 32 ? 32 : KW;  // a TMEM allocation is >= 32 columns
  const uint32_t taddr = tc_begin(&s_tmem, mbar, ncols);
  uint32_t ph[2] = {0, 0};
  const int p0 = blockIdx.x * kRows;
  const int rows = min(kRows, d.P - p0);
  auto item = [&](int, const float *&A, const float *&B, uint32_t &col) {
    A = xbuf + ((((size_t)bi * 2 + x) * d.C + c) * d.P + p0) * d.Kp;
    B = tcB + ((size_t)v * d.C + c) * Tw<KW, BF>::vc_floats +
        Tw<KW, BF>::NP * Tw<KW, BF>::B / 4;  // the pre planes
    col = 0;
  };
  if (!tc_pipeline<KW, BF>(1, d.Kp, rows, item, reinterpret_cast<unsigned char *>(sm), taddr,
                           mbar, ph, &s_ok)) {
    if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    tc_end(taddr, ncols);
    return;
  }
  float vv[KW];
  tc_ld<KW>(taddr, 0, vv);
  row_put<KW>(sm, vv);
  __syncthreads();
  rows_store<KW>(sm, pre + ((((size_t)(v - d.N) * d.C + c) * d.P) + p0) * d.Kp, d.Kp, rows,
                 nullptr);
  tc_end(taddr, ncols);
}

// S of both children of node u for category c into TMEM columns sd * KW;
// tips are skipped (their S is a table row).
template <int KW, bool BF>
__device__ __forceinline__ bool tc_children_S(const Dims &d, const int (&kid)[2], int c,
                                              const float *part, const float *tcB, int p0,
                                              int rows, float *sm, uint32_t taddr,
                                              uint64_t *mbar, uint32_t *ph, int *s_ok) {
  const bool st0 = kid[0] >= d.N, st1 = kid[1] >= d.N;
  const int n = (int)st0 + (int)st1;
  auto item = [&](int j, const float *&A, const float *&B, uint32_t &col) {
    const int sd = n == 2 ? j : (st0 ? 0 : 1);
    const int v = kid[sd];
    A = part + ((((size_t)(v - d.N) * d.C + c) * d.P) + p0) * d.Kp;
    B = tcB + ((size_t)v * d.C + c) * Tw<KW, BF>::vc_floats;  // the post planes
    col = (uint32_t)(sd * KW);
  };
  return tc_pipeline<KW, BF>(n, d.Kp, rows, item, reinterpret_cast<unsigned char *>(sm), taddr,
                             mbar, ph, s_ok);
}

// S of child sd (TMEM block sd, or the table row of a tip's code).
template <int KW>
__device__ __forceinline__ void child_S(const Dims &d, const float *PT, int kid, int c, int code,
                                        uint32_t taddr, int sd, float (&v)[KW]) {
  if (kid >= d.N)
    tc_ld<KW>(taddr, sd * KW, v);
  else
    row_get<KW>(PT + (((size_t)kid * d.C + c) * d.NR + code) * d.Kp, v);
}

// Cluster-wide barrier (every CTA of the cluster arrives, then waits).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
// The float at the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ float cluster_ld(const float *p, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(su32(p)), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
  return v;
}

// Post-order level: for node u, category c = blockIdx.z: S of each stored
// child by a tile product (tips: the table row of their code), then
// L_u = S_0 o S_1 rescaled per pattern by 2^-e, e the binary exponent of the
// max over (c, i) (frexp convention).  The C CTAs of a (tile, node) form a
// cluster: each publishes its rows' maxima over i in shared memory and reads
// the others' through distributed shared memory.  grid = (tiles of 128
// patterns, nodes, categories), cluster (1, 1, C).
template <int KW, bool BF>
__global__ void __launch_bounds__(kTcThr) k_tc_post(Dims d, const int *__restrict__ lvl_nodes,
                                                   int lvl_off, const int *__restrict__ child,
                                                   const float *__restrict__ PT,
                                                   const uint8_t *__restrict__ tips,
                                                   const float *__restrict__ tcB, float *part,
                                                   int16_t *__restrict__ scale, int *status) {
  extern __shared__ __align__(1024) float tsm[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int s_ok;
  __shared__ float s_m[kRows];
  __shared__ int s_e[kRows];
  float *sm = tc_smem(tsm);
  const int c = blockIdx.z;
  const int u = lvl_nodes[lvl_off + blockIdx.y];
  const int slot = u - d.N;
  const int kid[2] = {child[2 * slot], child[2 * slot + 1]};
  const uint32_t taddr = tc_begin(&s_tmem, mbar, 2 * KW);
  uint32_t ph[2] = {0, 0};
  const int p0 = blockIdx.x * kRows, rows = min(kRows, d.P - p0);
  const bool ok = tc_children_S<KW, BF>(d, kid, c, part, tcB, p0, rows, sm, taddr, mbar, ph, &s_ok);
  if (!ok && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
  const int r = threadIdx.x, p = p0 + r;
  const bool live = r < rows;
  int code[2] = {0, 0};
  for (int sd = 0; sd < 2; sd++)
    if (kid[sd] < d.N && live) code[sd] = tips[(size_t)kid[sd] * d.Pp + p];
  // unscaled L_u row of this category into the row buffer; its maximum
  float m = 0.f;
  if (ok) {
    float s0[KW], s1[KW];
    child_S<KW>(d, PT, kid[0], c, code[0], taddr, 0, s0);
    child_S<KW>(d, PT, kid[1], c, code[1], taddr, 1, s1);
#pragma unroll
    for (int j = 0; j < KW; j++) {
      s0[j] = j < d.K ? s0[j] * s1[j] : 0.f;
      m = fmaxf(m, s0[j]);
    }
    row_put<KW>(sm, s0);
  }
  s_m[r] = m;
  // every CTA of the cluster takes both barriers, whatever happened above
  cluster_sync();
  for (int q = 0; q < d.C; q++)
    if (q != c) m = fmaxf(m, cluster_ld(&s_m[r], (uint32_t)q));
  cluster_sync();  // the peers' maxima have been read: their CTAs may finish
  int e = 0;
  if (!(m <= 3.0e38f)) {
    if (live) atomicOr(status, ST_NONFINITE);
  } else if (m > 0.f) {
    frexpf(m, &e);
  }
  s_e[r] = e;
  if (live && c == 0) scale[(size_t)slot * d.Pp + p] = (int16_t)e;
  __syncthreads();
  if (ok)
    rows_store<KW>(sm, part + ((((size_t)slot * d.C + c) * d.P) + p0) * d.Kp, d.Kp, rows, s_e);
  tc_end(taddr, 2 * KW);
}

// Pre-order level, one category: X of both children of u,
//   X_0 = U_u o S_1 2^-e_u,  X_1 = U_u o S_0 2^-e_u,
// with S of stored children by tile products, into the adjoint scratch.
// grid = (tiles of 128 patterns, nodes, categories).
template <int KW, bool BF>
__global__ void __launch_bounds__(kTcThr) k_tc_pre_x(
    Dims d, const int *__restrict__ lvl_nodes, int lvl_off, const int *__restrict__ child, int root,
    const float *__restrict__ PT, const uint8_t *__restrict__ tips, const float *__restrict__ tcB,
    const float *__restrict__ part, const float *__restrict__ pre, const int16_t *__restrict__ scale,
    const double *__restrict__ pi, const double *__restrict__ catw,
    const double *__restrict__ site_inv, float *__restrict__ xbuf, int *status) {
  extern __shared__ __align__(1024) float tsm[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int s_ok;
  float *sm = tc_smem(tsm);
  const int bi = blockIdx.y, c = blockIdx.z;
  const int u = lvl_nodes[lvl_off + bi];
  const int slot = u - d.N;
  const int kid[2] = {child[2 * slot], child[2 * slot + 1]};
  const uint32_t taddr = tc_begin(&s_tmem, mbar, 2 * KW);
  uint32_t ph[2] = {0, 0};
  const int p0 = blockIdx.x * kRows, rows = min(kRows, d.P - p0);
  if (!tc_children_S<KW, BF>(d, kid, c, part, tcB, p0, rows, sm, taddr, mbar, ph, &s_ok)) {
    if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    tc_end(taddr, 2 * KW);
    return;
  }
  const int r = threadIdx.x, p = p0 + r;
  const bool live = r < rows;
  const int pc = live ? p : p0;
  int code[2] = {0, 0};
  for (int sd = 0; sd < 2; sd++)
    if (kid[sd] < d.N) code[sd] = tips[(size_t)kid[sd] * d.Pp + pc];
  const Pow2 f = pow2_neg(scale[(size_t)slot * d.Pp + pc]);
  // X_0 overwrites U_u in place: each thread reads its whole U row before it
  // writes that row of X_0
  float *ubuf = sm, *xb0 = sm, *xb1 = sm + Tw<KW, false>::buf;
  if (u != root)  // U_u rows, contiguous loads
    rows_load<KW>(pre + ((((size_t)slot * d.C + c) * d.P) + p0) * d.Kp, d.Kp, rows, ubuf);
  __syncthreads();
  const double rootw = (u == root) ? catw[c] * site_inv[pc] : 0.0;
  float s0[KW], s1[KW];
  child_S<KW>(d, PT, kid[0], c, code[0], taddr, 0, s0);
  child_S<KW>(d, PT, kid[1], c, code[1], taddr, 1, s1);
  const float *urow = ubuf + r * Tw<KW, false>::pad;
#pragma unroll
  for (int j = 0; j < KW; j++) {
    const float uu = (u == root) ? (j < d.K ? (float)(rootw * pi[j]) : 0.f) : urow[j];
    const float a = s1[j], b = s0[j];
    s0[j] = sc(uu * a, f);  // X_0 = U o S_1 2^-e
    s1[j] = sc(uu * b, f);  // X_1 = U o S_0 2^-e
  }
  row_put<KW>(xb0, s0);
  row_put<KW>(xb1, s1);
  __syncthreads();
  rows_store<KW>(xb0, xbuf + ((((size_t)bi * 2 + 0) * d.C + c) * d.P + p0) * d.Kp, d.Kp, rows,
                 nullptr);
  rows_store<KW>(xb1, xbuf + ((((size_t)bi * 2 + 1) * d.C + c) * d.P + p0) * d.Kp, d.Kp, rows,
                 nullptr);
  tc_end(taddr, 2 * KW);
}

}  // namespace

// Tile width 64 (32 < K <= 64), 32 (16 < K <= 32) or 16 (8 < K <= 16): the
// padded row length.
bool tc_path(const epoch_ctx *c) {
  const int kp = c->d.Kp;
  return is_tc_precision(c->precision) && !fast_k4(c) && (kp == 64 || kp == 32 || kp == 16) &&
         c->d.C <= 4;
}

namespace {

template <int KW, bool BF>
cudaError_t tc_post(epoch_ctx *c, int level) {
  const Dims &d = c->d;
  const int w = c->h_level_off[level + 1] - c->h_level_off[level];
  const size_t smem = tc_smem<KW, BF>();
  cudaFuncSetAttribute(k_tc_post<KW, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ceil_div(d.P, kRows), w, d.C);
  cfg.blockDim = dim3(kTcThr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;  // the categories of a (tile, node)
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = d.C;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tc_post<KW, BF>, d, (const int *)c->d_level_nodes,
                            c->h_level_off[level], (const int *)c->d_child,
                            (const float *)c->d_PT32, (const uint8_t *)c->d_tips,
                            (const float *)c->d_tcB, (float *)c->d_part, c->d_scale, c->d_status);
}

template <int KW, bool BF>
void tc_pre_x(epoch_ctx *c, int level, int root) {
  const Dims &d = c->d;
  const int w = c->h_level_off[level + 1] - c->h_level_off[level];
  const size_t smem = tc_smem<KW, BF>();
  cudaFuncSetAttribute(k_tc_pre_x<KW, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_tc_pre_x<KW, BF><<<dim3(ceil_div(d.P, kRows), w, d.C), kTcThr, smem, c->stream>>>(
      d, c->d_level_nodes, c->h_level_off[level], c->d_child, root, c->d_PT32, c->d_tips,
      c->d_tcB, (const float *)c->d_part, (const float *)c->d_pre, c->d_scale, c->d_pi,
      c->d_catw, c->d_site_inv, (float *)c->d_xbuf, c->d_status);
}

template <int KW, bool BF>
void tc_pre_u(epoch_ctx *c, int level) {
  const Dims &d = c->d;
  const int w = c->h_level_off[level + 1] - c->h_level_off[level];
  const size_t smem = tc_smem<KW, BF>();
  cudaFuncSetAttribute(k_tc_pre_u<KW, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_tc_pre_u<KW, BF><<<dim3(ceil_div(d.P, kRows), 2 * w, d.C), kTcThr, smem, c->stream>>>(
      d, c->d_level_nodes, c->h_level_off[level], c->d_child, (const float *)c->d_xbuf, c->d_tcB,
      (float *)c->d_pre, c->d_status);
}

// Dispatch on the tile width (Kp) and the operand format (precision).
template <class F>
auto by_shape(const epoch_ctx *c, F f) {
  const bool bf = c->precision == EPOCH_FP32_TC_BF16;
  const int kp = c->d.Kp;
  if (kp == 64) return bf ? f(std::integral_constant<int, 64>(), std::true_type())
                          : f(std::integral_constant<int, 64>(), std::false_type());
  if (kp == 32) return bf ? f(std::integral_constant<int, 32>(), std::true_type())
                          : f(std::integral_constant<int, 32>(), std::false_type());
  return bf ? f(std::integral_constant<int, 16>(), std::true_type())
            : f(std::integral_constant<int, 16>(), std::false_type());
}

}  // namespace

cudaError_t launch_tc_post(epoch_ctx *c, int level) {
  cudaError_t e = by_shape(c, [&](auto kw, auto bf) { return tc_post<kw.value, bf.value>(c, level); });
  c->launches++;
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_tc_pre_x(epoch_ctx *c, int level, int root) {
  by_shape(c, [&](auto kw, auto bf) {
    tc_pre_x<kw.value, bf.value>(c, level, root);
    return 0;
  });
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_tc_prep(epoch_ctx *c) {
  const Dims &d = c->d;
  by_shape(c, [&](auto kw, auto bf) {
    k_tc_prep<kw.value, bf.value><<<d.nn * d.C, 256, 0, c->stream>>>(d, c->d_P64, c->d_parent,
                                                                      c->d_tcB);
    return 0;
  });
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_tc_pre_u(epoch_ctx *c, int level) {
  by_shape(c, [&](auto kw, auto bf) {
    tc_pre_u<kw.value, bf.value>(c, level);
    return 0;
  });
  c->launches++;
  return cudaGetLastError();
}

size_t tc_operand_floats(const epoch_ctx *c) {
  return (size_t)(2 * c->max_taxa - 1) * c->d.C * 4 * c->d.Kp * c->d.Kp;
}

}  // namespace epoch
