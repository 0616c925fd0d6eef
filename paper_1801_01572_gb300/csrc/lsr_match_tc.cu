// lsr_match_tc.cu -- the feature pre-matching cache (Algorithm 1, "Parallel
// FPFH feature pre-matching") on the 5th-generation tensor cores.
//
// The squared descriptor distance |a - b|^2 = |a|^2 + |b|^2 - 2 a.b is a dense
// contraction. Descriptors are first centred on a mean descriptor c (distances
// do not change; the magnitudes that set the FP32 accumulation error shrink)
// and rounded to BF16. Two operand layouts:
//   plain (K = 48):  x ~ h = bf16(x); the contraction is h_a . h_b.
//   split (K = 112): x ~ h + l with l = bf16(x - h); the contraction is
//                    h_a.h_b + l_a.h_b + h_a.l_b (the l_a.l_b term, below
//                    2^-16 |a||b|, is left out and bounded).
// Three spare K columns carry |b~|^2 as three BF16 parts (query side 1.0) and
// the query side is pre-scaled by -2 (exact), so the FP32 accumulator holds the
// score s = |b~|^2 - 2 a~.b~ and the epilogue only compares.
//
// Each persistent CTA takes units of 128 or 256 queries (one or two M = 128
// tiles sharing every database tile; the shape is chosen per size by the
// autotuner) and streams the database in tiles of 128 rows: one thread issues
// tcgen05.mma from shared memory into TMEM (two accumulator buffers, so the
// tensor pipe runs while the epilogue drains the other), and four or eight
// epilogue warps, one query per thread, read a whole accumulator row with one
// wait, release the buffer at once, and keep the 8 smallest minima of 16-row
// chunks (a chunk enters when its minimum beats the lane's current 8th).
//
// The 128 rows of those 8 chunks are re-ranked with the exact FP32 distance of
// the original descriptors in the FP32 matcher's operation order. A
// certificate proves, per query, that the FP32 winner is among them:
//   D~^2 = s + |a~|^2 is within efp of |a~ - b~|^2 (accumulation, the left-out
//   term, the BF16 split of |b~|^2), and | |a - b| - |a~ - b~| | <= eta =
//   |a - c - a~| + max_b |b - c - b~| (+ the rounding of the centring);
//   every row outside the candidate chunks has s >= s_(8), the 8th smallest
//   chunk minimum, so its distance is at least lo8 = sqrt(s_(8) + |a~|^2 -
//   efp) - eta, while the row of the smallest score has one of at most hi1 =
//   sqrt(s_(1) + |a~|^2 + efp) + eta; if lo8 > hi1 beyond the FP32
//   evaluation error (35 roundings of 2^-24 on D^2), no outside row can win.
// The accumulation error is bounded with the truncating-adder model of tensor
// core FP32 accumulation: each MMA of 16 products adds at most 17 errors of
// 2^-23 times the largest magnitude involved, i.e. 15e-6 * sum |products| for
// the 7 MMAs of the split layout (the validation entry point measures it).
// Queries without the certificate are re-scanned exactly in FP32. The result
// (index and distance) equals the FP32 matcher's bit for bit.
//
// Tiles sit in global memory already in the layout the MMA reads from shared
// memory (K-major, no swizzle: 8 rows x 16 bytes per core matrix, K-adjacent
// core matrices 128 bytes apart, 8-row groups K/8 * 128 bytes apart), so every
// tile arrives with one bulk copy completed on an mbarrier. Every wait is
// bounded in time: a CTA that gives up records an error, stops issuing work,
// waits (bounded) for its copies and MMAs in flight, releases TMEM and returns.
#include <cuda_bf16.h>
#include <float.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kTcM = 128;                       // queries per MMA tile (TMEM lanes)
constexpr int kTcN = 128;                       // database rows per tile
constexpr int kLBO = 128;                       // bytes between K-adjacent core matrices
constexpr int kTopK = 8;                        // candidate chunks per query
constexpr int kChunkW = 16;                     // database rows per chunk
constexpr int kChunks = kTcN / kChunkW;         // chunks per tile
constexpr int kLoads = kTcN / 32;               // 32-column TMEM loads per accumulator row
constexpr unsigned long long kWaitNs = 2000000000ull;  // give up after 2 s (the default limit; drains always)
constexpr float kPadScore = 1.2676506e30f;      // 2^100: |b~|^2 of padding rows
constexpr float kAccErr = 1.5e-5f;              // accumulation error per unit of sum |products|
constexpr int kCenterGroups = 8;                // row groups of the centring kernel

// Operand layout of one mode: KS MMA k-steps of 16.
template <int KS>
struct Shape {
  static constexpr bool kSplit = KS == 7;
  static constexpr int K = 16 * KS;
  static constexpr int SBO = (K / 8) * 128;      // bytes between 8-row groups
  static constexpr int TileBytes = kTcM * K * 2;
  static constexpr int SqCol = kSplit ? 3 * kD : kD;  // first |b~|^2 column
  static_assert(SqCol + 3 <= K, "operand layout");
};

// Tile shape of the persistent CTA: QT query tiles of 128 per work unit.
//   QT = 2: 256 queries share every database tile; 4 copy stages; 512 TMEM
//           columns (two buffers of 2 x 128): one CTA per SM.
//   QT = 1: 128 queries; 3 stages; 256 TMEM columns: two CTAs per SM, so
//           small clouds still spread over every SM.
template <int KS, int QT>
struct Cfg {
  static constexpr int Stages = QT == 2 ? 4 : 3;
  static constexpr int EpiWarps = 4 * QT;        // warps 0..EpiWarps-1: epilogue; the next: copies + MMA
  static constexpr int Threads = (EpiWarps + 1) * 32;
  static constexpr int UnitQ = QT * kTcM;
  static constexpr uint32_t AccCols = QT * kTcN; // one accumulator buffer
  static constexpr uint32_t TmemCols = 2 * AccCols;
  static constexpr int CtasPerSm = QT == 2 ? 1 : 2;
  static constexpr int UnitBytes = QT * Shape<KS>::TileBytes;
  static constexpr int SmemUsed = UnitBytes + Stages * Shape<KS>::TileBytes + 128;
  // enough shared memory that no more CTAs than TMEM holds share an SM
  static constexpr int SmemFloor = CtasPerSm == 1 ? 120 * 1024 : 80 * 1024;
  static constexpr int SmemBytes = SmemUsed > SmemFloor ? SmemUsed : SmemFloor;
  static_assert(CtasPerSm * (SmemBytes + 1024) <= 228 * 1024, "shared memory plan");
  static_assert(CtasPerSm * TmemCols <= 512, "tensor memory plan");
};

template <int KS>
__host__ __device__ inline int tc_off(int r, int k) {
  return (r >> 3) * Shape<KS>::SBO + (k >> 3) * kLBO + (r & 7) * 16 + (k & 7) * 2;
}

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t s2u(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s2u(b)), "r"(count));
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(s2u(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity; gives up after limit_ns (flagging
// the CTA) or as soon as another thread of the CTA has given up.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *fail,
                                          unsigned long long limit_ns) {
  if (mbar_try(b, parity)) return true;
  unsigned long long t0 = gtime();
  for (;;) {
    if (mbar_try(b, parity)) return true;
    if (*fail) return false;
    if (gtime() - t0 > limit_ns) {
      *fail = 1;
      return false;
    }
  }
}
// Bounded wait used only while cleaning up after a failure.
__device__ __forceinline__ void mbar_drain(uint64_t *b, uint32_t parity) {
  unsigned long long t0 = gtime();
  while (!mbar_try(b, parity) && gtime() - t0 < kWaitNs) {
  }
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s2u(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s2u(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s2u(dst)),
      "l"(src), "r"(bytes), "r"(s2u(b))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row) byte offsets, all >> 4; fixed version bits 46-47 = 1; no swizzle.
template <int KS>
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
  uint64_t a = (uint64_t)((s2u(p) & 0x3FFFF) >> 4);
  return a | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(Shape<KS>::SBO >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t *b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s2u(b))
               : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (no wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
        "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]),
        "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]),
        "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- operand preparation
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Error-free transformations (Knuth's TwoSum; the FMA product error).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// The centre c: mean of up to 2048 evenly spaced database rows, summed in a
// fixed order (one block of kCenterGroups x 33 threads), so it is the same on
// every run.
__global__ void k_center(const float *__restrict__ FQ, int nQ, float *__restrict__ c) {
  __shared__ float part[kCenterGroups][kD];
  const int col = threadIdx.x % kD, grp = threadIdx.x / kD;
  const int step = nQ > 2048 ? nQ / 2048 : 1;
  const int m = (nQ + step - 1) / step;  // sampled rows 0, step, 2 step, ...
  if (grp < kCenterGroups) {
    float s = 0.f;
    for (int i = grp; i < m; i += kCenterGroups) s += FQ[(size_t)i * step * kDS + col];
    part[grp][col] = s;
  }
  __syncthreads();
  if (threadIdx.x < kD) {
    float s = 0.f;
    for (int g = 0; g < kCenterGroups; ++g) s += part[g][threadIdx.x];
    c[threadIdx.x] = s / (float)m;
  }
}

struct PrepOut {
  char *tiles;
  float *aa;             // query side: |a~|^2 (rows padded to the unit size)
  float *eta;            // query side: |a - c - a~| bound
  unsigned *eta_max;     // database side: max |b - c - b~| bound (float bits)
  unsigned *bb_max;      // database side: max |b~|^2 (float bits)
};

// One thread per (padded) row: centring, BF16 rounding (and split), the tile
// layout, |x~|^2 (compensated) and the rounding bound eta.
template <int KS>
__global__ void k_prep_tiles(const float *__restrict__ F, int n, int rows, bool query, const float *__restrict__ c,
                             PrepOut o) {
  using S = Shape<KS>;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    char *base = o.tiles + (size_t)(r / kTcM) * S::TileBytes;
    const int rr = r % kTcM;
    const bool real = r < n;
    auto put = [&](int k, float v) {
      *reinterpret_cast<__nv_bfloat16 *>(base + tc_off<KS>(rr, k)) = __float2bfloat16_rn(v);
    };
    float s_hi = 0.f, s_lo = 0.f, e2 = 0.f, x2 = 0.f;
    for (int k = 0; k < kD; ++k) {
      const float x = real ? F[(size_t)r * kDS + k] - __ldg(c + k) : 0.f;
      const float h = bf16r(x);
      const float l = S::kSplit ? bf16r(x - h) : 0.f;  // x - h is exact
      const float xt = h + l;                          // exact (at most 16 significant bits)
      const float res = x - xt;                        // exact
      e2 = fmaf(res, res, e2);
      x2 = fmaf(x, x, x2);
      const float p = xt * xt, pe = fmaf(xt, xt, -p);
      float t, e;
      two_sum(s_hi, p, t, e);
      s_hi = t;
      s_lo += e + pe;
      if (query) {
        put(k, -2.f * h);
        if (S::kSplit) put(kD + k, -2.f * l), put(2 * kD + k, -2.f * h);
      } else {
        put(k, h);
        if (S::kSplit) put(kD + k, h), put(2 * kD + k, l);
      }
    }
    float sq[3];
    if (query) {
      sq[0] = sq[1] = sq[2] = 1.f;
    } else if (real) {
      const float p0 = bf16r(s_hi), r1 = s_hi - p0;  // exact
      const float p1 = bf16r(r1);
      sq[0] = p0, sq[1] = p1, sq[2] = bf16r((r1 - p1) + s_lo);
    } else {
      sq[0] = kPadScore, sq[1] = sq[2] = 0.f;
    }
    for (int k = S::SqCol; k < S::K; ++k) put(k, k < S::SqCol + 3 ? sq[k - S::SqCol] : 0.f);
    // rounding of x~ plus the rounding of the centring (2^-24 |x| per component)
    const float eta = sqrtf(e2) * (1.f + 1e-5f) + 1.2e-7f * sqrtf(x2);
    if (query) {
      o.aa[r] = s_hi + s_lo;
      o.eta[r] = eta;
    } else if (real) {
      atomicMax(o.eta_max, __float_as_uint(eta));
      atomicMax(o.bb_max, __float_as_uint(s_hi + s_lo));
    }
  }
}

struct TcArgs {
  const char *A, *B;            // query units and database tiles (BF16, MMA layout)
  const float *aa, *eta_a;      // per query
  const unsigned *eta_b, *bb;   // database maxima (float bits)
  const float *FP, *FQ;         // FP32 descriptors (stride kDS) for the re-rank
  int nP, nQ, nU, nNT;
  int *nn;
  float *d1;
  int *fb_rows, *fb_count;      // queries left to the exact FP32 scan
  int *err;                     // set to 1 by a CTA that gave up
  float *d2;                    // optional: all D~^2 = s + |a~|^2 (nP x nNT * kTcN) instead of the top-8
  unsigned long long wait_ns;   // limit of every wait of the pipeline (the drain after a failure keeps kWaitNs)
  int stall;                    // fault injection: the producer issues nothing, so the first wait runs out
};

// Exact FP32 squared distance in the FP32 matcher's operation order (one
// fused multiply-add per bin, bins taken in desc_order; a already in it). The
// row is read as nine 16-byte loads, the order applied in registers.
__device__ __forceinline__ float exact_d2(const float (&a)[kD], const float *__restrict__ b) {
  float r[36];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const float4 x = __ldg(reinterpret_cast<const float4 *>(b) + q);
    r[4 * q] = x.x, r[4 * q + 1] = x.y, r[4 * q + 2] = x.z, r[4 * q + 3] = x.w;
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kD; ++k) {
    float t = a[k] - r[desc_order(k)];
    s = fmaf(t, t, s);
  }
  return s;
}

__device__ __forceinline__ void top8_insert(float (&ts)[kTopK], int (&ti)[kTopK], float v, int id) {
  if (!(v < ts[kTopK - 1])) return;
  ts[kTopK - 1] = v;
  ti[kTopK - 1] = id;
#pragma unroll
  for (int q = kTopK - 1; q > 0; --q)
    if (ts[q] < ts[q - 1]) {
      float a = ts[q];
      ts[q] = ts[q - 1];
      ts[q - 1] = a;
      int b = ti[q];
      ti[q] = ti[q - 1];
      ti[q - 1] = b;
    }
}

template <int KS, int QT>
__global__ void __launch_bounds__(Cfg<KS, QT>::Threads, Cfg<KS, QT>::CtasPerSm) k_match_tc(TcArgs g) {
  using S = Shape<KS>;
  using C = Cfg<KS, QT>;
  constexpr int kStages = C::Stages, kEpiWarps = C::EpiWarps, kUnitQ = C::UnitQ;
  constexpr uint32_t kAccCols = C::AccCols, kTmemCols = C::TmemCols;
  extern __shared__ __align__(128) unsigned char smem[];
  char *sA = reinterpret_cast<char *>(smem);
  char *sB = sA + C::UnitBytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + kStages * S::TileBytes);
  uint64_t *barA = bars;                 // 1
  uint64_t *barB = bars + 1;             // kStages
  uint64_t *barDone = barB + kStages;    // 2: accumulator buffer written
  uint64_t *barEmpty = barDone + 2;      // 2: accumulator buffer drained
  uint32_t *tslot = reinterpret_cast<uint32_t *>(barEmpty + 2);
  volatile int *fail = reinterpret_cast<volatile int *>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    mbar_init(barA, 1);
    for (int s = 0; s < kStages; ++s) mbar_init(barB + s, 1);
    for (int s = 0; s < 2; ++s) mbar_init(barDone + s, 1), mbar_init(barEmpty + s, kEpiWarps);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kEpiWarps) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s2u(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  int nuloc = 0;
  for (int u = blockIdx.x; u < g.nU; u += gridDim.x) ++nuloc;
  const int total = nuloc * g.nNT;  // (unit, database tile) steps of this CTA

  // producer state, kept for the clean-up after a failure
  int loaded[kStages];
  int last_commit = -1, a_pending = -1;
  for (int s = 0; s < kStages; ++s) loaded[s] = -1;

  if (warp == kEpiWarps) {
    // ------------------------------------------------ copies + MMA (one thread)
    if (lane == 0 && total > 0 && !g.stall) {
      auto load_b = [&](int jj) {
        int st = jj % kStages, t = jj % g.nNT;
        mbar_expect_tx(barB + st, S::TileBytes);
        bulk_g2s(sB + st * S::TileBytes, g.B + (size_t)t * S::TileBytes, S::TileBytes, barB + st);
        loaded[st] = jj;
      };
      for (int jj = 0; jj < total && jj < kStages; ++jj) load_b(jj);
      int units = 0;
      for (int j = 0; j < total; ++j) {
        const int t = j % g.nNT;
        if (t == 0) {
          // the previous unit's MMAs must be done reading the query tiles
          if (j > 0 && !mbar_wait(barDone + ((j - 1) & 1), ((j - 1) >> 1) & 1, fail, g.wait_ns)) break;
          int u = blockIdx.x + (j / g.nNT) * gridDim.x;
          mbar_expect_tx(barA, C::UnitBytes);
          bulk_g2s(sA, g.A + (size_t)u * C::UnitBytes, C::UnitBytes, barA);
          a_pending = units & 1;
          if (!mbar_wait(barA, units & 1, fail, g.wait_ns)) break;
          a_pending = -1;
          ++units;
        }
        const int st = j % kStages;
        if (!mbar_wait(barB + st, (j / kStages) & 1, fail, g.wait_ns)) break;
        loaded[st] = -1;
        if (j >= 2 && !mbar_wait(barEmpty + (j & 1), ((j - 2) >> 1) & 1, fail, g.wait_ns)) break;
        tc_fence_after();
        const uint32_t d = tbase + (uint32_t)((j & 1) * kAccCols);
#pragma unroll
        for (int qt = 0; qt < QT; ++qt)
#pragma unroll
          for (int k = 0; k < KS; ++k)
            mma_bf16(d + qt * kTcN, smem_desc<KS>(sA + qt * S::TileBytes + k * 2 * kLBO),
                     smem_desc<KS>(sB + st * S::TileBytes + k * 2 * kLBO), k > 0 ? 1u : 0u);
        mma_commit(barDone + (j & 1));
        last_commit = j;
        // refill the stage of tile j-1 with tile j+3 once its MMAs are done
        if (j >= 1 && j + kStages - 1 < total) {
          if (!mbar_wait(barDone + ((j - 1) & 1), ((j - 1) >> 1) & 1, fail, g.wait_ns)) break;
          load_b(j + kStages - 1);
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue: one query per thread
    const int qt = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int row_in_unit = qt * kTcM + 32 * (warp & 3) + lane;
    const int ncols = g.nNT * kTcN;
    int j = 0;
    bool ok = true;
    for (int m = 0; m < nuloc && ok; ++m) {
      const int u = blockIdx.x + m * gridDim.x;
      const int r = u * kUnitQ + row_in_unit;
      float ts[kTopK];
      int ti[kTopK];
#pragma unroll
      for (int q = 0; q < kTopK; ++q) ts[q] = FLT_MAX, ti[q] = -1;
      for (int t = 0; t < g.nNT; ++t, ++j) {
        const int buf = j & 1;
        ok = mbar_wait(barDone + buf, (j >> 1) & 1, fail, g.wait_ns);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc_fence_after();
        // the whole row of the accumulator with one wait
        const uint32_t row = tbase + lane_base + (uint32_t)(buf * kAccCols + qt * kTcN);
        float v[kTcN];
        __syncwarp();  // the loads below are warp-collective
#pragma unroll
        for (int q = 0; q < kLoads; ++q) tmem_ld32(row + q * 32, v + q * 32);
        tmem_wait_ld();
        const int c0 = t * kTcN;
        if (g.d2) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(barEmpty + buf);
          if (r < g.nP) {
            const float aa = g.aa[r];
            for (int k = 0; k < kTcN; ++k) g.d2[(size_t)r * ncols + c0 + k] = v[k] + aa;
          }
          continue;
        }
        // the scores are in registers: the buffer goes back to the MMA at once
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(barEmpty + buf);
        // minimum of each chunk; the 8 smallest chunk minima are kept
#pragma unroll
        for (int q = 0; q < kChunks; ++q) {
          const float *w = v + q * kChunkW;
          float a0 = w[0], a1 = w[1], a2 = w[2], a3 = w[3];
#pragma unroll
          for (int k = 4; k < kChunkW; k += 4) {
            a0 = fminf(a0, w[k]), a1 = fminf(a1, w[k + 1]);
            a2 = fminf(a2, w[k + 2]), a3 = fminf(a3, w[k + 3]);
          }
          top8_insert(ts, ti, fminf(fminf(a0, a1), fminf(a2, a3)), t * kChunks + q);
        }
      }
      if (!ok || g.d2 || r >= g.nP) continue;
      // exact FP32 re-rank of the rows of the candidate chunks
      float a[kD];
#pragma unroll
      for (int k = 0; k < kD; ++k) a[k] = __ldg(g.FP + (size_t)r * kDS + desc_order(k));
      float best = FLT_MAX;
      int bi = -1;
#pragma unroll 1
      for (int q = 0; q < kTopK; ++q) {
        if (ti[q] < 0) continue;
        const int c0 = ti[q] * kChunkW, c1 = min(g.nQ, c0 + kChunkW);
#pragma unroll 1
        for (int c = c0; c < c1; ++c) {
          if (!LSR_IN_BOUNDS(c, g.nQ, kSiteMatchRow)) break;
          const float d = exact_d2(a, g.FQ + (size_t)c * kDS);
          if (d < best || (d == best && c < bi)) best = d, bi = c;
        }
      }
      bool cert = g.nQ <= kTopK * kChunkW;
      if (!cert && ti[kTopK - 1] >= 0) {
        const float aa = g.aa[r], bbm = __uint_as_float(*g.bb);
        const float na = sqrtf(aa), nb = sqrtf(bbm);
        // accumulation (sum |products| <= 2.05 |a~||b~| + |b~|^2) and, split
        // layout, the left-out 2 l_a.l_b (<= 2^-15 |a~||b~|)
        const float efp = kAccErr * (2.05f * na * nb + bbm) + (S::kSplit ? 3.1e-5f * na * nb : 0.f);
        const float eta = g.eta_a[r] + __uint_as_float(*g.eta_b);
        const float lo8 = sqrtf(fmaxf(ts[kTopK - 1] + aa - efp, 0.f)) - eta;
        const float hi1 = sqrtf(fmaxf(ts[0] + aa + efp, 0.f)) + eta;
        cert = lo8 > hi1 * (1.f + 1e-5f);
      }
      g.nn[r] = bi;
      if (g.d1) g.d1[r] = best;
      if (!cert) {
        const int slot = atomicAdd(g.fb_count, 1);
        if (LSR_IN_BOUNDS(slot, g.nP, kSiteMatchQuery)) g.fb_rows[slot] = r;
      }
    }
  }

  // teardown: every epilogue warp has finished its TMEM reads
  tc_fence_before();
  __syncthreads();
  if (warp == kEpiWarps) {
    if (lane == 0 && *fail) {
      // a wait gave up: nothing may still write TMEM or shared memory
      if (last_commit >= 0) mbar_drain(barDone + (last_commit & 1), (last_commit >> 1) & 1);
      for (int s = 0; s < kStages; ++s)
        if (loaded[s] >= 0) mbar_drain(barB + s, (loaded[s] / kStages) & 1);
      if (a_pending >= 0) mbar_drain(barA, (uint32_t)a_pending);
      atomicExch(g.err, 1);
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols));
  }
}

struct TcLayout {
  char *A = nullptr, *B = nullptr;
  float *aa = nullptr, *eta = nullptr, *center = nullptr;
  unsigned *maxes = nullptr;  // eta_b, bb
  int *fb_rows = nullptr;
  unsigned long long *packed = nullptr;
  size_t bytes = 0;
};

// Query rows are padded to a multiple of 256 (a whole number of units for
// either tile shape); unit u of shape QT is tiles QT u .. QT u + QT - 1.
template <int KS>
TcLayout tc_layout(char *base, int nP, int nQ) {
  using S = Shape<KS>;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t tilesA = 2 * (size_t)lsr_div_up(nP, 2 * kTcM), nNT = (size_t)lsr_div_up(nQ, kTcN);
  size_t rowsA = tilesA * kTcM;
  size_t off = 0;
  TcLayout L;
  auto take = [&](size_t bytes) {
    char *p = base ? base + off : nullptr;
    off += al(bytes);
    return p;
  };
  L.A = take(tilesA * S::TileBytes);
  L.B = take(nNT * S::TileBytes);
  L.aa = reinterpret_cast<float *>(take(rowsA * 4));
  L.eta = reinterpret_cast<float *>(take(rowsA * 4));
  L.center = reinterpret_cast<float *>(take(kD * 4));
  L.maxes = reinterpret_cast<unsigned *>(take(2 * 4));
  L.fb_rows = reinterpret_cast<int *>(take((size_t)nP * 4));
  L.packed = reinterpret_cast<unsigned long long *>(take((size_t)nP * 8));
  L.bytes = off;
  return L;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 148;
  }
  return n > 0 ? n : 148;
}

template <int KS, int QT>
cudaError_t launch_tc(const TcLayout &L, const float *FP, int nP, const float *FQ, int nQ, int *nn, float *d1,
                      int *fb_count, int *err, float *d2, const TcFault &f, cudaStream_t s) {
  using C = Cfg<KS, QT>;
  const int nU = (int)lsr_div_up(nP, C::UnitQ), nNT = (int)lsr_div_up(nQ, kTcN);
  LSR_CUDA_TRY(cudaFuncSetAttribute(k_match_tc<KS, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SmemBytes));
  TcArgs g{L.A, L.B, L.aa, L.eta, L.maxes, L.maxes + 1, FP, FQ, nP, nQ, nU, nNT,
           nn, d1, L.fb_rows, fb_count, err, d2, f.wait_ns ? f.wait_ns : kWaitNs, f.stall};
  const int slots = sm_count() * C::CtasPerSm;
  const int grid = nU < slots ? nU : slots;
  LSR_LAUNCH(k_match_tc<KS, QT><<<grid, C::Threads, C::SmemBytes, s>>>(g));
  return cudaGetLastError();
}

template <int KS>
cudaError_t run_tc(const float *FP, int nP, const float *FQ, int nQ, int qt, char *ws, int *nn, float *d1,
                   int *fb_count, int *err, float *d2, const TcFault &f, cudaStream_t s) {
  TcLayout L = tc_layout<KS>(ws, nP, nQ);
  const int nNT = (int)lsr_div_up(nQ, kTcN);
  LSR_CUDA_TRY(cudaMemsetAsync(L.maxes, 0, 2 * sizeof(unsigned), s));
  LSR_CUDA_TRY(cudaMemsetAsync(fb_count, 0, sizeof(int), s));
  LSR_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  LSR_LAUNCH(k_center<<<1, kCenterGroups * kD, 0, s>>>(FQ, nQ, L.center));
  const int rowsA = 2 * (int)lsr_div_up(nP, 2 * kTcM) * kTcM, rowsB = nNT * kTcN;
  PrepOut pa{L.A, L.aa, L.eta, nullptr, nullptr};
  PrepOut pb{L.B, nullptr, nullptr, L.maxes, L.maxes + 1};
  LSR_LAUNCH(k_prep_tiles<KS><<<(int)lsr_div_up(rowsA, 256), 256, 0, s>>>(FP, nP, rowsA, true, L.center, pa));
  LSR_LAUNCH(k_prep_tiles<KS><<<(int)lsr_div_up(rowsB, 256), 256, 0, s>>>(FQ, nQ, rowsB, false, L.center, pb));
  if (qt == 1)
    LSR_CUDA_TRY((launch_tc<KS, 1>(L, FP, nP, FQ, nQ, nn, d1, fb_count, err, d2, f, s)));
  else
    LSR_CUDA_TRY((launch_tc<KS, 2>(L, FP, nP, FQ, nQ, nn, d1, fb_count, err, d2, f, s)));
  if (!d2) LSR_CUDA_TRY(launch_match_fp32_rows(FP, nP, FQ, nQ, L.fb_rows, fb_count, L.packed, nn, d1, s));
  return cudaGetLastError();
}

constexpr int kKsPlain = 3, kKsSplit = 7;

}  // namespace

LSR_CHECK_READER(match_tc)

size_t tc_workspace_bytes(int nP, int nQ, bool split) {
  return split ? tc_layout<kKsSplit>(nullptr, nP, nQ).bytes : tc_layout<kKsPlain>(nullptr, nP, nQ).bytes;
}

int tc_score_cols(int nQ) { return (int)lsr_div_up(nQ, kTcN) * kTcN; }

// One query tile per CTA (two CTAs per SM) unless the autotuner chose for the
// size: on the 150k-point room pair it takes 4.58 ms against 5.53 ms with two
// query tiles per CTA (one CTA per SM).
int tc_default_tile(int) { return 1; }

cudaError_t launch_match_bf16(const float *FP, int nP, const float *FQ, int nQ, bool split, int qt, char *ws, int *nn,
                              float *d1, int *fb_count, int *err, float *d2, cudaStream_t s, TcFault f) {
  if (nP < 1 || nQ < 1 || (qt != 0 && qt != 1 && qt != 2)) return cudaErrorInvalidValue;
  if (qt == 0) qt = tc_default_tile(nP);
  return split ? run_tc<kKsSplit>(FP, nP, FQ, nQ, qt, ws, nn, d1, fb_count, err, d2, f, s)
               : run_tc<kKsPlain>(FP, nP, FQ, nQ, qt, ws, nn, d1, fb_count, err, d2, f, s);
}

int device_sm_count() { return sm_count(); }

}  // namespace lsr
