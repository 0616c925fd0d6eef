// lsr_match.cu -- feature pre-matching cache on the FP32 cores (Algorithm 1,
// "Parallel FPFH feature pre-matching": nn[i] = NN of F(p_i) in F(Q)).
//
// Exact brute force: nn[i] = argmin_j sum_k (a_k - b_k)^2 with ties to the
// smallest j, accumulated as s = fma(t, t, s) over the 33 bins taken in
// desc_order (central bins first). Each thread keeps one query descriptor in
// registers; tiles of database descriptors are staged in shared memory in
// that order and read as broadcasts. The partial sums only grow (t^2 >= 0 and
// rounding is monotone), so a row whose partial sum already exceeds every
// query's current best in the warp can neither win nor tie: after 4, 8, 12, 16
// and 24 terms the warp tests that and skips the rest of the row (same
// result). Queries arrive in grid order (points sorted by feature-radius
// cell), so the 32 queries of a warp lie close together and have similar
// descriptors, and the test succeeds for most rows after the first four terms.
// (One query per thread prunes better and keeps more warps resident than two
// or four, which share every test.)
//
// Whole tiles are skipped as well. The database is in grid order too, so the
// 64 rows of a tile have similar descriptors; k_tile_bounds stores per tile
// and bin the minimum and maximum over its rows. For a query a, the bound
// L = sum_k g_k^2 with g_k = max(lo_k - a_k, a_k - hi_k, 0), accumulated in
// desc_order with the same fused multiply-adds, never exceeds the computed
// distance of any row of the tile: |fl(a_k - b_k)| >= g_k because rounding
// is monotone and lo_k <= b_k <= hi_k, and each fma step is monotone in both
// the product and the running sum. A warp whose queries all have L > best
// skips the tile (no row of it can win or tie); a block skips staging it when
// none of its warps needs it.
#include <float.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kMT = 128;   // threads per block
constexpr int kQF = 1;     // queries per thread, full scan (k_match_fp32)
constexpr int kQR = 2;     // queries per thread, listed rows (k_match_rows_chunked)
constexpr int kTile = 64;  // database rows per shared-memory tile
constexpr int kStageThreads = 9 * (kMT / 9);  // staging threads: one float4 column each
constexpr int kTB = 72;    // floats per tile bound: lo[36], hi[36], bins in desc_order
constexpr int kLB = 33;    // bins (desc_order) summed in the tile bound: all (fewer loosen it more than they save)
static_assert(kTile * 9 > kStageThreads, "staging covers the tile in several passes");

// Database rows [base, base + kTile) (zero past lim) into the tile, bin
// desc_order(k) at slot k and zeros at slots 33..35. Thread t < kStageThreads
// copies float4 column t % 9 of rows t / 9, t / 9 + kMT / 9, ...; rk holds the
// slots of that column's four bins (-1 past the descriptor).
__device__ __forceinline__ void stage_tile(float4 (*tile)[9], const float *__restrict__ FQ, int base, int lim,
                                           const int (&rk)[4]) {
  if (threadIdx.x >= kStageThreads) return;
  float *tf = reinterpret_cast<float *>(tile);
  const int c = threadIdx.x % 9;
  for (int r = threadIdx.x / 9; r < kTile; r += kMT / 9) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (base + r < lim) v = reinterpret_cast<const float4 *>(FQ + (size_t)(base + r) * kDS)[c];
    float *row = tf + r * 36;
    row[rk[0]] = v.x;
    if (rk[1] >= 0) {
      row[rk[1]] = v.y, row[rk[2]] = v.z, row[rk[3]] = v.w;
    } else {
      row[33] = 0.f, row[34] = 0.f, row[35] = 0.f;
    }
  }
}

__device__ __forceinline__ void stage_ranks(int (&rk)[4]) {
  const int c = threadIdx.x % 9;
#pragma unroll
  for (int i = 0; i < 4; ++i) rk[i] = 4 * c + i < kD ? desc_rank(4 * c + i) : -1;
}

// Scan the m staged rows for the Q queries of this thread (a in
// desc_order), updating best / bj; row j of the tile is database row base + j.
// kCount: add the terms evaluated per query to terms.
template <int Q, bool kCount = false>
__device__ __forceinline__ void scan_tile(const float4 (*tile)[9], int m, int base, const float (&a)[Q][kD],
                                          float (&best)[Q], int (&bj)[Q], unsigned *terms = nullptr) {
  for (int j = 0; j < m; ++j) {
    float s[Q];
#pragma unroll
    for (int u = 0; u < Q; ++u) s[u] = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c >= 1 && (c <= 4 || c == 6)) {
        bool past = true;
#pragma unroll
        for (int u = 0; u < Q; ++u) past &= s[u] > best[u];
        if (__all_sync(0xffffffffu, past)) break;
      }
      float4 b = tile[j][c];
      if (kCount) *terms += c == 7 ? 5 : 4;
#pragma unroll
      for (int u = 0; u < Q; ++u) {
        float t0 = a[u][4 * c] - b.x, t1 = a[u][4 * c + 1] - b.y, t2 = a[u][4 * c + 2] - b.z,
              t3 = a[u][4 * c + 3] - b.w;
        s[u] = fmaf(t0, t0, s[u]);
        s[u] = fmaf(t1, t1, s[u]);
        s[u] = fmaf(t2, t2, s[u]);
        s[u] = fmaf(t3, t3, s[u]);
      }
      if (c == 7) {
        float b32 = tile[j][8].x;
#pragma unroll
        for (int u = 0; u < Q; ++u) {
          float t = a[u][32] - b32;
          s[u] = fmaf(t, t, s[u]);
          if (s[u] < best[u]) best[u] = s[u], bj[u] = base + j;
        }
      }
    }
  }
}

// Per tile of kTile database rows: lo / hi of every bin over the tile's rows,
// in desc_order (block t, thread k < 33 reads bin desc_order(k) of each row).
__global__ void k_tile_bounds(const float *__restrict__ FQ, int nQ, float *__restrict__ tb) {
  const int t = blockIdx.x, k = threadIdx.x;
  if (k >= kD) return;
  const int r0 = t * kTile, r1 = min(nQ, r0 + kTile), col = desc_order(k);
  float lo = FLT_MAX, hi = -FLT_MAX;
  for (int r = r0; r < r1; ++r) {
    const float v = FQ[(size_t)r * kDS + col];
    lo = fminf(lo, v), hi = fmaxf(hi, v);
  }
  tb[(size_t)t * kTB + k] = lo;
  tb[(size_t)t * kTB + 36 + k] = hi;
}

// The bound of tile t for each query of this thread: no row of the tile has
// a computed distance below L[u].
template <int Q>
__device__ __forceinline__ void tile_bound(const float *__restrict__ tb, int t, const float (&a)[Q][kD],
                                           float (&L)[Q]) {
  const float *lo = tb + (size_t)t * kTB, *hi = lo + 36;
#pragma unroll
  for (int u = 0; u < Q; ++u) L[u] = 0.f;
#pragma unroll
  for (int k = 0; k < kLB; ++k) {
    const float l = __ldg(lo + k), h = __ldg(hi + k);
#pragma unroll
    for (int u = 0; u < Q; ++u) {
      const float g = fmaxf(fmaxf(l - a[u][k], a[u][k] - h), 0.f);
      L[u] = fmaf(g, g, L[u]);
    }
  }
}

// True if some query of this thread may find a row of tile t at or below its
// current best (the exact bound of the tile's rows does not exceed best).
template <int Q>
__device__ __forceinline__ bool tile_needed(const float *__restrict__ tb, int t, const float (&a)[Q][kD],
                                            const float (&best)[Q]) {
  float L[Q];
  tile_bound<Q>(tb, t, a, L);
  bool need = false;
#pragma unroll
  for (int u = 0; u < Q; ++u) need |= !(L[u] > best[u]);
  return need;
}

// kCount: also add the number of terms (a_k - b_k)^2 evaluated for the valid
// queries to *terms (a separate instantiation, used when profiling).
template <bool kCount>
__global__ void __launch_bounds__(kMT) k_match_fp32(const float *__restrict__ FP, int nP, const float *__restrict__ FQ,
                                                    int nQ, const float *__restrict__ tb, int *__restrict__ nn,
                                                    float *__restrict__ d1, unsigned long long *__restrict__ terms) {
  __shared__ float4 tile[kTile][9];
  float a[kQF][kD];
  int qi[kQF], rk[4];
  stage_ranks(rk);
#pragma unroll
  for (int u = 0; u < kQF; ++u) {
    qi[u] = blockIdx.x * (kMT * kQF) + u * kMT + threadIdx.x;
    const float *row = FP + (size_t)(qi[u] < nP ? qi[u] : 0) * kDS;
#pragma unroll
    for (int k = 0; k < kD; ++k) a[u][k] = row[desc_order(k)];
  }
  float best[kQF];
  int bj[kQF];
#pragma unroll
  for (int u = 0; u < kQF; ++u) best[u] = FLT_MAX, bj[u] = -1;
  unsigned nterm = 0;
  for (int base = 0, t = 0; base < nQ; base += kTile, ++t) {
    const bool need = __any_sync(0xffffffffu, tile_needed<kQF>(tb, t, a, best));
    // (also the barrier after the previous tile's scan)
    if (!__syncthreads_or(need)) continue;
    stage_tile(tile, FQ, base, nQ, rk);
    __syncthreads();
    if (need) scan_tile<kQF, kCount>(tile, nQ - base < kTile ? nQ - base : kTile, base, a, best, bj, &nterm);
  }
#pragma unroll
  for (int u = 0; u < kQF; ++u)
    if (qi[u] < nP) {
      nn[qi[u]] = bj[u];
      if (d1) d1[qi[u]] = best[u];
    }
  if (kCount) {
    int valid = 0;
#pragma unroll
    for (int u = 0; u < kQF; ++u) valid += qi[u] < nP;
    // nterm <= nQ * 33 < 2^32 (at most 2^26 points per cloud)
    unsigned long long mine = (unsigned long long)nterm * (unsigned)valid;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(terms, mine);
  }
}

// Exact FP32 scan of the queries rows[0..*nrows), split over database chunks
// (blockIdx.y) so that a short list still fills the GPU. Each block computes
// the chunk-local minimum exactly as k_match_fp32 does; chunks are combined
// with a 64-bit atomicMin on (distance bits << 32 | index), which for the
// non-negative distances keeps the smallest distance and, among equal
// distances, the smallest index -- the sequential scan's result.
__global__ void __launch_bounds__(kMT) k_match_rows_chunked(const float *__restrict__ FP, int nP,
                                                            const float *__restrict__ FQ, int nQ, int chunk,
                                                            const int *__restrict__ rows, const int *nrows,
                                                            unsigned long long *__restrict__ packed) {
  __shared__ float4 tile[kTile][9];
  const int nq = *nrows;
  const int j0 = blockIdx.y * chunk, j1 = min(nQ, j0 + chunk);
  if (j0 >= j1) return;
  int rk[4];
  stage_ranks(rk);
  for (int t0 = blockIdx.x; t0 * (kMT * kQR) < nq; t0 += gridDim.x) {
    float a[kQR][kD];
    int slot[kQR];
#pragma unroll
    for (int u = 0; u < kQR; ++u) {
      int q = t0 * (kMT * kQR) + u * kMT + threadIdx.x;
      slot[u] = q < nq ? q : -1;
      int qi = q < nq ? rows[q] : 0;
      const float *row = FP + (size_t)(qi < nP ? qi : 0) * kDS;
#pragma unroll
      for (int k = 0; k < kD; ++k) a[u][k] = row[desc_order(k)];
    }
    float best[kQR];
    int bj[kQR];
#pragma unroll
    for (int u = 0; u < kQR; ++u) best[u] = FLT_MAX, bj[u] = -1;
    for (int base = j0; base < j1; base += kTile) {
      __syncthreads();
      stage_tile(tile, FQ, base, j1, rk);
      __syncthreads();
      scan_tile<kQR>(tile, j1 - base < kTile ? j1 - base : kTile, base, a, best, bj);
    }
#pragma unroll
    for (int u = 0; u < kQR; ++u)
      if (slot[u] >= 0 && bj[u] >= 0 && LSR_IN_BOUNDS(slot[u], nP, kSiteMatchQuery))
        atomicMin(packed + slot[u], ((unsigned long long)__float_as_uint(best[u]) << 32) | (unsigned)bj[u]);
    __syncthreads();
  }
}

__global__ void k_rows_init(const int *nrows, int nP, unsigned long long *packed) {
  const int nq = *nrows;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x)
    if (LSR_IN_BOUNDS(q, nP, kSiteMatchQuery)) packed[q] = ~0ull;
}

__global__ void k_rows_finish(const int *rows, const int *nrows, int nP, const unsigned long long *packed, int *nn,
                              float *d1) {
  const int nq = *nrows;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    if (!LSR_IN_BOUNDS(q, nP, kSiteMatchQuery) || !LSR_IN_BOUNDS(rows[q], nP, kSiteMatchQuery)) continue;
    unsigned long long v = packed[q];
    int r = rows[q];
    bool none = v == ~0ull;
    nn[r] = none ? -1 : (int)(unsigned)(v & 0xFFFFFFFFu);
    if (d1) d1[r] = none ? FLT_MAX : __uint_as_float((unsigned)(v >> 32));
  }
}

}  // namespace

LSR_CHECK_READER(match)

size_t fp32_workspace_bytes(int nQ) { return sizeof(float) * kTB * (size_t)lsr_div_up(nQ, kTile) + 256; }

cudaError_t launch_match_fp32(const float *FP, int nP, const float *FQ, int nQ, void *ws, int *nn, float *d1,
                              cudaStream_t s, unsigned long long *terms) {
  int blocks = (int)lsr_div_up(nP, kMT * kQF);
  if (blocks < 1) blocks = 1;
  float *tb = static_cast<float *>(ws);
  LSR_LAUNCH(k_tile_bounds<<<(int)lsr_div_up(nQ, kTile), 64, 0, s>>>(FQ, nQ, tb));
  if (terms)
    LSR_LAUNCH(k_match_fp32<true><<<blocks, kMT, 0, s>>>(FP, nP, FQ, nQ, tb, nn, d1, terms));
  else
    LSR_LAUNCH(k_match_fp32<false><<<blocks, kMT, 0, s>>>(FP, nP, FQ, nQ, tb, nn, d1, nullptr));
  return cudaGetLastError();
}

cudaError_t launch_match_fp32_rows(const float *FP, int nP, const float *FQ, int nQ, const int *rows,
                                   const int *nrows, unsigned long long *packed, int *nn, float *d1,
                                   cudaStream_t s) {
  constexpr int kChunks = 64;
  int chunk = (int)lsr_div_up(lsr_div_up(nQ, kChunks), kTile) * kTile;
  int ny = (int)lsr_div_up(nQ, chunk);
  int nx = (int)lsr_div_up(nP, kMT * kQR);
  nx = nx < 1 ? 1 : (nx > 10 ? 10 : nx);
  int fin = (int)lsr_div_up(nP, 256);
  fin = fin < 1 ? 1 : (fin > 1216 ? 1216 : fin);
  LSR_LAUNCH(k_rows_init<<<fin, 256, 0, s>>>(nrows, nP, packed));
  LSR_LAUNCH(k_match_rows_chunked<<<dim3(nx, ny), kMT, 0, s>>>(FP, nP, FQ, nQ, chunk, rows, nrows, packed));
  LSR_LAUNCH(k_rows_finish<<<fin, 256, 0, s>>>(rows, nrows, nP, packed, nn, d1));
  return cudaGetLastError();
}

}  // namespace lsr
