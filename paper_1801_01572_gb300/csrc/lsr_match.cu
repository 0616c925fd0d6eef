// lsr_match.cu -- feature pre-matching cache on the FP32 cores (Algorithm 1,
// "Parallel FPFH feature pre-matching": nn[i] = NN of F(p_i) in F(Q)).
//
// Exact: nn[i] = argmin_j sum_k (a_k - b_k)^2 with ties to the smallest j,
// each distance accumulated as s = fma(t, t, s) over the 33 bins taken in
// desc_order (central bins first). What is exact is the result; the search
// visits only the database rows that could change it.
//
// Projection window. Both sets are ordered by their projection p = u . x on
// one unit direction u (the principal axis of a sample of the database,
// found by power iteration; any unit vector gives the same result, a good
// one visits fewer rows). By Cauchy-Schwarz |u . (a - b)| <= |u| |a - b|, so
// a database row whose projection lies farther than sqrt(best) from the
// query's cannot be nearer than the current best. One block takes 128
// consecutive queries of the projection order and scans database tiles of
// that order outward from its own projection, alternately to the right and
// to the left; a side ends once no query of the block can find a row there.
// The FP32 rounding of the projections (a bound per row from the error of an
// fma chain), of |u| and of the distance itself is taken into the test by
// directed rounding, so a row or a side is left out only when every
// computed distance in it exceeds the query's computed best: the nearest
// row and its ties are always scanned, and ties go to the smaller original
// index whatever the scan order. Ordering is a counting sort into as many
// buckets as points over the projections' range; the order within a bucket
// is arbitrary, so the per-tile projection bounds are made monotone by a
// suffix minimum (right side) and a prefix maximum (left side).
//
// Inside the window each thread keeps one query descriptor in registers;
// tiles of database descriptors are staged in shared memory in desc_order
// and read as broadcasts. The partial sums only grow (t^2 >= 0 and rounding
// is monotone), so a row whose partial sum already exceeds every query's
// current best in the warp can neither win nor tie: after 4, 8, 12, 16 and
// 24 terms the warp tests that and skips the rest of the row (same result).
// The 32 queries of a warp have nearly equal projections, and their best
// distances fall together.
#include <float.h>
#include <stddef.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kMT = 128;   // threads per block
constexpr int kQR = 2;     // queries per thread, listed rows (k_match_rows_chunked)
constexpr int kTile = 64;  // database rows per shared-memory tile
constexpr int kStageThreads = 9 * (kMT / 9);  // staging threads: one float4 column each
static_assert(kTile * 9 > kStageThreads, "staging covers the tile in several passes");
constexpr int kPcThreads = 256;  // k_pc1 block
constexpr int kPcSamples = 1024; // database rows sampled for the principal axis (in shared memory)
constexpr int kPcIters = 10;     // power iterations (the second axis of FPFH sets holds ~0.1 of the first's variance)
constexpr int kScanThreadsT = 1024;  // k_tile_scan block

// Direction and range of the projection order (one per matcher call).
struct ProjParams {
  float u[kD];       // unit direction, column order
  float fac;         // lower-bound factor of a squared projection gap (k_pc1)
  unsigned key_min;  // f2key of the smallest / largest finite projection
  unsigned key_max;
  int ntot;          // nQ + nP (read by the scan)
};

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
// desc_order), updating best / bj; row j of the tile is database row ids[j]
// (base + j when ids is null). A row replaces the best when its distance is
// smaller, or equal with a smaller index, so the result does not depend on
// the order in which rows are scanned. kCount: add the terms evaluated per
// query to terms.
template <int Q, bool kCount = false>
__device__ __forceinline__ void scan_tile(const float4 (*tile)[9], int m, int base, const int *ids,
                                          const float (&a)[Q][kD], float (&best)[Q], int (&bj)[Q],
                                          unsigned *terms = nullptr) {
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
        const int id = ids ? ids[j] : base + j;
#pragma unroll
        for (int u = 0; u < Q; ++u) {
          float t = a[u][32] - b32;
          s[u] = fmaf(t, t, s[u]);
          if (s[u] < best[u] || (s[u] == best[u] && id < bj[u])) best[u] = s[u], bj[u] = id;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- projection order
// Float <-> unsigned key whose unsigned order is the float order (finite values).
__device__ __forceinline__ unsigned f2key(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Block sum over the threads of w[k] for each of the kD components, in a
// fixed order (a butterfly within each warp, then the warps in order); out
// (shared) receives the kD sums. wred: kPcThreads / 32 x kD.
__device__ __forceinline__ void pc_block_sum(float (*wred)[kD], const float (&w)[kD], float *out) {
#pragma unroll
  for (int k = 0; k < kD; ++k) {
    float v = w[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kD) {
    float t = 0.f;
#pragma unroll
    for (int w8 = 0; w8 < kPcThreads / 32; ++w8) t += wred[w8][threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Principal axis of up to kPcSamples evenly spaced database rows (staged in
// shared memory, centred on their mean): kPcIters power iterations
// v <- sum_r c_r (c_r . v), normalised in FP32. Writes u, the factor
// fac = (1 - 6e-6) / |u|^2 (|u|^2 rounded up, the quotient down) by which a
// squared projection gap bounds a computed distance from below, and the
// initial keys of the projections' range.
__global__ void __launch_bounds__(kPcThreads) k_pc1(const float *__restrict__ FQ, int nQ, int nP, ProjParams *pp) {
  extern __shared__ float xs[];  // kPcSamples x kD
  __shared__ float wred[kPcThreads / 32][kD];
  __shared__ float mean[kD], v[kD], nv[kD];
  const int m = nQ < kPcSamples ? nQ : kPcSamples;
  float w[kD];
#pragma unroll
  for (int k = 0; k < kD; ++k) w[k] = 0.f;
  for (int i = threadIdx.x; i < m; i += kPcThreads) {
    const float *row = FQ + (size_t)((long long)i * nQ / m) * kDS;
#pragma unroll
    for (int k = 0; k < kD; ++k) {
      const float x = row[k];
      xs[i * kD + k] = x;
      w[k] += x;
    }
  }
  pc_block_sum(wred, w, mean);
  if (threadIdx.x < kD) {
    mean[threadIdx.x] = m > 0 ? mean[threadIdx.x] / (float)m : 0.f;
    // start away from any particular axis
    v[threadIdx.x] = 1.f + 0.25f * (float)((threadIdx.x * 7) % 5);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += kPcThreads)
#pragma unroll
    for (int k = 0; k < kD; ++k) xs[i * kD + k] -= mean[k];
  // (each thread reads back only its own rows until the first block sum)
  for (int it = 0; it < kPcIters; ++it) {
#pragma unroll
    for (int k = 0; k < kD; ++k) w[k] = 0.f;
    for (int i = threadIdx.x; i < m; i += kPcThreads) {
      const float *c = xs + i * kD;
      float d = 0.f;
#pragma unroll
      for (int k = 0; k < kD; ++k) d = fmaf(c[k], v[k], d);
#pragma unroll
      for (int k = 0; k < kD; ++k) w[k] = fmaf(d, c[k], w[k]);
    }
    pc_block_sum(wred, w, nv);
    if (threadIdx.x == 0) {
      float n2 = 0.f;
      for (int k = 0; k < kD; ++k) n2 = fmaf(nv[k], nv[k], n2);
      // a zero or non-finite update (identical rows) keeps the current axis
      if (n2 > 0.f && n2 <= FLT_MAX) {
        const float inv = rsqrtf(n2);
        for (int k = 0; k < kD; ++k) v[k] = nv[k] * inv;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    float n2 = 0.f;
    for (int k = 0; k < kD; ++k) n2 = fmaf(v[k], v[k], n2);
    const bool ok = n2 > 0.f && n2 <= FLT_MAX;
    const float inv = ok ? rsqrtf(n2) : 0.f;
    float r2 = 0.f;
    for (int k = 0; k < kD; ++k) {
      const float uk = ok ? v[k] * inv : (k == 0 ? 1.f : 0.f);
      pp->u[k] = uk;
      r2 = __fmaf_ru(uk, uk, r2);
    }
    // s >= (1 - 35 * 2^-24) |a - b|^2 for the fma chain of a distance, and
    // |a - b|^2 >= (u . (a - b))^2 / |u|^2
    pp->fac = __fdiv_rd(0.999994f, r2);
    pp->key_min = 0xFFFFFFFFu;
    pp->key_max = 0u;
    pp->ntot = nQ + nP;
  }
}

// Projection p = u . x (fma chain over the 33 bins in column order) and a
// bound e >= |p - u . x| (gamma_33 = 33 * 2^-24 / (1 - 33 * 2^-24) < 2e-6 of
// sum |u_k x_k|, rounded up) for every database row (elements 0..nQ) and
// every query (elements nQ..nQ+nP); the range of the finite projections.
__global__ void k_proj(const float *__restrict__ FP, int nP, const float *__restrict__ FQ, int nQ,
                       ProjParams *pp, float2 *__restrict__ pe) {
  __shared__ float su[kD];
  if (threadIdx.x < kD) su[threadIdx.x] = pp->u[threadIdx.x];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned kmin = 0xFFFFFFFFu, kmax = 0u;
  if (i < nQ + nP) {
    const float *row = i < nQ ? FQ + (size_t)i * kDS : FP + (size_t)(i - nQ) * kDS;
    float p = 0.f, S = 0.f;
#pragma unroll
    for (int k = 0; k < kD; ++k) {
      const float x = row[k];
      p = fmaf(su[k], x, p);
      S = __fmaf_ru(fabsf(su[k]), fabsf(x), S);
    }
    pe[i] = make_float2(p, __fmaf_ru(S, 2.0e-6f, 1e-37f));
    if (isfinite(p)) kmin = kmax = f2key(p);
  }
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  if ((threadIdx.x & 31) == 0 && kmin <= kmax) {
    atomicMin(&pp->key_min, kmin);
    atomicMax(&pp->key_max, kmax);
  }
}

// Bucket of every element: as many buckets per set as the set has elements,
// spread evenly over the projections' range (non-finite ones last); counts
// of the database's buckets first, then the queries'.
__global__ void k_bucket_count(const float2 *__restrict__ pe, int nQ, int nP, const ProjParams *pp,
                               int *__restrict__ slot, int *__restrict__ counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nQ + nP) return;
  const bool db = i < nQ;
  const int nb = db ? nQ : nP, off = db ? 0 : nQ;
  const unsigned k0 = pp->key_min, k1 = pp->key_max;
  const float lo = k0 <= k1 ? key2f(k0) : 0.f, hi = k0 <= k1 ? key2f(k1) : 0.f;
  const float inv = hi > lo ? (float)nb / (hi - lo) : 0.f;
  const float p = pe[i].x;
  int b = nb - 1;
  if (isfinite(p)) {
    const float f = (p - lo) * inv;
    b = f < (float)nb ? (int)f : nb - 1;
    b = b < 0 ? 0 : b;
  }
  slot[i] = off + b;
  atomicAdd(counts + off + b, 1);
}

// order[pos] = element at position pos of its set's bucket order (database
// positions 0..nQ, query positions nQ..nQ+nP); start is consumed as cursor.
__global__ void k_bucket_scatter(int n, const int *__restrict__ slot, int *start, int *__restrict__ order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int pos = atomicAdd(start + slot[i], 1);
  if (LSR_IN_BOUNDS(pos, n, kSiteMatchRow)) order[pos] = i;
}

// One block of kTile threads per database tile: the tile's rows in
// projection order (FQs), their original indices (dorig), and the tile's
// bounds lo <= p - e and hi >= p + e over its finite projections.
__global__ void __launch_bounds__(kTile) k_gather_db(const float *__restrict__ FQ, int nQ, const int *__restrict__ order,
                                                     const float2 *__restrict__ pe, float *__restrict__ FQs,
                                                     int *__restrict__ dorig, float *__restrict__ tlo,
                                                     float *__restrict__ thi) {
  __shared__ float slo[kTile / 32], shi[kTile / 32];
  const int pos = blockIdx.x * kTile + threadIdx.x;
  float lo = INFINITY, hi = -INFINITY;
  if (pos < nQ) {
    int i = order[pos];
    if (!LSR_IN_BOUNDS(i, nQ, kSiteMatchRow)) i = 0;
    const float4 *src = reinterpret_cast<const float4 *>(FQ + (size_t)i * kDS);
    float4 *dst = reinterpret_cast<float4 *>(FQs + (size_t)pos * kDS);
#pragma unroll
    for (int c = 0; c < kDS / 4; ++c) dst[c] = src[c];
    dorig[pos] = i;
    const float2 v = pe[i];
    if (isfinite(v.x)) lo = __fsub_rd(v.x, v.y), hi = __fadd_ru(v.x, v.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) slo[threadIdx.x >> 5] = lo, shi[threadIdx.x >> 5] = hi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kTile / 32; ++w) lo = fminf(lo, slo[w]), hi = fmaxf(hi, shi[w]);
    tlo[blockIdx.x] = lo;
    thi[blockIdx.x] = hi;
  }
}

// smin[t] = min over tiles t' >= t of tlo, hmax[t] = max over tiles t' <= t
// of thi: bounds that only grow to the right (shrink to the left), so a side
// of the window that no query needs stays unneeded.
__global__ void __launch_bounds__(kScanThreadsT) k_tile_scan(const float *__restrict__ tlo,
                                                             const float *__restrict__ thi, int nt,
                                                             float *__restrict__ smin, float *__restrict__ hmax) {
  __shared__ float a[kScanThreadsT], b[kScanThreadsT];
  const int per = (nt + kScanThreadsT - 1) / kScanThreadsT;
  const int t0 = threadIdx.x * per, t1 = min(nt, t0 + per);
  float lo = INFINITY, hi = -INFINITY;
  for (int t = t0; t < t1; ++t) lo = fminf(lo, tlo[t]), hi = fmaxf(hi, thi[t]);
  a[threadIdx.x] = lo, b[threadIdx.x] = hi;
  __syncthreads();
  // inclusive scans over the threads' segments: a from the right, b from the left
  for (int off = 1; off < kScanThreadsT; off <<= 1) {
    const int x = threadIdx.x;
    const float va = x + off < kScanThreadsT ? a[x + off] : INFINITY;
    const float vb = x >= off ? b[x - off] : -INFINITY;
    __syncthreads();
    a[x] = fminf(a[x], va), b[x] = fmaxf(b[x], vb);
    __syncthreads();
  }
  float run_lo = threadIdx.x + 1 < kScanThreadsT ? a[threadIdx.x + 1] : INFINITY;
  float run_hi = threadIdx.x > 0 ? b[threadIdx.x - 1] : -INFINITY;
  for (int t = t1 - 1; t >= t0; --t) run_lo = fminf(run_lo, tlo[t]), smin[t] = run_lo;
  for (int t = t0; t < t1; ++t) run_hi = fmaxf(run_hi, thi[t]), hmax[t] = run_hi;
}

// Squared projection gap g^2 (g rounded down, then the product and the
// factor) that bounds every computed distance on that side from below; 0 for
// gaps below 1e-18 (where subnormal terms of a distance lose their relative
// rounding bound) and for non-finite gaps other than +inf.
__device__ __forceinline__ float gap_bound(float g, float fac) {
  return g > 1e-18f ? __fmul_rd(__fmul_rd(g, g), fac) : 0.f;
}

// One block: the 128 queries at projection positions 128 b .. 128 b + 127.
// The window starts at the tile where the block's middle projection falls
// and grows alternately to the right and to the left; a side ends when no
// query of the block needs its next tile (the monotone bounds make that
// final), a warp scans a staged tile only if one of its queries needs it.
// kCount: also add the number of terms (a_k - b_k)^2 evaluated for the valid
// queries to *terms (a separate instantiation, used when profiling).
template <bool kCount>
__global__ void __launch_bounds__(kMT) k_match_win(const float *__restrict__ FP, int nP,
                                                   const float *__restrict__ FQs, const int *__restrict__ dorig,
                                                   int nQ, const int *__restrict__ order,
                                                   const float2 *__restrict__ pe, const float *__restrict__ smin,
                                                   const float *__restrict__ hmax, const ProjParams *pp,
                                                   int *__restrict__ nn, float *__restrict__ d1,
                                                   unsigned long long *__restrict__ terms) {
  __shared__ float4 tile[kTile][9];
  __shared__ int ids[kTile];
  const int nt = (int)lsr_div_up(nQ, kTile);
  const int k = blockIdx.x * kMT + threadIdx.x;
  const bool valid = k < nP;
  int qo = 0;
  if (valid) {
    qo = order[nQ + k] - nQ;
    if (!LSR_IN_BOUNDS(qo, nP, kSiteMatchQuery)) qo = 0;
  }
  float a[1][kD];
  {
    const float *row = FP + (size_t)qo * kDS;
#pragma unroll
    for (int j = 0; j < kD; ++j) a[0][j] = row[desc_order(j)];
  }
  const float2 q = pe[nQ + qo];
  const float fac = pp->fac;
  // invalid lanes: best below any distance, so they never hold a warp back
  float best[1] = {valid ? FLT_MAX : -1.f};
  int bj[1] = {-1};
  int rk[4];
  stage_ranks(rk);
  // start tile: the last one whose suffix minimum does not exceed the block's
  // middle projection (0 when it is not finite)
  int t0 = 0;
  {
    const int mid = min(blockIdx.x * kMT + kMT / 2, nP - 1);
    const float pm = pe[order[nQ + mid]].x;
    if (isfinite(pm) && nt > 0) {
      int lo = 0, hi = nt;  // first t with smin[t] > pm
      while (lo < hi) {
        const int md = (lo + hi) >> 1;
        if (smin[md] > pm) hi = md; else lo = md + 1;
      }
      t0 = lo > 0 ? lo - 1 : 0;
    }
  }
  unsigned nterm = 0;
  int r = t0, l = t0 - 1;
  bool rgo = r < nt, lgo = l >= 0, right_turn = true;
  while (rgo || lgo) {
    const bool right = rgo && (right_turn || !lgo);
    right_turn = !right;
    const int t = right ? r : l;
    const float g = right ? __fsub_rd(__fsub_rd(smin[t], q.x), q.y) : __fsub_rd(__fsub_rd(q.x, hmax[t]), q.y);
    const bool need = valid && !(gap_bound(g, fac) > best[0]);
    const bool wneed = __any_sync(0xffffffffu, need);
    // (also the barrier after the previous tile's scan)
    if (!__syncthreads_or(need)) {
      (right ? rgo : lgo) = false;
      continue;
    }
    if (right) rgo = ++r < nt;
    else lgo = --l >= 0;
    const int base = t * kTile, m = nQ - base < kTile ? nQ - base : kTile;
    stage_tile(tile, FQs, base, nQ, rk);
    if (threadIdx.x < kTile) ids[threadIdx.x] = threadIdx.x < m ? dorig[base + threadIdx.x] : 0x7FFFFFFF;
    __syncthreads();
    if (wneed) scan_tile<1, kCount>(tile, m, base, ids, a, best, bj, &nterm);
  }
  if (valid && LSR_IN_BOUNDS(qo, nP, kSiteMatchQuery)) {
    nn[qo] = bj[0];
    if (d1) d1[qo] = bj[0] >= 0 ? best[0] : FLT_MAX;
  }
  if (kCount) {
    // nterm <= nQ * 33 < 2^32 (at most 2^26 points per cloud)
    unsigned long long mine = valid ? (unsigned long long)nterm : 0ull;
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
      scan_tile<kQR>(tile, j1 - base < kTile ? j1 - base : kTile, base, nullptr, a, best, bj);
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

namespace {

struct Fp32Layout {
  ProjParams *pp;
  float2 *pe;                      // (p, e) of the nQ database rows, then the nP queries
  int *slot, *counts, *start, *order, *scan;
  float *FQs;                      // database rows in projection order
  int *dorig;                      // their original indices
  float *tlo, *thi, *smin, *hmax;  // per tile
  size_t bytes;
};

Fp32Layout fp32_layout(char *base, int nP, int nQ) {
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t n = (size_t)nP + (size_t)nQ, nt = (size_t)lsr_div_up(nQ, kTile);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *p = base ? base + off : nullptr;
    off += al(bytes > 0 ? bytes : 1);
    return p;
  };
  Fp32Layout L;
  L.pp = reinterpret_cast<ProjParams *>(take(sizeof(ProjParams)));
  L.pe = reinterpret_cast<float2 *>(take(sizeof(float2) * n));
  L.slot = reinterpret_cast<int *>(take(sizeof(int) * n));
  L.counts = reinterpret_cast<int *>(take(sizeof(int) * (n + 1)));
  L.start = reinterpret_cast<int *>(take(sizeof(int) * (n + 1)));
  L.order = reinterpret_cast<int *>(take(sizeof(int) * n));
  L.scan = reinterpret_cast<int *>(take(sizeof(int) * (size_t)scan_scratch_ints((int64_t)n)));
  L.FQs = reinterpret_cast<float *>(take(sizeof(float) * kDS * (size_t)nQ));
  L.dorig = reinterpret_cast<int *>(take(sizeof(int) * (size_t)nQ));
  L.tlo = reinterpret_cast<float *>(take(sizeof(float) * nt));
  L.thi = reinterpret_cast<float *>(take(sizeof(float) * nt));
  L.smin = reinterpret_cast<float *>(take(sizeof(float) * nt));
  L.hmax = reinterpret_cast<float *>(take(sizeof(float) * nt));
  L.bytes = off;
  return L;
}

}  // namespace

size_t fp32_workspace_bytes(int nP, int nQ) { return fp32_layout(nullptr, nP, nQ).bytes; }

cudaError_t launch_match_fp32(const float *FP, int nP, const float *FQ, int nQ, void *ws, int *nn, float *d1,
                              cudaStream_t s, unsigned long long *terms) {
  if (nP < 1) return cudaSuccess;
  Fp32Layout L = fp32_layout(static_cast<char *>(ws), nP, nQ);
  const int n = nP + nQ, nt = (int)lsr_div_up(nQ, kTile);
  LSR_CUDA_TRY(cudaMemsetAsync(L.counts, 0, sizeof(int) * ((size_t)n + 1), s));
  constexpr int kPcSmem = kPcSamples * kD * (int)sizeof(float);
  LSR_CUDA_TRY(cudaFuncSetAttribute(k_pc1, cudaFuncAttributeMaxDynamicSharedMemorySize, kPcSmem));
  LSR_LAUNCH(k_pc1<<<1, kPcThreads, kPcSmem, s>>>(FQ, nQ, nP, L.pp));
  const int eb = (int)lsr_div_up(n, 256);
  LSR_LAUNCH(k_proj<<<eb, 256, 0, s>>>(FP, nP, FQ, nQ, L.pp, L.pe));
  LSR_LAUNCH(k_bucket_count<<<eb, 256, 0, s>>>(L.pe, nQ, nP, L.pp, L.slot, L.counts));
  LSR_CUDA_TRY(scan_exclusive(L.counts, L.start,
                                  reinterpret_cast<int *>(reinterpret_cast<char *>(L.pp) + offsetof(ProjParams, ntot)),
                                  n, L.scan, s));
  LSR_LAUNCH(k_bucket_scatter<<<eb, 256, 0, s>>>(n, L.slot, L.start, L.order));
  if (nt > 0) {
    LSR_LAUNCH(k_gather_db<<<nt, kTile, 0, s>>>(FQ, nQ, L.order, L.pe, L.FQs, L.dorig, L.tlo, L.thi));
    LSR_LAUNCH(k_tile_scan<<<1, kScanThreadsT, 0, s>>>(L.tlo, L.thi, nt, L.smin, L.hmax));
  }
  const int blocks = (int)lsr_div_up(nP, kMT);
  if (terms)
    LSR_LAUNCH(k_match_win<true><<<blocks, kMT, 0, s>>>(FP, nP, L.FQs, L.dorig, nQ, L.order, L.pe, L.smin, L.hmax,
                                                        L.pp, nn, d1, terms));
  else
    LSR_LAUNCH(k_match_win<false><<<blocks, kMT, 0, s>>>(FP, nP, L.FQs, L.dorig, nQ, L.order, L.pe, L.smin, L.hmax,
                                                         L.pp, nn, d1, nullptr));
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
