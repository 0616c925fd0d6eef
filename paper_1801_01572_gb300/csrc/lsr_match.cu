// lsr_match.cu -- feature pre-matching cache on the FP32 cores (Algorithm 1,
// "Parallel FPFH feature pre-matching": nn[i] = NN of F(p_i) in F(Q)).
//
// Exact: nn[i] = argmin_j sum_k (a_k - b_k)^2 with ties to the smallest j,
// each distance accumulated as s = fma(t, t, s) over the 33 bins taken in
// desc_order (central bins first). What is exact is the result; the search
// visits only the database rows that could change it.
//
// Projection window. Both sets are ordered by their projections p1 = u1 . x
// and p2 = u2 . x on the first two principal axes of a sample of the
// database (power iteration; any pair of directions gives the same result,
// good ones visit fewer rows): by p1, then, inside slabs of 1024 consecutive
// rows, by p2. For the stored FP32 axes U = [u1 u2], |U^T (a - b)|^2 <=
// lambda |a - b|^2 with lambda bounding the Gram matrix's largest
// eigenvalue, so a database row whose projections lie farther than
// sqrt(lambda * best) from the query's, in the plane of the two axes, cannot
// be nearer than the current best. A warp takes 32 consecutive queries of
// that order (one query slab: close in p1 and in p2) and one database slab of
// their window at a time (persistent warps, work items taken breadth-first:
// every group's nearest slabs before any group's farther ones); in a slab it
// visits the tiles outward from its own p2, and a side ends once no query of
// the warp can find a row there. Best distances are shared between the warps
// of a group by a 64-bit atomic minimum of (distance, index). The FP32
// rounding of the projections (a bound per row from the error of an fma
// chain), of the axes and of the distance itself is taken into the test by
// directed rounding, so a row, a tile or a slab is left out only when every
// computed distance in it exceeds a distance some row has: the nearest row
// and its ties are always scanned, and ties go to the smaller original index
// whatever the scan order. Each ordering is a counting sort into as many
// buckets as rows over the projections' range; the order within a bucket is
// arbitrary, so the bounds that end a side are made monotone by suffix minima
// (right) and prefix maxima (left).
//
// Inside the window each thread keeps one query descriptor in registers and
// reads the database rows (bins in desc_order, chunk-major per tile) through
// L1 as warp broadcasts. The partial sums only grow (t^2 >= 0 and rounding is
// monotone), so a row whose partial sum already exceeds every query's
// current best in the warp can neither win nor tie: after 4, 8, 12, 16 and
// 24 terms the warp tests that and skips the rest of the row (same result).
// The 32 queries of a warp have nearly equal projections, and their best
// distances fall together. The listed-rows scan of the tensor-core path's
// exact fallback (k_match_rows_chunked) stages tiles in shared memory.
#include <float.h>
#include <stddef.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kMT = 128;   // threads per block
constexpr int kQR = 2;     // queries per thread, listed rows (k_match_rows_chunked)
constexpr int kTile = 32;  // database rows per tile (32 measured faster than 64 or 128 in the window search)
constexpr int kStageThreads = 9 * (kMT / 9);  // staging threads: one float4 column each
static_assert(kTile * 9 > kStageThreads, "staging covers the tile in several passes");
constexpr int kSlab = 1024;      // rows of a slab: consecutive in p1, ordered by p2 inside
constexpr int kTilesPerSlab = kSlab / kTile;
static_assert(kSlab % kTile == 0 && kSlab % kMT == 0, "tiles and query blocks do not straddle slabs");
constexpr int kPcThreads = 256;  // k_pc block
constexpr int kPcSamples = 1024; // database rows sampled for the principal axes (in shared memory)
constexpr int kPcIters = 10;     // power iterations per axis (FPFH sets: variance ratios ~0.1 and ~0.4)
constexpr int kScanThreadsT = 1024;  // k_bound_scan block
constexpr int kItemRun = 2;          // matcher work items taken per counter increment (more: later slabs overtake nearer ones)

// Directions and ranges of the projection order (one per matcher call).
struct ProjParams {
  float u[2][kD];       // the two unit directions, column order
  float fac;            // lower-bound factor of a sum of squared projection gaps (k_pc)
  unsigned key_min[2];  // f2key of the smallest / largest finite projection per direction
  unsigned key_max[2];
  int ntot;             // nQ + nP (read by the first sort's scan)
  int ncap2;            // buckets of the second sort (read by its scan)
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

// kPcIters power iterations v <- sum_r c_r (c_r . v) over the centred
// samples cs (m x kD, shared), removing the component along `away` (unit,
// or null) after each product; v is normalised in FP32, and kept when an
// update is zero or not finite.
__device__ void pc_power(const float *cs, int m, float (*wred)[kD], float *v, float *nv, const float *away) {
  for (int it = 0; it < kPcIters; ++it) {
    float w[kD];
#pragma unroll
    for (int k = 0; k < kD; ++k) w[k] = 0.f;
    for (int i = threadIdx.x; i < m; i += kPcThreads) {
      const float *c = cs + i * kD;
      float d = 0.f;
#pragma unroll
      for (int k = 0; k < kD; ++k) d = fmaf(c[k], v[k], d);
#pragma unroll
      for (int k = 0; k < kD; ++k) w[k] = fmaf(d, c[k], w[k]);
    }
    pc_block_sum(wred, w, nv);
    if (threadIdx.x == 0) {
      if (away) {
        float d = 0.f;
        for (int k = 0; k < kD; ++k) d = fmaf(nv[k], away[k], d);
        for (int k = 0; k < kD; ++k) nv[k] = fmaf(-d, away[k], nv[k]);
      }
      float n2 = 0.f;
      for (int k = 0; k < kD; ++k) n2 = fmaf(nv[k], nv[k], n2);
      if (n2 > 0.f && n2 <= FLT_MAX) {
        const float inv = rsqrtf(n2);
        for (int k = 0; k < kD; ++k) v[k] = nv[k] * inv;
      }
    }
    __syncthreads();
  }
}

// The first two principal axes u1, u2 of up to kPcSamples evenly spaced
// database rows (staged in shared memory, centred on their mean), by power
// iteration (u2 kept orthogonal to u1). Writes both, the factor fac by which
// the sum of the two squared projection gaps bounds a computed distance from
// below, the initial keys of the two projections' ranges and the sizes the
// sorts read. fac = (1 - 6e-6) / lambda, lambda >= the largest eigenvalue of
// the 2 x 2 Gram matrix of the stored FP32 axes (max |u_i|^2 + |u1 . u2|,
// Gershgorin, all rounded up): |U^T x|^2 <= lambda |x|^2 for U = [u1 u2],
// and a computed distance is >= (1 - 35 * 2^-24) |a - b|^2.
__global__ void __launch_bounds__(kPcThreads) k_pc(const float *__restrict__ FQ, int nQ, int nP, int ncap2,
                                                   ProjParams *pp) {
  extern __shared__ float xs[];  // kPcSamples x kD
  __shared__ float wred[kPcThreads / 32][kD];
  __shared__ float mean[kD], v1[kD], v2[kD], nv[kD];
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
    // starts away from any particular axis and from each other
    v1[threadIdx.x] = 1.f + 0.25f * (float)((threadIdx.x * 7) % 5);
    v2[threadIdx.x] = (threadIdx.x & 1) ? 1.f : -0.75f - 0.125f * (float)(threadIdx.x % 3);
  }
  __syncthreads();
  // each thread centres its own rows, which it alone reads until the first block sum
  for (int i = threadIdx.x; i < m; i += kPcThreads)
#pragma unroll
    for (int k = 0; k < kD; ++k) xs[i * kD + k] -= mean[k];
  pc_power(xs, m, wred, v1, nv, nullptr);
  if (threadIdx.x == 0) {
    // v1 as stored (normalised, or the first coordinate axis when no
    // iteration produced a direction)
    float n2 = 0.f;
    for (int k = 0; k < kD; ++k) n2 = fmaf(v1[k], v1[k], n2);
    const bool ok = n2 > 0.f && n2 <= FLT_MAX;
    const float inv = ok ? rsqrtf(n2) : 0.f;
    for (int k = 0; k < kD; ++k) v1[k] = ok ? v1[k] * inv : (k == 0 ? 1.f : 0.f);
  }
  __syncthreads();
  pc_power(xs, m, wred, v2, nv, v1);
  if (threadIdx.x == 0) {
    // final re-orthogonalisation and normalisation of u2 (the second
    // coordinate axis when nothing is left)
    float d = 0.f;
    for (int k = 0; k < kD; ++k) d = fmaf(v2[k], v1[k], d);
    for (int k = 0; k < kD; ++k) v2[k] = fmaf(-d, v1[k], v2[k]);
    float n2 = 0.f;
    for (int k = 0; k < kD; ++k) n2 = fmaf(v2[k], v2[k], n2);
    const bool ok = n2 > 1e-12f && n2 <= FLT_MAX;
    const float inv = ok ? rsqrtf(n2) : 0.f;
    float r1 = 0.f, r2 = 0.f, c = 0.f;
    for (int k = 0; k < kD; ++k) {
      const float a = v1[k], b = ok ? v2[k] * inv : (k == 1 ? 1.f : 0.f);
      pp->u[0][k] = a;
      pp->u[1][k] = b;
      r1 = __fmaf_ru(a, a, r1);
      r2 = __fmaf_ru(b, b, r2);
      c = fmaf(a, b, c);
    }
    // |u1 . u2| <= |c| + gamma_33 |u1| |u2| (both norms below 1 + 1e-6)
    const float lam = __fadd_ru(fmaxf(r1, r2), __fadd_ru(fabsf(c), 2.1e-6f));
    pp->fac = __fdiv_rd(0.999994f, lam);
    pp->key_min[0] = pp->key_min[1] = 0xFFFFFFFFu;
    pp->key_max[0] = pp->key_max[1] = 0u;
    pp->ntot = nQ + nP;
    pp->ncap2 = ncap2;
  }
}

// Projections p_j = u_j . x (fma chains over the 33 bins in column order)
// and bounds e_j >= |p_j - u_j . x| (gamma_33 = 33 * 2^-24 / (1 - 33 * 2^-24)
// < 2e-6 of sum |u_jk x_k|, rounded up) for every database row (elements
// 0..nQ) and every query (elements nQ..nQ+nP), as (p1, e1, p2, e2); the
// ranges of the finite projections.
__global__ void k_proj(const float *__restrict__ FP, int nP, const float *__restrict__ FQ, int nQ,
                       ProjParams *pp, float4 *__restrict__ pe) {
  __shared__ float su[2][kD];
  if (threadIdx.x < 2 * kD) su[threadIdx.x / kD][threadIdx.x % kD] = pp->u[threadIdx.x / kD][threadIdx.x % kD];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned kmin[2] = {0xFFFFFFFFu, 0xFFFFFFFFu}, kmax[2] = {0u, 0u};
  if (i < nQ + nP) {
    const float *row = i < nQ ? FQ + (size_t)i * kDS : FP + (size_t)(i - nQ) * kDS;
    float p[2] = {0.f, 0.f}, S[2] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kD; ++k) {
      const float x = row[k];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        p[j] = fmaf(su[j][k], x, p[j]);
        S[j] = __fmaf_ru(fabsf(su[j][k]), fabsf(x), S[j]);
      }
    }
    pe[i] = make_float4(p[0], __fmaf_ru(S[0], 2.0e-6f, 1e-37f), p[1], __fmaf_ru(S[1], 2.0e-6f, 1e-37f));
#pragma unroll
    for (int j = 0; j < 2; ++j)
      if (isfinite(p[j])) kmin[j] = kmax[j] = f2key(p[j]);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const unsigned lo = __reduce_min_sync(0xffffffffu, kmin[j]), hi = __reduce_max_sync(0xffffffffu, kmax[j]);
    if ((threadIdx.x & 31) == 0 && lo <= hi) {
      atomicMin(&pp->key_min[j], lo);
      atomicMax(&pp->key_max[j], hi);
    }
  }
}

// Bucket in [0, nb) of a projection over the range of direction j (non-finite
// values last).
__device__ __forceinline__ int proj_bucket(float p, const ProjParams *pp, int j, int nb) {
  const unsigned k0 = pp->key_min[j], k1 = pp->key_max[j];
  if (!(k0 <= k1) || !isfinite(p)) return nb - 1;
  const float lo = key2f(k0), hi = key2f(k1);
  const float inv = hi > lo ? (float)nb / (hi - lo) : 0.f;
  const float f = (p - lo) * inv;
  const int b = f < (float)nb ? (int)f : nb - 1;
  return b < 0 ? 0 : b;
}

// First sort, by p1: as many buckets per set as the set has elements; counts
// of the database's buckets first, then the queries'.
__global__ void k_bucket1(const float4 *__restrict__ pe, int nQ, int nP, const ProjParams *pp,
                          int *__restrict__ slot, int *__restrict__ counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nQ + nP) return;
  const bool db = i < nQ;
  const int s = (db ? 0 : nQ) + proj_bucket(pe[i].x, pp, 0, db ? nQ : nP);
  slot[i] = s;
  atomicAdd(counts + s, 1);
}

// Second sort: position pos of the p1 order lies in slab pos / kSlab of its
// set; inside the slab, kSlab buckets of p2. Database slabs first (capD
// buckets), then the queries'.
__global__ void k_bucket2(const float4 *__restrict__ pe, const int *__restrict__ order1, int nQ, int nP, int capD,
                          const ProjParams *pp, int *__restrict__ slot, int *__restrict__ counts) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nQ + nP) return;
  const bool db = pos < nQ;
  const int r = db ? pos : pos - nQ;
  const int i = order1[pos];
  const int s = (db ? 0 : capD) + (r / kSlab) * kSlab + proj_bucket(pe[i].z, pp, 1, kSlab);
  slot[pos] = s;
  atomicAdd(counts + s, 1);
}

// out[start[slot[j]]++] = src ? src[j] : j (start is consumed as cursor).
__global__ void k_bucket_scatter(int n, const int *__restrict__ slot, int *start, const int *__restrict__ src,
                                 int *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int pos = atomicAdd(start + slot[j], 1);
  if (LSR_IN_BOUNDS(pos, n, kSiteMatchRow)) out[pos] = src ? src[j] : j;
}

// One block of kTile threads per database tile: the tile's rows in the final
// order (FQs: per tile, float4 chunk c of row j at c * kTile + j, bins in
// desc_order, zeros in slots 33..35), their original indices (dorig), and the tile's box of the
// projection intervals, (lo1, hi1, lo2, hi2) with lo <= p - e and hi >= p + e
// over its finite projections (empty: +inf, -inf).
__global__ void __launch_bounds__(kTile) k_gather_db(const float *__restrict__ FQ, int nQ, const int *__restrict__ order,
                                                     const float4 *__restrict__ pe, float *__restrict__ FQs,
                                                     int *__restrict__ dorig, float4 *__restrict__ tbox) {
  __shared__ float4 sb[kTile / 32];
  const int pos = blockIdx.x * kTile + threadIdx.x;
  float lo1 = INFINITY, hi1 = -INFINITY, lo2 = INFINITY, hi2 = -INFINITY;
  if (pos < nQ) {
    int i = order[pos];
    if (!LSR_IN_BOUNDS(i, nQ, kSiteMatchRow)) i = 0;
    const float *src = FQ + (size_t)i * kDS;
    float4 *dst = reinterpret_cast<float4 *>(FQs) + (size_t)blockIdx.x * (9 * kTile) + threadIdx.x;
#pragma unroll
    for (int c = 0; c < kDS / 4; ++c) {
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = 4 * c + e < kD ? src[desc_order(4 * c + e)] : 0.f;
      dst[c * kTile] = make_float4(v[0], v[1], v[2], v[3]);
    }
    dorig[pos] = i;
    const float4 v = pe[i];
    if (isfinite(v.x)) lo1 = __fsub_rd(v.x, v.y), hi1 = __fadd_ru(v.x, v.y);
    if (isfinite(v.z)) lo2 = __fsub_rd(v.z, v.w), hi2 = __fadd_ru(v.z, v.w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
    hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
    lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
    hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
  }
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = make_float4(lo1, hi1, lo2, hi2);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kTile / 32; ++w)
      lo1 = fminf(lo1, sb[w].x), hi1 = fmaxf(hi1, sb[w].y), lo2 = fminf(lo2, sb[w].z), hi2 = fmaxf(hi2, sb[w].w);
    tbox[blockIdx.x] = make_float4(lo1, hi1, lo2, hi2);
  }
}

// One thread per database slab: the slab's p1 interval (slo1, shi1) and,
// over its tiles in order, the suffix minimum of lo2 (smin2) and the prefix
// maximum of hi2 (hmax2): p2 bounds that only grow to the right (shrink to
// the left) within the slab.
__global__ void k_slab_bounds(const float4 *__restrict__ tbox, int nt, int ns, float *__restrict__ slo1,
                              float *__restrict__ shi1, float *__restrict__ smin2, float *__restrict__ hmax2) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const int a = s * kTilesPerSlab, b = min(nt, a + kTilesPerSlab);
  float lo = INFINITY, hi = -INFINITY, run = -INFINITY;
  for (int t = a; t < b; ++t) {
    const float4 x = tbox[t];
    lo = fminf(lo, x.x), hi = fmaxf(hi, x.y);
    run = fmaxf(run, x.w), hmax2[t] = run;
  }
  run = INFINITY;
  for (int t = b - 1; t >= a; --t) run = fminf(run, tbox[t].z), smin2[t] = run;
  slo1[s] = lo;
  shi1[s] = hi;
}

// smin[t] = min over entries t' >= t of lo, hmax[t] = max over t' <= t of
// hi (one block): bounds that only grow to the right (shrink to the left).
__global__ void __launch_bounds__(kScanThreadsT) k_bound_scan(const float *__restrict__ lo_in,
                                                              const float *__restrict__ hi_in, int nt,
                                                              float *__restrict__ smin, float *__restrict__ hmax) {
  __shared__ float a[kScanThreadsT], b[kScanThreadsT];
  const int per = (nt + kScanThreadsT - 1) / kScanThreadsT;
  const int t0 = threadIdx.x * per, t1 = min(nt, t0 + per);
  float lo = INFINITY, hi = -INFINITY;
  for (int t = t0; t < t1; ++t) lo = fminf(lo, lo_in[t]), hi = fmaxf(hi, hi_in[t]);
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
  for (int t = t1 - 1; t >= t0; --t) run_lo = fminf(run_lo, lo_in[t]), smin[t] = run_lo;
  for (int t = t0; t < t1; ++t) run_hi = fmaxf(run_hi, hi_in[t]), hmax[t] = run_hi;
}

// Lower bound of every computed distance from a query whose projection
// intervals are separated by gaps g1, g2 (rounded down, >= 0) from those of
// the rows: (g1^2 + g2^2) * fac, rounded down. Gaps below 1e-18 count as 0
// (subnormal terms of a distance lose their relative rounding bound); +inf
// gives +inf.
__device__ __forceinline__ float gap_bound(float g1, float g2, float fac) {
  const float a = g1 > 1e-18f ? __fmul_rd(g1, g1) : 0.f, b = g2 > 1e-18f ? __fmul_rd(g2, g2) : 0.f;
  return __fmul_rd(__fadd_rd(a, b), fac);
}

// Gap, rounded down and >= 0, between the query's interval [ql, qh] and [lo, hi].
__device__ __forceinline__ float interval_gap(float lo, float hi, float ql, float qh) {
  return fmaxf(fmaxf(__fsub_rd(lo, qh), __fsub_rd(ql, hi)), 0.f);
}

// Scan the m rows of database tile t (final order, chunk-major: float4 chunk
// c of row j at T4[c * kTile + j], bins in desc_order) for this lane's query
// a, with the same partial-sum exits as scan_tile. The rows are read through
// L1 as warp broadcasts; consecutive rows share the cache lines of a chunk,
// and the next row's first chunk is loaded ahead (L1 prefetches of the lines
// further ahead measured slower: 4.74 against 4.57 ms). best is the lane's
// pruning bound (its own best or a smaller one another warp published); a
// row is taken when its distance is smaller, or equal with a smaller index
// than a row already taken (bj = -2: the bound came from elsewhere, so an
// equal row is taken and the atomic minimum of the published pairs decides);
// taken marks that there is a pair to publish.
template <bool kCount>
__device__ __forceinline__ void scan_rows(const float4 *__restrict__ T4, const int *__restrict__ ids, int m,
                                          const float (&a)[kD], float &best, int &bj, bool &taken, unsigned &terms) {
  float4 nxt = __ldg(T4);
#pragma unroll 4
  for (int j = 0; j < m; ++j) {
    float4 b = nxt;
    if (j + 1 < m) nxt = __ldg(T4 + j + 1);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c >= 1) {
        if (c <= 4 || c == 6)
          if (__all_sync(0xffffffffu, s > best)) break;
        b = __ldg(T4 + c * kTile + j);
      }
      if (kCount) terms += c == 7 ? 5 : 4;
      const float t0 = a[4 * c] - b.x, t1 = a[4 * c + 1] - b.y, t2 = a[4 * c + 2] - b.z, t3 = a[4 * c + 3] - b.w;
      s = fmaf(t0, t0, s);
      s = fmaf(t1, t1, s);
      s = fmaf(t2, t2, s);
      s = fmaf(t3, t3, s);
      if (c == 7) {
        const float t = a[32] - __ldg(reinterpret_cast<const float *>(T4 + 8 * kTile + j));
        s = fmaf(t, t, s);
        if (s < best || (s == best && bj != -1)) {
          const int id = __ldg(ids + j);
          if (s < best || (unsigned)id < (unsigned)bj) best = s, bj = id, taken = true;
        }
      }
    }
  }
}

__device__ __forceinline__ unsigned long long pack_pair(float d, int j) {
  return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)j;
}

// Queries in the final order: desc_order rows (FPs, zeros in slots 33..35)
// and their original indices (qorig); one thread per query position.
__global__ void k_gather_q(const float *__restrict__ FP, int nP, int nQ, const int *__restrict__ order,
                           float *__restrict__ FPs, int *__restrict__ qorig) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nP) return;
  int i = order[nQ + pos] - nQ;
  if (!LSR_IN_BOUNDS(i, nP, kSiteMatchQuery)) i = 0;
  const float *src = FP + (size_t)i * kDS;
  float4 *dst = reinterpret_cast<float4 *>(FPs + (size_t)pos * kDS);
#pragma unroll
  for (int c = 0; c < kDS / 4; ++c) {
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = 4 * c + e < kD ? src[desc_order(4 * c + e)] : 0.f;
    dst[c] = make_float4(v[0], v[1], v[2], v[3]);
  }
  qorig[pos] = i;
}

// Per query group (32 consecutive query positions): the slab where its
// middle p1 falls (the last whose suffix minimum of lo1 does not exceed it;
// 0 when it is not finite) and its middle p2.
__global__ void k_group_start(const float4 *__restrict__ pe, const int *__restrict__ qorig, int nP, int nQ,
                              const float *__restrict__ smin1, int *__restrict__ gs0, float *__restrict__ gm2) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int G = (int)lsr_div_up(nP, 32), ns = (int)lsr_div_up(nQ, kSlab);
  if (g >= G) return;
  const float4 q = pe[nQ + qorig[min(g * 32 + 16, nP - 1)]];
  int s0 = 0;
  if (isfinite(q.x)) {
    int lo = 0, hi = ns;
    while (lo < hi) {
      const int md = (lo + hi) >> 1;
      if (smin1[md] > q.x) hi = md; else lo = md + 1;
    }
    s0 = lo > 0 ? lo - 1 : 0;
  }
  gs0[g] = s0;
  gm2[g] = q.z;
}

// One warp per work item: the 32 queries at positions 32 g .. 32 g + 31 of
// the final query order (one query slab, close in p1 and in p2) and one
// database slab of their window. Item u = k * G + g (G groups) takes the
// k-th slab of the group's window in the order s0, s0 - 1, s0 + 1, s0 - 2,
// ... (s0: the slab where the group's middle p1 falls; even k to the right,
// odd k to the left), so all groups' nearest slabs are scanned before any
// group's farther ones. Items are taken from a counter in runs of
// kItemRun consecutive groups at the same k (neighbouring groups read the
// same tiles, so they share L1). Each lane publishes its best (distance,
// index) with a 64-bit atomic minimum and prunes with the smallest
// published distance: rows, tiles and slabs are left out only when their
// bound exceeds a distance some row really has, so the minimum over the
// published pairs is the exact result. A slab that no lane's p1 bound
// reaches ends its side for the group from that slab on (the bound is
// monotone over slabs): done keeps the smallest such offset per side, and
// items of that side at or beyond it return at once (nearer ones still run,
// as another warp may have ended the side while they wait). In a
// slab: its tiles outward from the one where the group's middle p2 falls,
// alternately right and left, a side ending when no lane's bound from the
// slab's p1 gap and the side's monotone p2 gap reaches the next tile.
// kCount: also add the number of terms (a_k - b_k)^2 evaluated for the
// valid queries to *terms (a separate instantiation, used when profiling).
template <bool kCount>
__global__ void __launch_bounds__(kMT, 8) k_match_win(const float *__restrict__ FPs, const int *__restrict__ qorig,
                                                   int nP, const float *__restrict__ FQs,
                                                   const int *__restrict__ dorig, int nQ,
                                                   const float4 *__restrict__ pe, const float *__restrict__ slo1,
                                                   const float *__restrict__ shi1, const float *__restrict__ smin1,
                                                   const float *__restrict__ hmax1, const float *__restrict__ smin2,
                                                   const float *__restrict__ hmax2, const int *__restrict__ gs0,
                                                   const float *__restrict__ gm2, int *done,
                                                   const ProjParams *pp, unsigned long long *packed, unsigned long long *work,
                                                   unsigned long long *__restrict__ terms) {
  const int lane = threadIdx.x & 31;
  const int nt = (int)lsr_div_up(nQ, kTile), ns = (int)lsr_div_up(nQ, kSlab);
  const int G = (int)lsr_div_up(nP, 32);
  const long long nitems = 2ll * ns * G;
  const float4 *F4 = reinterpret_cast<const float4 *>(FQs);
  const float fac = pp->fac;
  unsigned long long nterm = 0;
  for (;;) {
    long long u0 = 0;
    if (lane == 0) u0 = (long long)atomicAdd(work, (unsigned long long)kItemRun);
    u0 = __shfl_sync(0xffffffffu, u0, 0);
    if (u0 >= nitems) break;
    for (long long u = u0; u < u0 + kItemRun && u < nitems; ++u) {
      const int kk = (int)(u / G), g = (int)(u % G);
      const bool to_right = (kk & 1) == 0;
      const int s = to_right ? gs0[g] + (kk >> 1) : gs0[g] - 1 - (kk >> 1);
      if (s < 0 || s >= ns) continue;
      // (one lane reads what other warps record, so the warp takes one decision)
      int end_off = 0;
      if (lane == 0) end_off = *reinterpret_cast<volatile int *>(done + 2 * g + (to_right ? 0 : 1));
      if ((kk >> 1) >= __shfl_sync(0xffffffffu, end_off, 0)) continue;
      const int k = g * 32 + lane;
      const bool valid = k < nP;
      const int kq = valid ? k : 0;
      float ql1, qh1, ql2, qh2;
      {
        const float4 q = pe[nQ + qorig[kq]];
        ql1 = __fsub_rd(q.x, q.y), qh1 = __fadd_ru(q.x, q.y), ql2 = __fsub_rd(q.z, q.w), qh2 = __fadd_ru(q.z, q.w);
      }
      // invalid lanes: bound below any distance, so they never hold the warp
      // back; valid ones start from the smallest distance published so far
      float best = -1.f;
      int bj = -1;
      if (valid) {
        const unsigned long long pv = __ldcg(packed + qorig[kq]);
        best = pv == ~0ull ? FLT_MAX : __uint_as_float((unsigned)(pv >> 32));
        bj = pv == ~0ull ? -1 : -2;
      }
      const float gs = to_right ? fmaxf(__fsub_rd(smin1[s], qh1), 0.f) : fmaxf(__fsub_rd(ql1, hmax1[s]), 0.f);
      if (!__any_sync(0xffffffffu, valid && !(gap_bound(gs, 0.f, fac) > best))) {
        if (lane == 0) atomicMin(done + 2 * g + (to_right ? 0 : 1), kk >> 1);
        continue;
      }
      float a[kD];
      {
        const float4 *row = reinterpret_cast<const float4 *>(FPs + (size_t)kq * kDS);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = __ldg(row + c);
          a[4 * c] = v.x, a[4 * c + 1] = v.y, a[4 * c + 2] = v.z, a[4 * c + 3] = v.w;
        }
        a[32] = __ldg(reinterpret_cast<const float *>(row + 8));
      }
      bool taken = false;
      unsigned uterm = 0;  // terms of this item (at most 33 per database row)
      const float g1 = interval_gap(slo1[s], shi1[s], ql1, qh1);
      const int ta = s * kTilesPerSlab, tb = min(nt, ta + kTilesPerSlab);
      // start tile: the last of the slab whose suffix minimum of lo2 does not exceed m2
      const float m2 = gm2[g];
      int t0 = ta;
      if (isfinite(m2)) {
        int lo = ta, hi = tb;
        while (lo < hi) {
          const int md = (lo + hi) >> 1;
          if (smin2[md] > m2) hi = md; else lo = md + 1;
        }
        t0 = lo > ta ? lo - 1 : ta;
      }
      int r = t0, l = t0 - 1;
      bool rgo = true, lgo = l >= ta, turn = true;
      while (rgo || lgo) {
        const bool right = rgo && (turn || !lgo);
        turn = !right;
        const int t = right ? r : l;
        const float g2 = right ? fmaxf(__fsub_rd(smin2[t], qh2), 0.f) : fmaxf(__fsub_rd(ql2, hmax2[t]), 0.f);
        if (!__any_sync(0xffffffffu, valid && !(gap_bound(g1, g2, fac) > best))) {
          (right ? rgo : lgo) = false;
          continue;
        }
        if (right) rgo = ++r < tb;
        else lgo = --l >= ta;
        const int base = t * kTile;
        scan_rows<kCount>(F4 + (size_t)t * (9 * kTile), dorig + base, nQ - base < kTile ? nQ - base : kTile, a,
                          best, bj, taken, uterm);
      }
      if (valid && taken) {
        const int qo = qorig[kq];
        if (LSR_IN_BOUNDS(qo, nP, kSiteMatchQuery)) atomicMin(packed + qo, pack_pair(best, bj));
      }
      if (kCount && valid) nterm += uterm;
    }
  }
  if (kCount) {
    unsigned long long mine = nterm;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
    if (lane == 0) atomicAdd(terms, mine);
  }
}

// nn / d1 from the published minimum of every query (none: -1 / FLT_MAX).
__global__ void k_win_finish(const unsigned long long *__restrict__ packed, int nP, int *__restrict__ nn,
                             float *__restrict__ d1) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nP) return;
  const unsigned long long v = packed[q];
  const bool none = v == ~0ull;
  nn[q] = none ? -1 : (int)(unsigned)(v & 0xFFFFFFFFu);
  if (d1) d1[q] = none ? FLT_MAX : __uint_as_float((unsigned)(v >> 32));
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
  float4 *pe;                         // (p1, e1, p2, e2) of the nQ database rows, then the nP queries
  int *slot1, *counts1, *start1, *order1;
  int *slot2, *counts2, *start2, *order, *scan;
  float *FQs;                         // database rows in the final order, chunk-major per tile
  int *dorig;                         // their original indices
  float4 *tbox;                       // per tile
  float *smin2, *hmax2;               // per tile, within its slab
  float *slo1, *shi1, *smin1, *hmax1; // per slab
  unsigned long long *packed;         // per query: published (distance bits << 32 | index) minimum
  unsigned long long *work;           // work-item counter
  float *FPs;                         // queries in the final order (desc_order rows)
  int *qorig;                         // their original indices
  int *gs0;                           // per query group: start slab
  float *gm2;                         // per query group: middle p2
  int *done;                          // per query group and side: offset from which no slab is needed
  int capD, ncap2;
  size_t bytes;
};

Fp32Layout fp32_layout(char *base, int nP, int nQ) {
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t n = (size_t)nP + (size_t)nQ, nt = (size_t)lsr_div_up(nQ, kTile), ns = (size_t)lsr_div_up(nQ, kSlab);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *p = base ? base + off : nullptr;
    off += al(bytes > 0 ? bytes : 1);
    return p;
  };
  Fp32Layout L;
  L.capD = (int)(ns * kSlab);
  L.ncap2 = L.capD + (int)(lsr_div_up(nP, kSlab) * kSlab);
  const size_t n2 = (size_t)L.ncap2;
  L.pp = reinterpret_cast<ProjParams *>(take(sizeof(ProjParams)));
  L.pe = reinterpret_cast<float4 *>(take(sizeof(float4) * n));
  L.slot1 = reinterpret_cast<int *>(take(sizeof(int) * n));
  L.counts1 = reinterpret_cast<int *>(take(sizeof(int) * (n + 1)));
  L.start1 = reinterpret_cast<int *>(take(sizeof(int) * (n + 1)));
  L.order1 = reinterpret_cast<int *>(take(sizeof(int) * n));
  L.slot2 = reinterpret_cast<int *>(take(sizeof(int) * n));
  L.counts2 = reinterpret_cast<int *>(take(sizeof(int) * (n2 + 1)));
  L.start2 = reinterpret_cast<int *>(take(sizeof(int) * (n2 + 1)));
  L.order = reinterpret_cast<int *>(take(sizeof(int) * n));
  L.scan = reinterpret_cast<int *>(take(sizeof(int) * (size_t)scan_scratch_ints((int64_t)(n2 > n ? n2 : n))));
  // whole tiles: chunk c of the last tile's rows lies at c * kTile within it
  L.FQs = reinterpret_cast<float *>(take(sizeof(float) * kDS * kTile * nt));
  L.dorig = reinterpret_cast<int *>(take(sizeof(int) * (size_t)nQ));
  L.tbox = reinterpret_cast<float4 *>(take(sizeof(float4) * nt));
  L.smin2 = reinterpret_cast<float *>(take(sizeof(float) * nt));
  L.hmax2 = reinterpret_cast<float *>(take(sizeof(float) * nt));
  L.slo1 = reinterpret_cast<float *>(take(sizeof(float) * ns));
  L.shi1 = reinterpret_cast<float *>(take(sizeof(float) * ns));
  L.smin1 = reinterpret_cast<float *>(take(sizeof(float) * ns));
  L.hmax1 = reinterpret_cast<float *>(take(sizeof(float) * ns));
  L.packed = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long) * (size_t)nP));
  L.work = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long)));
  const size_t G = (size_t)lsr_div_up(nP, 32);
  L.FPs = reinterpret_cast<float *>(take(sizeof(float) * kDS * (size_t)nP));
  L.qorig = reinterpret_cast<int *>(take(sizeof(int) * (size_t)nP));
  L.gs0 = reinterpret_cast<int *>(take(sizeof(int) * G));
  L.gm2 = reinterpret_cast<float *>(take(sizeof(float) * G));
  L.done = reinterpret_cast<int *>(take(sizeof(int) * 2 * G));
  L.bytes = off;
  return L;
}

int *pp_field(ProjParams *pp, size_t offset) { return reinterpret_cast<int *>(reinterpret_cast<char *>(pp) + offset); }

}  // namespace

size_t fp32_workspace_bytes(int nP, int nQ) { return fp32_layout(nullptr, nP, nQ).bytes; }

cudaError_t launch_match_fp32(const float *FP, int nP, const float *FQ, int nQ, void *ws, int *nn, float *d1,
                              cudaStream_t s, unsigned long long *terms) {
  if (nP < 1) return cudaSuccess;
  Fp32Layout L = fp32_layout(static_cast<char *>(ws), nP, nQ);
  const int n = nP + nQ, nt = (int)lsr_div_up(nQ, kTile), ns = (int)lsr_div_up(nQ, kSlab);
  const int eb = (int)lsr_div_up(n, 256);
  LSR_CUDA_TRY(cudaMemsetAsync(L.counts1, 0, sizeof(int) * ((size_t)n + 1), s));
  LSR_CUDA_TRY(cudaMemsetAsync(L.counts2, 0, sizeof(int) * ((size_t)L.ncap2 + 1), s));
  constexpr int kPcSmem = kPcSamples * kD * (int)sizeof(float);
  LSR_CUDA_TRY(cudaFuncSetAttribute(k_pc, cudaFuncAttributeMaxDynamicSharedMemorySize, kPcSmem));
  LSR_LAUNCH(k_pc<<<1, kPcThreads, kPcSmem, s>>>(FQ, nQ, nP, L.ncap2, L.pp));
  LSR_LAUNCH(k_proj<<<eb, 256, 0, s>>>(FP, nP, FQ, nQ, L.pp, L.pe));
  // by p1, then by p2 inside slabs of kSlab consecutive positions
  LSR_LAUNCH(k_bucket1<<<eb, 256, 0, s>>>(L.pe, nQ, nP, L.pp, L.slot1, L.counts1));
  LSR_CUDA_TRY(scan_exclusive(L.counts1, L.start1, pp_field(L.pp, offsetof(ProjParams, ntot)), n, L.scan, s));
  LSR_LAUNCH(k_bucket_scatter<<<eb, 256, 0, s>>>(n, L.slot1, L.start1, nullptr, L.order1));
  LSR_LAUNCH(k_bucket2<<<eb, 256, 0, s>>>(L.pe, L.order1, nQ, nP, L.capD, L.pp, L.slot2, L.counts2));
  LSR_CUDA_TRY(scan_exclusive(L.counts2, L.start2, pp_field(L.pp, offsetof(ProjParams, ncap2)), L.ncap2, L.scan, s));
  LSR_LAUNCH(k_bucket_scatter<<<eb, 256, 0, s>>>(n, L.slot2, L.start2, L.order1, L.order));
  if (nt > 0) {
    LSR_LAUNCH(k_gather_db<<<nt, kTile, 0, s>>>(FQ, nQ, L.order, L.pe, L.FQs, L.dorig, L.tbox));
    LSR_LAUNCH(k_slab_bounds<<<(int)lsr_div_up(ns, 128), 128, 0, s>>>(L.tbox, nt, ns, L.slo1, L.shi1, L.smin2,
                                                                       L.hmax2));
    LSR_LAUNCH(k_bound_scan<<<1, kScanThreadsT, 0, s>>>(L.slo1, L.shi1, ns, L.smin1, L.hmax1));
  }
  LSR_CUDA_TRY(cudaMemsetAsync(L.packed, 0xFF, sizeof(unsigned long long) * (size_t)nP, s));
  LSR_CUDA_TRY(cudaMemsetAsync(L.work, 0, sizeof(unsigned long long), s));
  const int G = (int)lsr_div_up(nP, 32);
  // 0x7F7F7F7F: no side has ended yet
  LSR_CUDA_TRY(cudaMemsetAsync(L.done, 0x7F, sizeof(int) * 2 * (size_t)G, s));
  LSR_LAUNCH(k_gather_q<<<(int)lsr_div_up(nP, 256), 256, 0, s>>>(FP, nP, nQ, L.order, L.FPs, L.qorig));
  if (nt > 0) {
    LSR_LAUNCH(k_group_start<<<(int)lsr_div_up(G, 256), 256, 0, s>>>(L.pe, L.qorig, nP, nQ, L.smin1, L.gs0, L.gm2));
    // persistent warps: as many blocks as fit on the GPU at once, or fewer
    int per_sm = 0;
    LSR_CUDA_TRY(terms ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match_win<true>, kMT, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match_win<false>, kMT, 0));
    const long long items = 2ll * ns * G;
    long long blocks = lsr_div_up(lsr_div_up(items, kItemRun), kMT / 32);
    const long long resident = (long long)(per_sm > 0 ? per_sm : 1) * device_sm_count();
    if (blocks > resident) blocks = resident;
    if (terms)
      LSR_LAUNCH(k_match_win<true><<<(int)blocks, kMT, 0, s>>>(L.FPs, L.qorig, nP, L.FQs, L.dorig, nQ, L.pe, L.slo1,
                                                               L.shi1, L.smin1, L.hmax1, L.smin2, L.hmax2, L.gs0,
                                                               L.gm2, L.done, L.pp, L.packed, L.work, terms));
    else
      LSR_LAUNCH(k_match_win<false><<<(int)blocks, kMT, 0, s>>>(L.FPs, L.qorig, nP, L.FQs, L.dorig, nQ, L.pe, L.slo1,
                                                                L.shi1, L.smin1, L.hmax1, L.smin2, L.hmax2, L.gs0,
                                                                L.gm2, L.done, L.pp, L.packed, L.work, nullptr));
  }
  LSR_LAUNCH(k_win_finish<<<(int)lsr_div_up(nP, 256), 256, 0, s>>>(L.packed, nP, nn, d1));
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
