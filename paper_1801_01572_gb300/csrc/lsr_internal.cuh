// lsr_internal.cuh -- internal declarations shared by the CUDA translation
// units of the registration library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lsr {

constexpr int kD = 33;       // FPFH length: 3 features x 11 bins
constexpr int kNB = 11;      // bins per feature
constexpr int kDS = 36;      // stored row stride of SPFH / FPFH (16-byte aligned rows)
constexpr int kWarp = 32;
constexpr int kSms = 152;    // GB300 streaming multiprocessors (2 dies x 76): grid caps are multiples of it

// Order in which the FP32 descriptor distance sum_k (a_k - b_k)^2 is
// accumulated: the central bin of each of the three 11-bin sub-histograms,
// then the bins one step out on either side, two steps out, and so on. The
// angular features of smooth surfaces pile up around the central bins, so
// this order front-loads the mass of the distance and lets a partial sum pass
// the running minimum after few terms. desc_order(k) is the bin added k-th;
// desc_rank is its inverse. Every exact FP32 distance of the matchers uses it.
__host__ __device__ constexpr int desc_order(int k) {
  return k < 3 ? kNB * k + kNB / 2
               : kNB * (((k - 3) % 6) / 2) + kNB / 2 + (((k - 3) % 2) ? 1 : -1) * ((k - 3) / 6 + 1);
}
__host__ __device__ constexpr int desc_rank(int col) {
  return (col % kNB == kNB / 2) ? col / kNB
                                : 3 + 6 * ((col % kNB > kNB / 2 ? col % kNB - kNB / 2 : kNB / 2 - col % kNB) - 1) +
                                      2 * (col / kNB) + (col % kNB > kNB / 2 ? 1 : 0);
}

// Uniform 3D grid of eq. (1): cell index = floor((x - origin) / cell), stored
// densely over the cloud's bounding box. When the box holds more cells than
// the allocated capacity, the y and z (and if needed x) cell coordinates wrap
// modulo the stored extents; wrapped cells share storage, which only adds
// candidates that the exact distance test then rejects. The cell edge is the
// search radius times (1 + delta), delta >= 1e-4 growing with the box extent
// to cover the FP32 rounding of the cell coordinates, so every point within
// the radius of a query lies in the 3 x 3 x 3 block of cells around it.
struct GridParams {
  // Optional bitmap over storage cells: bit set if the 3 x 3 x 3 block around
  // the cell holds a point. A query whose own cell has a clear bit has no
  // neighbour within the radius and skips the range lookups (most consensus
  // queries of wrong hypotheses land in empty space).
  const unsigned *nbmask;
  float ox, oy, oz;  // origin (bounding-box minimum)
  float cell, inv_cell;
  int nx, ny, nz;    // extent of the bounding box in cells
  int wx, wy, wz;    // stored extents (<= n*, equal unless wrapped)
  int ncells;        // wx * wy * wz
  int npts;
  int pad_;
};

// Device view of one cloud after packing and grid building. "Internal order"
// is the order of the feature-radius grid (points sorted by cell, then by
// caller index), which keeps neighbourhoods contiguous in memory.
struct CloudDev {
  int n;
  const float4 *X;        // n, internal order; w = caller index (int bits)
  const int *inv;         // n, caller index -> internal index
  const GridParams *gf;   // feature-radius grid over X (its sorted array is X)
  const int *start_f;     // gf->ncells + 1
  const GridParams *gn;   // normal-radius grid
  const int *start_n;
  const float4 *Xn;       // n, sorted by normal grid; w = internal index
  const GridParams *ge;   // eps grid (consensus / refinement / objective)
  const int *start_e;
  const float4 *Xe;       // n, sorted by eps grid; w = internal index
  const float4 *N;        // n normals (internal order); w = curvature, -1 if invalid
  const float *F;         // n x kDS FPFH (internal order)
};

// ----------------------------------------------------------------- helpers
__host__ __device__ inline int64_t lsr_div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Checked build (-DLSR_CHECKED): the index checks below record the first
// violation of a translation unit (site, index, bound) in that unit's device
// words instead of trapping, and the guarded access is skipped; the host reads
// the words after each synchronising call (check_report) and returns
// LSR_E_CHECK. In the normal build every check is the constant true.
enum CheckSite : int {
  kSiteGridRow = 1,   // grid walk: cell-start index of a row of cells
  kSiteGridSlot,      // grid walk (wrapped storage): cell-start index of a cell
  kSiteGridPoint,     // grid walk: sorted point index
  kSiteHypSample,     // hypotheses: sampled point index
  kSiteHypMatch,      // hypotheses: descriptor NN of a sampled point
  kSiteMatchRow,      // matchers: database row of a candidate
  kSiteMatchQuery,    // matchers: query row written
  kSiteProbe,         // test probe (lsr_debug_inject LSR_INJECT_CHECK): never an access
};
struct CheckReport {
  unsigned long long site;
  long long index, bound;
};
#ifdef LSR_CHECKED
static __device__ unsigned long long g_check_site;
static __device__ long long g_check_index, g_check_bound;
__device__ __forceinline__ bool check_in_bounds(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicCAS(&g_check_site, 0ull, (unsigned long long)site) == 0ull) {
    g_check_index = i;
    g_check_bound = n;
  }
  return false;
}
#define LSR_IN_BOUNDS(i, n, site) ::lsr::check_in_bounds((long long)(i), (long long)(n), (site))
// Host reader of this translation unit's words (clears them).
#define LSR_CHECK_READER(unit)                                                                \
  cudaError_t check_read_##unit(CheckReport *r) {                                             \
    CheckReport z{0, 0, 0};                                                                   \
    cudaError_t e = cudaMemcpyFromSymbol(&r->site, g_check_site, sizeof(r->site));            \
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&r->index, g_check_index, sizeof(r->index)); \
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&r->bound, g_check_bound, sizeof(r->bound)); \
    if (e == cudaSuccess && r->site) e = cudaMemcpyToSymbol(g_check_site, &z.site, sizeof(z.site)); \
    return e;                                                                                 \
  }
#else
#define LSR_IN_BOUNDS(i, n, site) true
#define LSR_CHECK_READER(unit)                     \
  cudaError_t check_read_##unit(CheckReport *r) { \
    r->site = 0;                                   \
    r->index = r->bound = 0;                       \
    return cudaSuccess;                            \
  }
#endif
// Readers of the units that hold checks.
cudaError_t check_read_features(CheckReport *r);
cudaError_t check_read_match(CheckReport *r);
cudaError_t check_read_match_tc(CheckReport *r);
cudaError_t check_read_ransac(CheckReport *r);
cudaError_t check_read_classify(CheckReport *r);
cudaError_t check_read_refine(CheckReport *r);
cudaError_t check_read_nn(CheckReport *r);
cudaError_t check_read_implicit(CheckReport *r);
cudaError_t check_probe_arm(cudaStream_t s);

// Kernel launches of this library, counted process-wide (lsr_launch_count).
extern unsigned long long g_launches;
inline void count_launch() { __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED); }

// Per-kernel CUDA-event timing (lsr_set_kernel_timing): while a timer is
// installed for the calling thread, every launch whose kernel name starts with
// the timer's filter is bracketed by two events recorded on the timer's stream
// (the stream every launch of that call is ordered on).
struct KernelTimer;
extern thread_local KernelTimer *g_ktimer;
void ktimer_mark(const char *launch_expr, bool after);
#define LSR_LAUNCH(...)                                                                  \
  (::lsr::count_launch(), ::lsr::g_ktimer ? ::lsr::ktimer_mark(#__VA_ARGS__, false) : void(), \
   __VA_ARGS__, ::lsr::g_ktimer ? ::lsr::ktimer_mark(#__VA_ARGS__, true) : void())

// Launch with programmatic stream serialisation: the kernel may be scheduled
// before the previous kernel in the stream has finished (that kernel allows
// it with griddepcontrol.launch_dependents) and must execute
// griddepcontrol.wait before it touches anything the previous kernel writes.
template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

#define LSR_CUDA_TRY(call)                         \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return e_;              \
  } while (0)

// Visit the sorted-point ranges that can hold points within one cell of the
// query (the 27 cells around it): f(b, e) is called for each range [b, e) of
// the grid's sorted array. Without wrapping, the three x-adjacent cells of a
// row are one contiguous range (9 calls). With wrapping, each distinct storage
// cell is visited once. Queries more than one cell outside the box visit
// nothing.
template <class F>
__device__ __forceinline__ void grid_ranges(const GridParams &g, const int *__restrict__ start, float x, float y,
                                            float z, F &&f) {
  float fx = (x - g.ox) * g.inv_cell, fy = (y - g.oy) * g.inv_cell, fz = (z - g.oz) * g.inv_cell;
  if (!(fx >= -1.f && fx < (float)g.nx + 1.f && fy >= -1.f && fy < (float)g.ny + 1.f && fz >= -1.f &&
        fz < (float)g.nz + 1.f))
    return;
  int cx = __float2int_rd(fx), cy = __float2int_rd(fy), cz = __float2int_rd(fz);
  int x0 = cx - 1 < 0 ? 0 : cx - 1, x1 = cx + 1 > g.nx - 1 ? g.nx - 1 : cx + 1;
  if (x0 > x1) return;
  bool wrapped = (g.wx != g.nx) | (g.wy != g.ny) | (g.wz != g.nz);
  if (g.nbmask && cx >= 0 && cx < g.nx && cy >= 0 && cy < g.ny && cz >= 0 && cz < g.nz) {
    int slot = wrapped ? ((cz % g.wz) * g.wy + (cy % g.wy)) * g.wx + (cx % g.wx) : (cz * g.wy + cy) * g.wx + cx;
    if (!((__ldg(g.nbmask + (slot >> 5)) >> (slot & 31)) & 1u)) return;
  }
  if (!wrapped) {
    for (int dz = -1; dz <= 1; ++dz) {
      int iz = cz + dz;
      if (iz < 0 || iz >= g.nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        int iy = cy + dy;
        if (iy < 0 || iy >= g.ny) continue;
        int row = (iz * g.wy + iy) * g.wx;
        if (!LSR_IN_BOUNDS(row + x1 + 1, g.ncells + 1, kSiteGridRow) || !LSR_IN_BOUNDS(row + x0, g.ncells + 1, kSiteGridRow))
          continue;
#ifdef LSR_CHECKED
        {
          const int b = start[row + x0], e = start[row + x1 + 1];
          if (e > b && (!LSR_IN_BOUNDS(e - 1, g.npts, kSiteGridPoint) || !LSR_IN_BOUNDS(b, g.npts, kSiteGridPoint)))
            continue;
        }
#endif
        f(start[row + x0], start[row + x1 + 1]);
      }
    }
    return;
  }
  int seen[27];
  int ns = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int iz = cz + dz;
    if (iz < 0 || iz >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int iy = cy + dy;
      if (iy < 0 || iy >= g.ny) continue;
      for (int ix = x0; ix <= x1; ++ix) {
        int slot = ((iz % g.wz) * g.wy + (iy % g.wy)) * g.wx + (ix % g.wx);
        bool dup = false;
        for (int k = 0; k < ns; ++k) dup |= (seen[k] == slot);
        if (dup) continue;
        seen[ns++] = slot;
        if (!LSR_IN_BOUNDS(slot + 1, g.ncells + 1, kSiteGridSlot) || !LSR_IN_BOUNDS(slot, g.ncells + 1, kSiteGridSlot))
          continue;
#ifdef LSR_CHECKED
        {
          const int b = start[slot], e = start[slot + 1];
          if (e > b && (!LSR_IN_BOUNDS(e - 1, g.npts, kSiteGridPoint) || !LSR_IN_BOUNDS(b, g.npts, kSiteGridPoint)))
            continue;
        }
#endif
        f(start[slot], start[slot + 1]);
      }
    }
  }
}

// Exact nearest neighbour within sqrt(eps2) of (x, y, z) by a group of G
// lanes (G divides 32, the group's lanes are consecutive and all query the
// same point): the lanes walk the concatenated candidate ranges with stride
// G, so work spreads evenly across range boundaries, then combine (distance,
// index) minima with shuffles. Ties go to the smaller carried index (w of the
// grid's sorted points). Every lane returns the group's result; bt = -1 if no
// point is within the radius.
//
// The query's own row of cells is searched first; each of the other eight
// rows, and the x-neighbour cells of every row, is visited only if its
// distance from the query (less a margin of 2e-4 cells, above the FP32
// rounding of cell coordinates) can still reach the group's best so far. A
// skipped cell holds no point at or below that best, so the result is the
// one of the full walk. (Grids with wrapped storage walk all cells.)
//
// seed (optional, >= 0): an index into Xe known to be a candidate (the
// previous refinement step's neighbour of the same point). Its distance,
// computed exactly as the walk computes distances, starts the search when it
// is below eps2, so cells beyond it are skipped; the result is the walk's
// result without a seed (the nearest point wins either way, ties to the
// smaller carried index).
__device__ __forceinline__ float nn_d2(float4 q, float x, float y, float z) {
  float dx = q.x - x, dy = q.y - y, dz = q.z - z;
  return dx * dx + dy * dy + dz * dz;
}

template <int G>
__device__ __forceinline__ void group_nn(const GridParams &g, const int *__restrict__ start,
                                         const float4 *__restrict__ Xe, float x, float y, float z, float eps2,
                                         float &best, int &bt, int &bidx, int seed = -1) {
  int sub = threadIdx.x & (G - 1);
  best = eps2;
  bt = -1;
  bidx = 0x7fffffff;
  if (seed >= 0 && LSR_IN_BOUNDS(seed, g.npts, kSiteGridPoint)) {
    const float4 q = Xe[seed];
    const float d2 = nn_d2(q, x, y, z);
    if (d2 < eps2) best = d2, bt = seed, bidx = __float_as_int(q.w);
  }
  int next = sub, base = 0;
  auto scan = [&](int b, int e) {
    int len = e - b;
    // four independent loads in flight per lane, then the remainder
#ifdef LSR_CHECKED
    if (len > 0 && (!LSR_IN_BOUNDS(e - 1, g.npts, kSiteGridPoint) || !LSR_IN_BOUNDS(b, g.npts, kSiteGridPoint))) {
      for (; next < base + len; next += G) {
      }
      base += len;
      return;
    }
#endif
    for (; next + 3 * G < base + len; next += 4 * G) {
      int t = b + next - base;
      float4 q[4] = {Xe[t], Xe[t + G], Xe[t + 2 * G], Xe[t + 3 * G]};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float d2 = nn_d2(q[k], x, y, z);
        int qi = __float_as_int(q[k].w);
        if (d2 < best || (d2 == best && qi < bidx)) best = d2, bt = t + k * G, bidx = qi;
      }
    }
    for (; next < base + len; next += G) {
      int t = b + next - base;
      float4 q = Xe[t];
      float d2 = nn_d2(q, x, y, z);
      int qi = __float_as_int(q.w);
      if (d2 < best || (d2 == best && qi < bidx)) best = d2, bt = t, bidx = qi;
    }
    base += len;
  };
  const bool wrapped = (g.wx != g.nx) | (g.wy != g.ny) | (g.wz != g.nz);
  if (wrapped) {
    grid_ranges(g, start, x, y, z, scan);
  } else {
    const float fx = (x - g.ox) * g.inv_cell, fy = (y - g.oy) * g.inv_cell, fz = (z - g.oz) * g.inv_cell;
    bool go = fx >= -1.f && fx < (float)g.nx + 1.f && fy >= -1.f && fy < (float)g.ny + 1.f && fz >= -1.f &&
              fz < (float)g.nz + 1.f;
    const int cx = go ? __float2int_rd(fx) : 0, cy = go ? __float2int_rd(fy) : 0, cz = go ? __float2int_rd(fz) : 0;
    const int x0 = cx - 1 < 0 ? 0 : cx - 1, x1 = cx + 1 > g.nx - 1 ? g.nx - 1 : cx + 1;
    go = go && x0 <= x1;
    if (go && g.nbmask && cx >= 0 && cx < g.nx && cy >= 0 && cy < g.ny && cz >= 0 && cz < g.nz) {
      const int slot = (cz * g.wy + cy) * g.wx + cx;
      go = (__ldg(g.nbmask + (slot >> 5)) >> (slot & 31)) & 1u;
    }
    if (go) {
      const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
      const float mg = 2e-4f * g.cell;
      auto gsq = [&](float d) {
        const float t = fmaxf(d - mg, 0.f);
        return t * t;
      };
      // squared distances to the lower / upper faces of the query's cell
      const float gxl = gsq((fx - (float)cx) * g.cell), gxh = gsq(((float)cx + 1.f - fx) * g.cell);
      const float gyl = gsq((fy - (float)cy) * g.cell), gyh = gsq(((float)cy + 1.f - fy) * g.cell);
      const float gzl = gsq((fz - (float)cz) * g.cell), gzh = gsq(((float)cz + 1.f - fz) * g.cell);
      constexpr float kShrink = 1.f - 1e-6f;  // the FP32 rounding of d^2 itself
      float gb = best;  // eps2, or the seed's distance (the same on every lane of the group)
#pragma unroll 1
      for (int k = 0; k < 9; ++k) {
        // rows: own, then the four edge neighbours, then the four corners
        const int dy = k == 1 ? -1 : k == 2 ? 1 : (k >= 5 ? ((k & 1) ? -1 : 1) : 0);
        const int dz = k == 3 ? -1 : k == 4 ? 1 : (k >= 5 ? (k < 7 ? -1 : 1) : 0);
        const int iy = cy + dy, iz = cz + dz;
        if (iy < 0 || iy >= g.ny || iz < 0 || iz >= g.nz) continue;
        const float r2 = (dy < 0 ? gyl : dy > 0 ? gyh : 0.f) + (dz < 0 ? gzl : dz > 0 ? gzh : 0.f);
        if (r2 * kShrink > gb) continue;
        int a = x0, e = x1;
        if (a < cx && (r2 + gxl) * kShrink > gb) a = cx;
        if (e > cx && (r2 + gxh) * kShrink > gb) e = cx;
        if (a > e) continue;
        const int row = (iz * g.wy + iy) * g.wx;
        if (!LSR_IN_BOUNDS(row + e + 1, g.ncells + 1, kSiteGridRow) || !LSR_IN_BOUNDS(row + a, g.ncells + 1, kSiteGridRow))
          continue;
        scan(start[row + a], start[row + e + 1]);
        float m = best;
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) m = fminf(m, __shfl_xor_sync(gmask, m, off));
        gb = m;
      }
    }
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    float ob = __shfl_xor_sync(0xffffffffu, best, off);
    int ot = __shfl_xor_sync(0xffffffffu, bt, off);
    int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
    if (ob < best || (ob == best && oi < bidx)) best = ob, bt = ot, bidx = oi;
  }
}

// Squared distance with an explicit operation order: every kernel that
// decides d^2 < eps^2 for the same pair of points decides it the same way.
__device__ __forceinline__ float dist2(float4 q, float x, float y, float z) {
  float dx = q.x - x, dy = q.y - y, dz = q.z - z;
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// x = R p + t for a row-major [R | t] (12 floats), in one fixed order.
struct Rigid12 {
  float r0, r1, r2, t0, r3, r4, r5, t1, r6, r7, r8, t2;
  __device__ __forceinline__ void load(const float *T) {
    r0 = T[0], r1 = T[1], r2 = T[2], t0 = T[3], r3 = T[4], r4 = T[5], r5 = T[6], t1 = T[7];
    r6 = T[8], r7 = T[9], r8 = T[10], t2 = T[11];
  }
  __device__ __forceinline__ void apply(float4 p, float &x, float &y, float &z) const {
    x = fmaf(r0, p.x, fmaf(r1, p.y, fmaf(r2, p.z, t0)));
    y = fmaf(r3, p.x, fmaf(r4, p.y, fmaf(r5, p.z, t1)));
    z = fmaf(r6, p.x, fmaf(r7, p.y, fmaf(r8, p.z, t2)));
  }
};

// Sums nq per-block partials (partials[b * stride + k], b < nb) with the whole
// block: thread t adds quantity t % nq over the blocks t / nq, t / nq + S, ...
// (S = blockDim.x / nq segments, eight loads in flight), then threads k < nq add
// the S segment sums in order. The order is fixed, so the sums are
// deterministic. seg: shared scratch of at least blockDim.x doubles; out[k] for
// k < nq is valid after the call (which ends with a barrier).
__device__ __forceinline__ void block_sum_partials(const double *__restrict__ partials, int nb, int nq, int stride,
                                                   double *seg, double *out) {
  const int S = (int)blockDim.x / nq, k = (int)threadIdx.x % nq, sg = (int)threadIdx.x / nq;
  if (sg < S) {
    double sum = 0.0;
    int b = sg;
    for (; b + 7 * S < nb; b += 8 * S) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(partials + (size_t)(b + u * S) * stride + k);
#pragma unroll
      for (int u = 0; u < 8; ++u) sum += v[u];
    }
    for (; b < nb; b += S) sum += __ldcg(partials + (size_t)b * stride + k);
    seg[sg * nq + k] = sum;
  }
  __syncthreads();
  if ((int)threadIdx.x < nq) {
    double t = 0.0;
    for (int q = 0; q < S; ++q) t += seg[q * nq + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ int warp_sum(int v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// ----------------------------------------------------------------- grid build (lsr_grid.cu)
// Bounding box and centroid of a float32 xyz array (AoS) or a float4 array,
// reduced through kBoxPart doubles per block into box[kBox] = (min xyz, max
// xyz, non-finite flag, finite count, centroid xyz, 0).
constexpr int kBox = 12;
constexpr int kBoxPart = 11;
cudaError_t launch_bbox_xyz(const float *xyz, int n, double *partials, int nblk_cap, float *box, cudaStream_t s);
cudaError_t launch_bbox_f4(const float4 *x, int n, double *partials, int nblk_cap, float *box, cudaStream_t s);
int bbox_blocks(int n);

// Fill a GridParams from a bounding box on the device (no neighbourhood mask).
cudaError_t launch_grid_params(const float *box, float radius, int npts, int cap_cells, GridParams *g, cudaStream_t s);
// Build the neighbourhood bitmap of a built grid (nbmask_words(cap) words)
// and attach it to g.
int64_t nbmask_words(int cap_cells);
cudaError_t build_nbmask(GridParams *g, const int *start, int cap_cells, unsigned *mask, cudaStream_t s);

// Counting sort of points into the grid: out[k] = point sorted k-th by (cell,
// source index) with w replaced by the carried index (source index if
// carry == nullptr). start gets the exclusive cell offsets (ncells + 1).
// Scratch: slot (n ints), counts (cap + 1 ints), scan scratch (scan_scratch_ints(cap)).
struct GridScratch {
  int *slot;
  int *counts;
  int *tmp;       // n ints
  int *scan;      // scan_scratch_ints(cap + 1)
};
int64_t scan_scratch_ints(int64_t n);
cudaError_t build_grid_xyz(const float *xyz, int n, const GridParams *g, int cap_cells, int *start, float4 *out,
                           int *inv_out, GridScratch sc, cudaStream_t s);
cudaError_t build_grid_f4(const float4 *x, int n, const GridParams *g, int cap_cells, int *start, float4 *out,
                          GridScratch sc, cudaStream_t s);

// Exclusive scan of in[0..*n_dev) into out[0..*n_dev] (out[n] = total).
cudaError_t scan_exclusive(const int *in, int *out, const int *n_dev, int cap, int *scratch, cudaStream_t s);

// ----------------------------------------------------------------- features (lsr_features.cu)
cudaError_t launch_normals(const float4 *X, int n, const GridParams *gn, const int *start_n, const float4 *Xn,
                           float r, float3 vp, float4 *N, int *count, cudaStream_t s);
// scratch: n x 36 ints of device memory (the pair counts; the FPFH output
// buffer may serve, as SPFH comes first).
cudaError_t launch_spfh(const float4 *X, const float4 *N, int n, const GridParams *gf, const int *start_f, float r,
                        float *spfh, int *k, void *scratch, cudaStream_t s);
cudaError_t launch_fpfh(const float4 *X, const float4 *N, const float *spfh, int n, const GridParams *gf,
                        const int *start_f, float r, float *fpfh, cudaStream_t s);

// ----------------------------------------------------------------- matching (lsr_match.cu)
// ws: fp32_workspace_bytes(nP, nQ) of device memory, 256-byte aligned (the
// projection order: a copy of FQ in that order and per-tile bounds);
// terms (optional): add the number of descriptor terms evaluated (profiling)
size_t fp32_workspace_bytes(int nP, int nQ);
// SMs of the current device (148 if the query fails).
int device_sm_count();
cudaError_t launch_match_fp32(const float *FP, int nP, const float *FQ, int nQ, void *ws, int *nn, float *d1,
                              cudaStream_t s, unsigned long long *terms = nullptr);
// Exact FP32 scan of the queries rows[0..*nrows) (count read on the device),
// split over database chunks; packed: scratch of nP 64-bit words.
cudaError_t launch_match_fp32_rows(const float *FP, int nP, const float *FQ, int nQ, const int *rows,
                                   const int *nrows, unsigned long long *packed, int *nn, float *d1,
                                   cudaStream_t s);
// BF16 tensor-core matcher (split: hi/lo BF16 pairs, K = 112; else K = 48)
// with exact FP32 re-rank and certified fallback; ws: tc_workspace_bytes.
// fb_count: queries re-scanned in FP32; err: 1 if a CTA gave up waiting. With
// d2 != null it writes D~^2 = |b~|^2 - 2 a~.b~ + |a~|^2 for every pair (nP
// rows of tc_score_cols(nQ)) instead of matching.
// qt: query tiles of 128 per CTA work unit (1 or 2; 0 = tc_default_tile(nP)).
// f: the limit of the pipeline's waits (0 = 2 s) and the test-only stall
// (the producer issues no copy or MMA, so the epilogue's first wait runs out
// and err is set; see lsr_debug_inject).
struct TcFault {
  unsigned long long wait_ns = 0;
  int stall = 0;
};
size_t tc_workspace_bytes(int nP, int nQ, bool split);
int tc_score_cols(int nQ);
int tc_default_tile(int nP);
cudaError_t launch_match_bf16(const float *FP, int nP, const float *FQ, int nQ, bool split, int qt, char *ws, int *nn,
                              float *d1, int *fb_count, int *err, float *d2, cudaStream_t s, TcFault f = TcFault());

// ----------------------------------------------------------------- RANSAC (lsr_ransac.cu)
// Device-side counters and selection state of one registration.
struct RansacState {
  int n_surv;          // survivors written (capped at surv_cap)
  int n_surv_total;    // survivors found
  int n_normal_ok;
  int best;            // survivor slot of the best hypothesis, -1 none
  int best_h;
  int best_count;
  float best_fit;
  int status;          // 0 aligned, 1 no alignment
  int active;          // refinement still iterating
  int iters_done;
  int final_count;
  int level_iters;     // refinement steps taken at the current level
  unsigned ticket;     // blocks finished in the current refinement step
  int match_fallbacks; // BF16 matcher: queries re-scanned exactly in FP32
  int match_err;       // BF16 matcher: a CTA gave up waiting (result invalid)
  int n_tie;           // hypotheses tied at the top exact count (their sums are computed)
  unsigned long long match_terms;  // FP32 matcher, counting launch: terms evaluated
  double final_sumd2;
  double T[16];        // current pose (refinement), row-major
  double T_hyp[16];
  float pose_f[12];    // FP32 copy of the pose used by consensus-type kernels
  double center[3];    // linearisation centre of the refinement (centroid of Q)
  double last_step;
};

int hyp_blocks(int64_t H);
// ints of the per-block survivor regions (local) for H hypotheses
int64_t hyp_local_ints(int64_t H);
// local: hyp_local_ints(H) ints of scratch; survivors are written there while
// they are counted and placed in order after the scan.
cudaError_t launch_hypotheses(const float4 *XP, const int *invP, const float4 *NP, int nP, const float4 *XQ,
                              const float4 *NQ, int nQ, const int *nn, const uint8_t *vP_ext, const uint8_t *vQ_ext,
                              int64_t H, uint64_t seed, uint64_t pair, float tau, int *block_counts, int *block_offsets,
                              int *scan_scratch, int *surv, int surv_cap, RansacState *st, int *local,
                              cudaStream_t s);
// Pose of each survivor from its 4 pairs + the normal check. pose: cap x 12 floats, ok: cap bytes.
cudaError_t launch_rigid_survivors(const float4 *XP, const int *invP, const float4 *NP, int nP, const float4 *XQ,
                                   const float4 *NQ, const int *nn, const int *surv, const RansacState *st,
                                   uint64_t seed, uint64_t pair, float cos_normal, float *pose, uint8_t *ok,
                                   int *n_normal_ok, cudaStream_t s);
cudaError_t launch_rigid4(const float *ps, const float *qs, int nh, float *pose, cudaStream_t s);
// Consensus: for every pose k < *n_dev (or n_host if n_dev is null) with ok[k] (or ok == null),
// count[k] / sum[k] (fixed point, 2^-40 m^2 units) over all P points.
// list (optional, device): count only the poses list[0 .. *n_dev) (ok is then
// ignored); few poses get P split into smaller chunks so that every block works.
cudaError_t launch_consensus(const float4 *XP, int nP, const GridParams *ge, const int *start_e, const float4 *Xe,
                             const float *pose, const uint8_t *ok, const int *n_dev, int n_host, float eps,
                             int *count, unsigned long long *sum, cudaStream_t s, int lanes = 1,
                             const int *list = nullptr);
cudaError_t launch_select(const int *surv, const int *count, const unsigned long long *sum, const uint8_t *ok,
                          const float *pose, int nP, float min_ratio, RansacState *st, cudaStream_t s);

// ----------------------------------------------------------------- classified consensus (lsr_classify.cu)
// A voxel table over Q's box (voxel h = eps / k): bit IN set only if every
// point of the voxel has a Q point closer than eps, bit NEAR clear only if no
// point of the voxel has one. Consensus counts then need the exact eps-grid
// test only for voxels with NEAR set and IN clear.
// Bits are stored in bricks: a 32-bit word holds 4 x 4 x 2 voxels (x, y, z),
// and eight consecutive words (a 32-byte sector) a 2 x 2 x 2 block of bricks,
// 8 x 8 x 4 voxels, so the nearby points of a warp read few sectors. wx, wy:
// sectors along x and y.
struct ClsParams {
  float ox, oy, oz, h, inv_h, r_in2, r_near, m;
  int nx, ny, nz, wx, wy, R, all_amb;
};
__host__ __device__ inline size_t cls_word(const ClsParams &c, int x, int y, int z) {
  return ((((size_t)(z >> 2) * c.wy + (y >> 3)) * c.wx + (x >> 3)) << 3) | (size_t)((((z >> 1) & 1) << 2) |
                                                                                    (((y >> 2) & 1) << 1) |
                                                                                    ((x >> 2) & 1));
}
__host__ __device__ inline int cls_bit(int x, int y, int z) { return (x & 3) | ((y & 3) << 2) | ((z & 1) << 4); }
constexpr int kClsCapWords = 1 << 23;  // words per bit-set (32 MB)
cudaError_t launch_cls_build(const float *boxQ, float eps, const float4 *XQ, int nQ, ClsParams *cp, unsigned *in_bits,
                             unsigned *near_bits, cudaStream_t s);
// Inlier counts (as launch_consensus, without the distance sums).
cudaError_t launch_consensus_count(const float4 *XP, int nP, const ClsParams *cp, const unsigned *in_bits,
                                   const unsigned *near_bits, const GridParams *ge, const int *start_e,
                                   const float4 *Xe, const float *pose, const uint8_t *ok, const int *n_dev,
                                   int n_host, float eps, int *count, cudaStream_t s);
// Bounds without exact tests over the points XP[v * stride]: in_count =
// points in IN voxels (a lower bound of the inlier count), amb_count = points
// in undecided voxels. With c0 (device; a count some hypothesis reaches) and
// prog (device, one zeroed 64-bit word per hypothesis): a hypothesis whose
// upper bound falls below c0 part-way is left out, its remaining points added
// to amb_count (stride must be 1).
cudaError_t launch_consensus_bounds(const float4 *XP, int nP, int stride, const ClsParams *cp,
                                    const unsigned *in_bits, const unsigned *near_bits, const float *pose,
                                    const uint8_t *ok, const int *n_dev, int *in_count, int *amb_count,
                                    const int *c0, unsigned long long *prog, cudaStream_t s);
// Exact counts (count += ...) that give up on a hypothesis as soon as its
// count can no longer reach c0 (device), from the upper bounds ub_lo + ub_extra
// of a bounds pass; prog: one zeroed 64-bit word per hypothesis. A count given
// up on stays partial and below c0.
cudaError_t launch_consensus_count_bar(const float4 *XP, int nP, const ClsParams *cp, const unsigned *in_bits,
                                       const unsigned *near_bits, const GridParams *ge, const int *start_e,
                                       const float4 *Xe, const float *pose, const uint8_t *ok, const int *n_dev,
                                       float eps, int *count, const int *c0, const int *ub_lo, const int *ub_extra,
                                       unsigned long long *prog, cudaStream_t s);
// out (device) = max over sel of exact.
cudaError_t launch_sel_max(const int *exact, const uint8_t *sel, const int *n_dev, int *out, cudaStream_t s);
// sel: the K ok hypotheses with the largest lo + extra (ties to the smaller id).
cudaError_t launch_top_upper(const int *lo, const int *extra, const uint8_t *ok, const int *n_dev, int K,
                             uint8_t *sel, cudaStream_t s);
// With C = max over sel of exact: rest = ok && !sel && lo + extra >= C, and
// all = sel | rest.
cudaError_t launch_reach_rest(const int *lo, const int *extra, const int *exact, const uint8_t *sel, const uint8_t *ok,
                              const int *n_dev, uint8_t *rest, uint8_t *all, cudaStream_t s);
// With L = max over ok of lo: mask[k] = ok[k] && lo[k] + extra[k] >= L. If L is
// 0: every ok hypothesis when extra is given, none otherwise.
// n_mask, list (optional, device): the number of set entries and their indices.
cudaError_t launch_reach_mask(const int *lo, const int *extra, const uint8_t *ok, const int *n_dev, uint8_t *mask, int *n_mask,
                              int *list,
                              cudaStream_t s);
constexpr double kFixScale = 1099511627776.0;  // 2^40

// ----------------------------------------------------------------- refinement (lsr_refine.cu)
int refine_blocks(int nP);
// Doubles of a refinement partial-sum buffer (block and group sums, then the
// group tickets), and the reset of its tickets (before a refinement's first step).
int64_t refine_partial_doubles();
cudaError_t refine_reset_tickets(double *partials, cudaStream_t s);
// Starting pose (T_in, or the selected hypothesis already in st) and the first
// linearisation centre (the centroid of P, boxP[8..10], moved by that pose).
cudaError_t launch_refine_init(RansacState *st, const float *boxP, const double *T_in, cudaStream_t s);
constexpr int kRefAcc = 32;  // per-block partial sums of one refinement step
constexpr int kMaxLevels = 8;
// Subsampling stride of graduated refinement level l of L for a cloud of n points.
int gnc_stride(int64_t n, int level, int levels);
cudaError_t launch_refine_level_begin(RansacState *st, cudaStream_t s);
// One IRLS step on the points of P (internal order, w = caller index) whose
// caller index is a multiple of strideP, against the given grid of Q. seeds
// (nP ints, -1 = none; set to -1 at the start of a level): each point's
// neighbour of the previous step, read as the search's start and rewritten.
// chained: launched as a programmatic dependent of the previous step, which
// must be the kernel directly before it in s.
cudaError_t launch_refine_step(const float4 *XP, int nP, int strideP, const GridParams *ge, const int *start_e,
                               const float4 *Xe, float eps_r, float mu, int max_iters, RansacState *st,
                               double *partials, int *seeds, bool chained, cudaStream_t s);
// out[m] = (Q[m * stride], m) for m < ceil(n / stride); Q caller-order xyz.
cudaError_t launch_subsample(const float *xyz, int n, int stride, float4 *out, cudaStream_t s);
cudaError_t launch_final_pose(RansacState *st, float *pose, cudaStream_t s);
cudaError_t launch_final_count(const int *count, const unsigned long long *sum, RansacState *st, cudaStream_t s);

// Objective forward / backward for one pair (lsr_refine.cu). P: caller-order
// float32 xyz; the eps grid of Q carries caller indices in Xe.w. out7 (device):
// E, g_v[3], g_w[3]. dP / dQ (device, caller order) are written when want_grad
// (dQ must be zeroed by the caller), scaled by `scale`.
int objective_blocks(int nP);
// Voxel downsampling (Algorithm 1, first line; lsr_voxel.cu). kb: 6 ints (key
// minima, maxima). launch_vox_cells needs kb's box on the host (ncells) and on
// the device (ncells_dev); cnt, flag: ncells ints, pos: ncells + 1 ints, sums:
// 3 ncells 64-bit words, scan: scan_scratch_ints(ncells) ints; writes at most
// cap points to out and the number of voxels to *n_out.
cudaError_t launch_vox_bounds(const float *P, int64_t n, float leaf, int *kb, cudaStream_t s);
cudaError_t launch_vox_cells(const float *P, int64_t n, float leaf, const int *kb, int64_t ncells,
                             const int *ncells_dev, int *cnt, unsigned long long *sums, int *flag, int *pos,
                             int *scan, float *out, int64_t cap, int64_t *n_out, cudaStream_t s);

// Dense model correction (eq. (7), lsr_surfel.cu). Per keyframe: A = T_old^-1
// and M = T_new T_old^-1 as row-major 3 x 4 (camera-to-world poses).
struct KfPose {
  float A[12], M[12];
};
struct SurfelCam {
  float fx, fy, cx, cy, w, h, dmax;
};
cudaError_t launch_surfel_correct(int64_t n, const float *pos, const float *nrm, const float *t0, const float *tu,
                                  int m, const KfPose *kf, const float *t_kf, const SurfelCam &cam, float *pos_out,
                                  float *nrm_out, uint8_t *keep, unsigned long long *n_keep, cudaStream_t s);

// Information matrix of eq. (5)-(6) for the pose [R | t]: out[0..35] row-major
// Lambda, out[36] = |K|. boxQ: Q's box (lo, hi); partials: 10 x
// information_blocks(nP) doubles.
int information_blocks(int nP);
cudaError_t launch_information(const float *P, int nP, const GridParams *ge, const int *start_e, const float4 *Xe,
                               const float *boxQ, const float R[9], const float t[3], float eps, double *partials,
                               double *out, cudaStream_t s);
// Nearest-neighbour modes (lsr_nn.cu). The single-cell lattice: cell edge
// exact, anchored at the centroid of the box (box[8..10]).
cudaError_t launch_cell_grid_params(const float *box, float cell, int npts, int cap_cells, GridParams *g,
                                    cudaStream_t s);
// nn / d2 of every query (caller-order xyz): exact (nearest within r over the
// grid of cell r) or single (own cell of the single-cell lattice).
cudaError_t launch_nn_stage(const float *X, int nX, const GridParams *g, const int *start, const float4 *Xs, float r,
                            int single, int *nn, float *d2, cudaStream_t s);
// Consensus of the ok hypotheses with the single-cell lookup and/or the
// per-inlier normal check (count / sum as launch_consensus).
cudaError_t launch_consensus_variant(const float4 *XP, int nP, const float4 *NP, const GridParams *g,
                                     const int *start, const float4 *Xs, const float4 *NQ, int nQ, const float *pose,
                                     const uint8_t *ok, const int *n_dev, float eps, bool single, bool normals,
                                     float cos_normal, int *count, unsigned long long *sum, cudaStream_t s);

// Implicit gradient of the refined pose (lsr_implicit.cu): partials holds
// implicit_partials(nP) doubles; out 50 doubles (g 6, H 36, lambda 6, count,
// singular flag); dl_dev: dL/dxi (6 doubles, device); dQ must be zeroed.
int implicit_partials(int nP);
cudaError_t launch_implicit(const float *P, int nP, const GridParams *ge, const int *start_e, const float4 *Xe,
                            int nQ, const double T[16], float eps, double mu, const double *dl_dev,
                            double *partials, double *out, float *dP, float *dQ, cudaStream_t s);
cudaError_t launch_objective(const float *P, int nP, const GridParams *ge, const int *start_e, const float4 *Xe,
                             const double T[16], const double v[3], float eps, float mu, double scale,
                             int want_grad, double *partials, double *out7, float *dP, float *dQ, cudaStream_t s);

}  // namespace lsr
