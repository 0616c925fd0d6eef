// lsr_grid.cu -- bounding boxes, the uniform 3D grid of eq. (1) and its
// construction by a deterministic counting sort.
//
// The grid replaces a k-d tree for neighbour search (Sec. IV: O(1) cell
// lookup, no data-dependent branching on the search path). Cells are stored
// densely over the bounding box; points are sorted by cell so that the three
// x-adjacent cells of a row form one contiguous range, and a radius query
// reads at most nine contiguous ranges.
#include <float.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kBoxThreads = 256;
constexpr int kBoxItems = 8;

__device__ __forceinline__ float3 load_xyz(const float *xyz, int i) {
  return make_float3(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
}

// Per block: min (3), max (3), non-finite flag, count and coordinate sums (3)
// of the finite points, as kBoxPart doubles.
template <bool kF4>
__global__ void __launch_bounds__(kBoxThreads) k_bbox_partial(const void *src, int n, double *partials) {
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  float bad = 0.f, cnt = 0.f;
  float sum[3] = {0.f, 0.f, 0.f};
  int base = blockIdx.x * kBoxThreads * kBoxItems;
  for (int k = 0; k < kBoxItems; ++k) {
    int i = base + k * kBoxThreads + threadIdx.x;
    if (i >= n) break;
    float3 p;
    if (kF4) {
      float4 q = reinterpret_cast<const float4 *>(src)[i];
      p = make_float3(q.x, q.y, q.z);
    } else {
      p = load_xyz(reinterpret_cast<const float *>(src), i);
    }
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) {
      bad = 1.f;
      continue;
    }
    lo[0] = fminf(lo[0], p.x), lo[1] = fminf(lo[1], p.y), lo[2] = fminf(lo[2], p.z);
    hi[0] = fmaxf(hi[0], p.x), hi[1] = fmaxf(hi[1], p.y), hi[2] = fmaxf(hi[2], p.z);
    sum[0] += p.x, sum[1] += p.y, sum[2] += p.z;
    cnt += 1.f;
  }
  for (int off = 16; off > 0; off >>= 1) {
    for (int d = 0; d < 3; ++d) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
      sum[d] += __shfl_xor_sync(0xffffffffu, sum[d], off);
    }
    bad = fmaxf(bad, __shfl_xor_sync(0xffffffffu, bad, off));
    cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
  }
  __shared__ float sm[kBoxThreads / 32][kBoxPart];
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) {
    for (int d = 0; d < 3; ++d) sm[w][d] = lo[d], sm[w][3 + d] = hi[d], sm[w][8 + d] = sum[d];
    sm[w][6] = bad;
    sm[w][7] = cnt;
  }
  __syncthreads();
  if (threadIdx.x < kBoxPart) {
    int t = threadIdx.x;
    double v = sm[0][t];
    for (int k = 1; k < kBoxThreads / 32; ++k) {
      double u = sm[k][t];
      v = t < 3 ? fmin(v, u) : (t < 7 ? fmax(v, u) : v + u);
    }
    partials[(size_t)kBoxPart * blockIdx.x + t] = v;
  }
}

// box: min (3), max (3), non-finite flag, number of finite points, centroid (3).
__global__ void k_bbox_final(const double *partials, int nblk, float *box) {
  __shared__ double acc[kBoxPart];
  int t = threadIdx.x;
  if (t < kBoxPart) {
    double v = partials[t];
    for (int b = 1; b < nblk; ++b) {
      double u = partials[(size_t)kBoxPart * b + t];
      v = t < 3 ? fmin(v, u) : (t < 7 ? fmax(v, u) : v + u);
    }
    acc[t] = v;
  }
  __syncthreads();
  if (t < 8) box[t] = (float)acc[t];
  if (t >= 8 && t < 11) box[t] = acc[7] > 0.0 ? (float)(acc[t] / acc[7]) : 0.f;
  if (t == 11) box[t] = 0.f;
}

__global__ void k_grid_params(const float *box, float radius, int npts, int cap, GridParams *g) {
  if (threadIdx.x != 0) return;
  GridParams q;
  float ext[3] = {box[3] - box[0], box[4] - box[1], box[5] - box[2]};
  // Cell coordinates (x - origin) / cell are computed in FP32 with a relative
  // error of a few units of 2^-24 of the box extent; the cell is enlarged by
  // that margin (at least 1e-4) so that two points within the radius never
  // land more than one cell apart.
  float emax = fmaxf(fmaxf(ext[0], ext[1]), ext[2]);
  if (!(emax >= 0.f) || !isfinite(emax)) emax = 0.f;
  float delta = fmaxf(1e-4f, 8.f * 5.9604645e-8f * emax / radius);
  float cell = radius * (1.f + delta);
  q.cell = cell;
  q.inv_cell = 1.0f / cell;
  q.ox = box[0], q.oy = box[1], q.oz = box[2];
  int nn[3];
  for (int d = 0; d < 3; ++d) {
    float e = ext[d] * q.inv_cell;
    if (!(e >= 0.f)) e = 0.f;            // empty or non-finite input
    if (e > 1073741824.f) e = 1073741824.f;
    nn[d] = (int)floorf(e) + 1;
  }
  q.nx = nn[0], q.ny = nn[1], q.nz = nn[2];
  long long cx = nn[0], cy = nn[1], cz = nn[2];
  long long wx = cx, wy = cy, wz = cz;
  if (wx * wy * wz > cap) {
    if (wx * wy <= cap) {
      wz = cap / (wx * wy);
    } else {
      wz = 1;
      if (wx <= cap) {
        wy = cap / wx;
      } else {
        wy = 1;
        wx = cap;
      }
    }
    if (wz < 1) wz = 1;
    if (wy < 1) wy = 1;
  }
  q.wx = (int)wx, q.wy = (int)wy, q.wz = (int)wz;
  q.ncells = (int)(wx * wy * wz);
  q.npts = npts;
  q.pad_ = 0;
  q.nbmask = nullptr;
  *g = q;
}

// Dilate the occupied storage cells into their 3 x 3 x 3 neighbourhoods
// (neighbourhoods are symmetric, so a query cell's bit is set iff some point
// lies in the block around it; wrapped axes dilate modulo the stored extent,
// which can only add bits).
__global__ void k_nbmask(const GridParams *gp, const int *start, unsigned *mask) {
  const GridParams g = *gp;
  bool wx = g.wx != g.nx, wy = g.wy != g.ny, wz = g.wz != g.nz;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncells; c += gridDim.x * blockDim.x) {
    if (start[c + 1] == start[c]) continue;
    int sx = c % g.wx, sy = (c / g.wx) % g.wy, sz = c / (g.wx * g.wy);
    for (int dz = -1; dz <= 1; ++dz) {
      int z = sz + dz;
      if (z < 0 || z >= g.wz) {
        if (!wz) continue;
        z = (z + g.wz) % g.wz;
      }
      for (int dy = -1; dy <= 1; ++dy) {
        int y = sy + dy;
        if (y < 0 || y >= g.wy) {
          if (!wy) continue;
          y = (y + g.wy) % g.wy;
        }
        for (int dx = -1; dx <= 1; ++dx) {
          int x = sx + dx;
          if (x < 0 || x >= g.wx) {
            if (!wx) continue;
            x = (x + g.wx) % g.wx;
          }
          int s = (z * g.wy + y) * g.wx + x;
          atomicOr(&mask[s >> 5], 1u << (s & 31));
        }
      }
    }
  }
}

__global__ void k_set_mask(GridParams *g, const unsigned *mask) {
  if (threadIdx.x == 0) g->nbmask = mask;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int cell_slot(const GridParams &g, float x, float y, float z) {
  int cx = clampi(__float2int_rd((x - g.ox) * g.inv_cell), 0, g.nx - 1);
  int cy = clampi(__float2int_rd((y - g.oy) * g.inv_cell), 0, g.ny - 1);
  int cz = clampi(__float2int_rd((z - g.oz) * g.inv_cell), 0, g.nz - 1);
  return ((cz % g.wz) * g.wy + (cy % g.wy)) * g.wx + (cx % g.wx);
}

template <bool kF4>
__global__ void k_slots(const void *src, int n, const GridParams *gp, int *slot, int *counts) {
  GridParams g = *gp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float3 p;
    if (kF4) {
      float4 q = reinterpret_cast<const float4 *>(src)[i];
      p = make_float3(q.x, q.y, q.z);
    } else {
      p = load_xyz(reinterpret_cast<const float *>(src), i);
    }
    int s = cell_slot(g, p.x, p.y, p.z);
    slot[i] = s;
    atomicAdd(&counts[s], 1);
  }
}

__global__ void k_scatter(int n, const int *slot, const int *start, int *cursor, int *tmp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int s = slot[i];
    tmp[start[s] + atomicAdd(&cursor[s], 1)] = i;
  }
}

// One warp per cell: order the cell's entries by source index (rank = number
// of smaller indices in the cell) and write the sorted points.
template <bool kF4>
__global__ void k_cell_order(const void *src, const GridParams *gp, const int *start, const int *tmp, float4 *out,
                             int *inv_out) {
  int ncells = gp->ncells;
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int c = warp; c < ncells; c += nwarps) {
    int b = start[c], e = start[c + 1];
    for (int t = b + lane; t < e; t += 32) {
      int v = tmp[t];
      int rank = 0;
      for (int u = b; u < e; ++u) rank += tmp[u] < v;
      int k = b + rank;
      float4 o;
      if (kF4) {
        o = reinterpret_cast<const float4 *>(src)[v];
      } else {
        float3 p = load_xyz(reinterpret_cast<const float *>(src), v);
        o = make_float4(p.x, p.y, p.z, 0.f);
      }
      o.w = __int_as_float(v);
      out[k] = o;
      if (inv_out) inv_out[v] = k;
    }
  }
}

// ---------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int *sm_warp, int *total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int off = 1; off < 32; off <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) sm_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < (kScanThreads / 32) ? sm_warp[lane] : 0;
    for (int off = 1; off < 32; off <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += y;
    }
    if (lane < (kScanThreads / 32)) sm_warp[lane] = s;
  }
  __syncthreads();
  int warp_off = w > 0 ? sm_warp[w - 1] : 0;
  *total = sm_warp[kScanThreads / 32 - 1];
  __syncthreads();
  return warp_off + x - v;
}

// Scans in[0..n] with in[n] taken as 0, so out[n] is the total.
__global__ void __launch_bounds__(kScanThreads) k_scan_local(const int *in, int *out, const int *n_dev, int *block_sums) {
  __shared__ int sm[kScanThreads / 32];
  int n1 = *n_dev + 1;
  int base = blockIdx.x * kScanTile;
  if (base >= n1) {
    if (threadIdx.x == 0) block_sums[blockIdx.x] = 0;
    return;
  }
  int v[kScanItems];
  int sum = 0;
  int i0 = base + threadIdx.x * kScanItems;
  for (int k = 0; k < kScanItems; ++k) {
    int i = i0 + k;
    v[k] = (i < n1 - 1) ? in[i] : 0;
    sum += v[k];
  }
  int total;
  int pre = block_exclusive_scan(sum, sm, &total);
  for (int k = 0; k < kScanItems; ++k) {
    int i = i0 + k;
    if (i < n1) out[i] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(int *block_sums, int nblocks) {
  __shared__ int sm[kScanThreads / 32];
  int carry = 0;
  for (int base = 0; base < nblocks; base += kScanThreads) {
    int i = base + threadIdx.x;
    int v = i < nblocks ? block_sums[i] : 0;
    int total;
    int pre = block_exclusive_scan(v, sm, &total);
    if (i < nblocks) block_sums[i] = carry + pre;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int *out, const int *n_dev, const int *block_sums) {
  int n1 = *n_dev + 1;
  int base = blockIdx.x * kScanTile;
  if (base >= n1 || blockIdx.x == 0) return;
  int add = block_sums[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    int i = base + k;
    if (i < n1) out[i] += add;
  }
}

__global__ void k_ncells_ptr(const GridParams *g, int *dst) {
  if (threadIdx.x == 0) *dst = g->ncells;
}

inline int grid_blocks(int n, int threads = 256) {
  int b = (int)lsr_div_up(n, threads);
  return b < 1 ? 1 : (b > 65535 * 8 ? 65535 * 8 : b);
}

}  // namespace

int bbox_blocks(int n) { return (int)lsr_div_up(n > 0 ? n : 1, kBoxThreads * kBoxItems); }

cudaError_t launch_bbox_xyz(const float *xyz, int n, double *partials, int nblk_cap, float *box, cudaStream_t s) {
  int nb = bbox_blocks(n);
  if (nb > nblk_cap) return cudaErrorInvalidValue;
  LSR_LAUNCH(k_bbox_partial<false><<<nb, kBoxThreads, 0, s>>>(xyz, n, partials));
  LSR_LAUNCH(k_bbox_final<<<1, 32, 0, s>>>(partials, nb, box));
  return cudaGetLastError();
}

cudaError_t launch_bbox_f4(const float4 *x, int n, double *partials, int nblk_cap, float *box, cudaStream_t s) {
  int nb = bbox_blocks(n);
  if (nb > nblk_cap) return cudaErrorInvalidValue;
  LSR_LAUNCH(k_bbox_partial<true><<<nb, kBoxThreads, 0, s>>>(x, n, partials));
  LSR_LAUNCH(k_bbox_final<<<1, 32, 0, s>>>(partials, nb, box));
  return cudaGetLastError();
}

cudaError_t launch_grid_params(const float *box, float radius, int npts, int cap_cells, GridParams *g, cudaStream_t s) {
  LSR_LAUNCH(k_grid_params<<<1, 32, 0, s>>>(box, radius, npts, cap_cells, g));
  return cudaGetLastError();
}

int64_t nbmask_words(int cap_cells) { return cap_cells / 32 + 2; }

cudaError_t build_nbmask(GridParams *g, const int *start, int cap_cells, unsigned *mask, cudaStream_t s) {
  LSR_CUDA_TRY(cudaMemsetAsync(mask, 0, sizeof(unsigned) * (size_t)nbmask_words(cap_cells), s));
  int b = (int)lsr_div_up(cap_cells, 256);
  LSR_LAUNCH(k_nbmask<<<b < kSms * 16 ? b : kSms * 16, 256, 0, s>>>(g, start, mask));
  LSR_LAUNCH(k_set_mask<<<1, 32, 0, s>>>(g, mask));
  return cudaGetLastError();
}

int64_t scan_scratch_ints(int64_t n) { return lsr_div_up(n + 1, kScanTile) + 64; }

cudaError_t scan_exclusive(const int *in, int *out, const int *n_dev, int cap, int *scratch, cudaStream_t s) {
  int nblocks = (int)lsr_div_up((int64_t)cap + 1, kScanTile);
  LSR_LAUNCH(k_scan_local<<<nblocks, kScanThreads, 0, s>>>(in, out, n_dev, scratch));
  LSR_LAUNCH(k_scan_blocks<<<1, kScanThreads, 0, s>>>(scratch, nblocks));
  LSR_LAUNCH(k_scan_add<<<nblocks, kScanThreads, 0, s>>>(out, n_dev, scratch));
  return cudaGetLastError();
}

template <bool kF4>
static cudaError_t build_grid_impl(const void *src, int n, const GridParams *g, int cap_cells, int *start, float4 *out,
                                   int *inv_out, GridScratch sc, cudaStream_t s) {
  LSR_CUDA_TRY(cudaMemsetAsync(sc.counts, 0, sizeof(int) * ((size_t)cap_cells + 1), s));
  LSR_LAUNCH(k_slots<kF4><<<grid_blocks(n), 256, 0, s>>>(src, n, g, sc.slot, sc.counts));
  // the cell count lives in device memory; keep a copy next to the counts
  int *ncells_dev = sc.counts + cap_cells;  // counts[cap] is never used as a cell
  LSR_LAUNCH(k_ncells_ptr<<<1, 32, 0, s>>>(g, ncells_dev));
  LSR_CUDA_TRY(scan_exclusive(sc.counts, start, ncells_dev, cap_cells, sc.scan, s));
  LSR_CUDA_TRY(cudaMemsetAsync(sc.counts, 0, sizeof(int) * (size_t)cap_cells, s));
  LSR_LAUNCH(k_scatter<<<grid_blocks(n), 256, 0, s>>>(n, sc.slot, start, sc.counts, sc.tmp));
  // warps stride over the cells (most are empty: a block per cell would spend
  // the kernel on scheduling blocks)
  const int cells_warps = cap_cells < kSms * 16 * 8 ? cap_cells : kSms * 16 * 8;
  LSR_LAUNCH(k_cell_order<kF4><<<grid_blocks(cells_warps * 32, 256), 256, 0, s>>>(src, g, start, sc.tmp, out, inv_out));
  return cudaGetLastError();
}

cudaError_t build_grid_xyz(const float *xyz, int n, const GridParams *g, int cap_cells, int *start, float4 *out,
                           int *inv_out, GridScratch sc, cudaStream_t s) {
  return build_grid_impl<false>(xyz, n, g, cap_cells, start, out, inv_out, sc, s);
}

cudaError_t build_grid_f4(const float4 *x, int n, const GridParams *g, int cap_cells, int *start, float4 *out,
                          GridScratch sc, cudaStream_t s) {
  return build_grid_impl<true>(x, n, g, cap_cells, start, out, nullptr, sc, s);
}

}  // namespace lsr
