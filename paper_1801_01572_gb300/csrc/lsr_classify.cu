// lsr_classify.cu -- hypothesis testing (Alg. 1, "Find all inliers") through a
// voxel classification of Q.
//
// Inlier counting asks, for every (hypothesis, point of P), whether the
// transformed point x has a Q point closer than eps. Most x are either deep
// inside the eps-neighbourhood of Q's surface or far from it, so the answer is
// read from a table: Q's box (grown by eps) is cut into voxels of h = eps / k
// (k = 8, 6, 4, ... as fits the table), and two bit-sets are splatted from the
// Q points, with c the voxel centre and rho = sqrt(3) h / 2 its half diagonal:
//   IN   some q has |c - q| <= eps - rho - m: every x of the voxel is an inlier;
//   NEAR some q has |c - q| <= eps + rho + m: without it no x of the voxel is.
// m covers the FP32 rounding of voxel coordinates and of the distance test, so
// a voxel is IN or not-NEAR only if the exact test (d^2 < eps^2 in FP32 over the
// eps grid of eq. (1)) gives the same answer for every point it can contain.
// Points in NEAR-but-not-IN voxels take that exact test, one query at a time
// across a whole warp, stopping at the first Q point within eps; the counts
// are then identical to the exact consensus kernel's.
//
// Selection (the largest count wins, then the smaller mean squared distance)
// does not need every count: without the exact tests the table bounds each
// hypothesis's count between #IN and #IN + #undecided. The registration
// pipeline counts exactly the K hypotheses with the largest upper bounds, takes
// the largest of those counts as C, and counts exactly only the hypotheses
// whose upper bound reaches C: no other can win or tie. The distance sums are
// then computed for the hypotheses tied at the top.
#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kClsThreads = 256;
constexpr int kClsChunk = 2048;
constexpr int kClsMinBlocks = 8;  // resident blocks per SM

// Table geometry from Q's box: the finest voxel (eps / k) whose two bit-sets
// fit kClsCapWords words each; all_amb = 1 if none does (every point then
// takes the exact test).
__global__ void k_cls_params(const float *box, float eps, ClsParams *cp) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float ks[] = {8.f, 6.f, 4.f, 3.f, 2.f, 1.5f, 1.f, 0.5f, 0.25f, 0.125f, 0.0625f};
  ClsParams c{};
  c.all_amb = 1;
  float lo[3] = {box[0], box[1], box[2]}, hi[3] = {box[3], box[4], box[5]};
  float ext = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
  float mag = fmaxf(fmaxf(fmaxf(fabsf(lo[0]), fabsf(hi[0])), fmaxf(fabsf(lo[1]), fabsf(hi[1]))),
                    fmaxf(fabsf(lo[2]), fabsf(hi[2])));
  if (box[6] == 0.f && ext >= 0.f && isfinite(ext) && isfinite(mag)) {
    // rounding of coordinates relative to the table and of the FP32 distance test
    c.m = 1e-6f * (ext + 2.f * eps) + 4e-7f * (mag + eps) + 1e-7f * eps + 1e-9f;
    for (float k : ks) {
      float h = eps / k;
      float pad = eps + 2.f * h + c.m;
      long long n[3];
      bool fits = true;
      for (int d = 0; d < 3; ++d) {
        float e = (hi[d] - lo[d] + 2.f * pad) / h;
        if (!(e < 1e9f)) fits = false;
        n[d] = fits ? (long long)e + 2 : 0;
      }
      const long long sx = (n[0] + 7) / 8, sy = (n[1] + 7) / 8, sz = (n[2] + 3) / 4;
      if (!fits || sx * sy * sz * 8 > kClsCapWords) continue;
      c.ox = lo[0] - pad, c.oy = lo[1] - pad, c.oz = lo[2] - pad;
      c.h = h;
      c.inv_h = 1.f / h;
      c.nx = (int)n[0], c.ny = (int)n[1], c.nz = (int)n[2], c.wx = (int)sx, c.wy = (int)sy;
      float rho = 0.8660254f * h * (1.f + 1e-6f);
      float r_in = eps - rho - c.m;
      c.r_in2 = r_in > 0.f ? r_in * r_in * (1.f - 1e-6f) : -1.f;
      c.r_near = (eps + rho + c.m) * (1.f + 1e-6f);
      c.R = (int)ceilf(c.r_near / h) + 1;
      c.all_amb = 0;
      break;
    }
  }
  *cp = c;
}

// One thread per (Q point, voxel plane dz around it), looping over the rows
// dy in the aligned groups of four that share a brick row: the NEAR bits of a
// row are set over an interval widened beyond the ball (a superset), the IN
// bits over the interval of voxels that pass an explicit distance check (a
// subset); one atomic per brick and bit-set collects the four rows.
__global__ void k_cls_splat(const float4 *__restrict__ XQ, int nQ, const ClsParams *__restrict__ cpp,
                            unsigned *__restrict__ in_bits, unsigned *__restrict__ near_bits) {
  const ClsParams c = *cpp;
  if (c.all_amb) return;
  const int side = 2 * c.R + 1;
  const long long total = (long long)nQ * side;
  const float rn2 = c.r_near * c.r_near;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / side);
    const int dz = (int)(t - (long long)i * side) - c.R;
    const float4 q = XQ[i];
    const float fx = (q.x - c.ox) * c.inv_h, fy = (q.y - c.oy) * c.inv_h, fz = (q.z - c.oz) * c.inv_h;
    const int iz = (int)floorf(fz) + dz;
    if (iz < 0 || iz >= c.nz) continue;
    const float ez = fmaf((float)iz + 0.5f, c.h, c.oz) - q.z;
    if (ez * ez > rn2) continue;
    const int iy0 = (int)floorf(fy);
    const int ylo = max(iy0 - c.R, 0), yhi = min(iy0 + c.R, c.ny - 1);
    const int zsh = (iz & 1) << 4;
    for (int gy = ylo >> 2; gy <= (yhi >> 2); ++gy) {
      int x0r[4], x1r[4], inl[4], inr[4];
      int xmin = 0x7fffffff, xmax = -1;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        x0r[r] = 1, x1r[r] = 0, inl[r] = 1, inr[r] = 0;
        const int iy = 4 * gy + r;
        if (iy < ylo || iy > yhi) continue;
        const float ey = fmaf((float)iy + 0.5f, c.h, c.oy) - q.y;
        const float rem = rn2 - ey * ey - ez * ez;
        if (rem < 0.f) continue;
        const float half = sqrtf(rem) * (1.f + 1e-5f) + c.m;
        int x0 = (int)floorf(fx - half * c.inv_h - 0.5f) - 1, x1 = (int)ceilf(fx + half * c.inv_h - 0.5f) + 1;
        x0 = x0 < 0 ? 0 : x0;
        x1 = x1 >= c.nx ? c.nx - 1 : x1;
        if (x0 > x1) continue;
        x0r[r] = x0, x1r[r] = x1;
        xmin = min(xmin, x0), xmax = max(xmax, x1);
        // IN voxels of the row: those passing the explicit test, an interval
        // (ex grows with the voxel index, the test is monotone in |ex|): an
        // estimate from the ball, each end then settled by the test itself
        const float eyz = fmaf(ey, ey, ez * ez);
        if (c.r_in2 > 0.f && eyz <= c.r_in2) {
          auto pass = [&](int b) {
            const float ex = fmaf((float)b + 0.5f, c.h, c.ox) - q.x;
            return fmaf(ex, ex, eyz) <= c.r_in2;
          };
          const float rr = sqrtf(c.r_in2 - eyz);
          int lo = (int)floorf((q.x - rr - c.ox) * c.inv_h - 0.5f), hi = (int)ceilf((q.x + rr - c.ox) * c.inv_h - 0.5f);
          lo = max(lo, x0), hi = min(hi, x1);
          while (lo <= hi && !pass(lo)) ++lo;
          while (lo <= hi && lo > x0 && pass(lo - 1)) --lo;
          while (hi >= lo && !pass(hi)) --hi;
          while (hi >= lo && hi < x1 && pass(hi + 1)) ++hi;
          inl[r] = lo, inr[r] = hi;
        }
      }
      if (xmax < 0) continue;
      for (int bx = xmin >> 2; bx <= (xmax >> 2); ++bx) {
        unsigned near = 0u, in = 0u;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int b0 = max(x0r[r], 4 * bx), b1 = min(x1r[r], 4 * bx + 3);
          if (b0 > b1) continue;
          near |= ((((1u << (b1 - 4 * bx + 1)) - 1u) & ~((1u << (b0 - 4 * bx)) - 1u)) << (4 * r));
          const int i0 = max(inl[r], 4 * bx), i1 = min(inr[r], 4 * bx + 3);
          if (i0 <= i1) in |= ((((1u << (i1 - 4 * bx + 1)) - 1u) & ~((1u << (i0 - 4 * bx)) - 1u)) << (4 * r));
        }
        if (!near) continue;
        const size_t word = cls_word(c, 4 * bx, 4 * gy, iz);
        atomicOr(near_bits + word, near << zsh);
        if (in) atomicOr(in_bits + word, in << zsh);
      }
    }
  }
}

// Whether a Q point lies closer than eps to (x, y, z): all 32 lanes walk the
// eps-grid candidates of the same query and stop at the first hit. Without
// wrapped storage the nine row ranges (the x-adjacent cells of a row are one
// range) are read at once, one row per lane, and then scanned in the order of
// grid_ranges, 32 candidates at a time.
__device__ __forceinline__ bool warp_any_within(const GridParams &g, const int *__restrict__ start,
                                                const float4 *__restrict__ Xe, float x, float y, float z,
                                                float eps2) {
  const int lane = threadIdx.x & 31;
  const bool wrapped = (g.wx != g.nx) | (g.wy != g.ny) | (g.wz != g.nz);
  if (wrapped) {
    bool hit = false;
    grid_ranges(g, start, x, y, z, [&](int b, int e) {
      if (hit) return;
      for (int base = b; base < e; base += 32) {
        int t = base + lane;
        bool h = t < e && dist2(Xe[t], x, y, z) < eps2;
        if (__any_sync(0xffffffffu, h)) {
          hit = true;
          return;
        }
      }
    });
    return hit;
  }
  const float fx = (x - g.ox) * g.inv_cell, fy = (y - g.oy) * g.inv_cell, fz = (z - g.oz) * g.inv_cell;
  if (!(fx >= -1.f && fx < (float)g.nx + 1.f && fy >= -1.f && fy < (float)g.ny + 1.f && fz >= -1.f &&
        fz < (float)g.nz + 1.f))
    return false;
  const int cx = __float2int_rd(fx), cy = __float2int_rd(fy), cz = __float2int_rd(fz);
  const int x0 = cx - 1 < 0 ? 0 : cx - 1, x1 = cx + 1 > g.nx - 1 ? g.nx - 1 : cx + 1;
  if (x0 > x1) return false;
  if (g.nbmask && cx >= 0 && cx < g.nx && cy >= 0 && cy < g.ny && cz >= 0 && cz < g.nz) {
    const int slot = (cz * g.wy + cy) * g.wx + cx;
    if (!((__ldg(g.nbmask + (slot >> 5)) >> (slot & 31)) & 1u)) return false;
  }
  int b = 0, e = 0;
  if (lane < 9) {
    const int iz = cz + lane / 3 - 1, iy = cy + lane % 3 - 1;
    if (iz >= 0 && iz < g.nz && iy >= 0 && iy < g.ny) {
      const int row = (iz * g.wy + iy) * g.wx;
      if (LSR_IN_BOUNDS(row + x1 + 1, g.ncells + 1, kSiteGridRow) && LSR_IN_BOUNDS(row + x0, g.ncells + 1, kSiteGridRow)) {
        b = start[row + x0], e = start[row + x1 + 1];
#ifdef LSR_CHECKED
        if (e > b && (!LSR_IN_BOUNDS(e - 1, g.npts, kSiteGridPoint) || !LSR_IN_BOUNDS(b, g.npts, kSiteGridPoint)))
          b = e = 0;
#endif
      }
    }
  }
  for (int k = 0; k < 9; ++k) {
    const int bk = __shfl_sync(0xffffffffu, b, k), ek = __shfl_sync(0xffffffffu, e, k);
    for (int base = bk; base < ek; base += 32) {
      const int t = base + lane;
      const bool h = t < ek && dist2(Xe[t], x, y, z) < eps2;
      if (__any_sync(0xffffffffu, h)) return true;
    }
  }
  return false;
}

// One thread block per (hypothesis, chunk of P), as the exact kernel; a lane
// per point. kBounds: count IN points into count and undecided ones into amb.
// Otherwise the undecided lanes are resolved by the whole warp, one at a time,
// and count receives the exact inlier count. The points are XP[v * stride]
// for v < ceil(nP / stride).
// Bounds with c0 (a device count no larger than the winning count, e.g. the
// exact count of some hypothesis): items run chunk-major, so each hypothesis's
// chunks come in order, and prog[s] accumulates (points done << 32 | IN +
// undecided) in one 64-bit word, read as one consistent pair. A chunk whose
// hypothesis already has IN + undecided + points not yet done < c0 is left
// out: that upper bound only falls as chunks finish, so the hypothesis can
// neither win nor tie. (k_bounds_finish then adds the points left out to amb,
// keeping IN + amb an upper bound.)
// Exact counts with c0 and the upper bounds ub_lo + ub_extra of a bounds pass:
// items run chunk-major too, prog[s] accumulates (IN + undecided of the chunks
// done << 32 | their exact count), and a chunk whose hypothesis has exact so
// far + (its upper bound - the upper bound of the chunks done) < c0 is left
// out: its count can no longer reach c0, so it can neither win nor tie (its
// count stays partial, below c0).
template <bool kBounds>
__global__ void __launch_bounds__(kClsThreads, kClsMinBlocks) k_consensus_count(
    const float4 *__restrict__ XP, int nP, int stride, const ClsParams *__restrict__ cpp,
    const unsigned *__restrict__ in_bits, const unsigned *__restrict__ near_bits, const GridParams *__restrict__ gep,
    const int *__restrict__ start, const float4 *__restrict__ Xe, const float *__restrict__ pose,
    const uint8_t *__restrict__ ok, const int *n_dev, int n_host, float eps2, int *__restrict__ count,
    int *__restrict__ amb_count, const int *c0, unsigned long long *prog, const int *__restrict__ ub_lo,
    const int *__restrict__ ub_extra) {
  const ClsParams c = *cpp;
  const GridParams g = kBounds ? GridParams{} : *gep;
  const int nh = n_dev ? *n_dev : n_host;
  const int nv = (nP + stride - 1) / stride;
  const int chunks = (nv + kClsChunk - 1) / kClsChunk;
  const int64_t items = (int64_t)nh * chunks;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool abandon = c0 != nullptr;
  const int cbar = abandon ? *c0 : 0;
  __shared__ int s_cnt[kClsThreads / 32], s_amb[kClsThreads / 32], s_in[kClsThreads / 32], s_skip;
  // item = major * inner + minor (s-major: (s, chunk); chunk-major: (chunk, s)),
  // stepped by gridDim.x without a 64-bit division per item
  const int64_t inner = abandon ? nh : chunks;
  if (inner <= 0) return;
  int64_t major = (int64_t)blockIdx.x / inner, minor = (int64_t)blockIdx.x % inner;
  const int64_t step_major = (int64_t)gridDim.x / inner, step_minor = (int64_t)gridDim.x % inner;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int s = (int)(abandon ? minor : major), ch = (int)(abandon ? major : minor);
    major += step_major, minor += step_minor;
    if (minor >= inner) minor -= inner, ++major;
    if (ok && !ok[s]) continue;
    if (abandon) {
      // (one thread reads the pair, so the whole block takes one decision)
      if (threadIdx.x == 0) {
        const unsigned long long pv = __ldcg(prog + s);
        const long long lo32 = (long long)(unsigned)pv, hi32 = (long long)(pv >> 32);
        s_skip = kBounds ? lo32 + ((long long)nP - hi32) < (long long)cbar
                         : lo32 + ((long long)ub_lo[s] + (long long)ub_extra[s] - hi32) < (long long)cbar;
      }
      __syncthreads();
      const bool skip = s_skip != 0;
      __syncthreads();
      if (skip) continue;
    }
    Rigid12 T;
    T.load(pose + (size_t)s * 12);
    const int i0 = ch * kClsChunk, i1 = min(nv, (ch + 1) * kClsChunk);
    int cnt = 0, namb = 0, nin = 0;
    for (int r = i0; r < i1; r += kClsThreads) {
      const int i = r + threadIdx.x;
      bool in = false, amb = false;
      float x = 0.f, y = 0.f, z = 0.f;
      if (i < i1) {
        T.apply(XP[(size_t)i * stride], x, y, z);
        if (c.all_amb) {
          amb = true;
        } else {
          float fx = (x - c.ox) * c.inv_h, fy = (y - c.oy) * c.inv_h, fz = (z - c.oz) * c.inv_h;
          if (fx >= 0.f && fx < (float)c.nx && fy >= 0.f && fy < (float)c.ny && fz >= 0.f && fz < (float)c.nz) {
            int ix = (int)fx, iy = (int)fy, iz = (int)fz;
            size_t word = cls_word(c, ix, iy, iz);
            unsigned bit = 1u << cls_bit(ix, iy, iz);
            if (__ldg(in_bits + word) & bit)
              in = true;
            else
              amb = (__ldg(near_bits + word) & bit) != 0u;
          }
        }
      }
      cnt += in;
      nin += in;
      namb += amb;
      if (kBounds) continue;
      unsigned pend = __ballot_sync(0xffffffffu, amb);
      while (pend) {
        const int src = __ffs(pend) - 1;
        pend &= pend - 1;
        float qx = __shfl_sync(0xffffffffu, x, src), qy = __shfl_sync(0xffffffffu, y, src),
              qz = __shfl_sync(0xffffffffu, z, src);
        bool hit = warp_any_within(g, start, Xe, qx, qy, qz, eps2);
        if (lane == src) cnt += hit;
      }
    }
    cnt = warp_sum(cnt);
    namb = warp_sum(namb);
    if (!kBounds) nin = warp_sum(nin);
    if (lane == 0) s_cnt[w] = cnt, s_amb[w] = namb, s_in[w] = nin;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tc = 0, ta = 0, ti = 0;
      for (int k = 0; k < kClsThreads / 32; ++k) tc += s_cnt[k], ta += s_amb[k], ti += s_in[k];
      if (tc) atomicAdd(&count[s], tc);
      if (kBounds && ta) atomicAdd(&amb_count[s], ta);
      if (abandon)
        atomicAdd(prog + s, kBounds ? ((unsigned long long)(i1 - i0) << 32) | (unsigned)(tc + ta)
                                    : ((unsigned long long)(ti + ta) << 32) | (unsigned)tc);
    }
    __syncthreads();
  }
}

// After bounds with abandonment: amb[s] += the points of s left out, so that
// IN + amb stays an upper bound of the count (below c0 for those left out).
__global__ void k_bounds_finish(const unsigned long long *__restrict__ prog, const uint8_t *__restrict__ ok,
                                const int *n_dev, int nP, int *__restrict__ amb) {
  const int n = *n_dev;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (ok && !ok[k]) continue;
    const int done = (int)(prog[k] >> 32);
    if (done < nP) amb[k] += nP - done;
  }
}

// out = the largest exact[k] over sel[k] (0 if none): a count some hypothesis
// reaches, so no smaller upper bound can win.
__global__ void __launch_bounds__(1024) k_sel_max(const int *__restrict__ exact, const uint8_t *__restrict__ sel,
                                                  const int *n_dev, int *out) {
  __shared__ int s_max[32];
  const int n = *n_dev;
  int mx = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (sel[k]) mx = max(mx, exact[k]);
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_max[w]);
    *out = m;
  }
}

// One block: L = the maximum of lo over the ok hypotheses, then
// mask[k] = ok[k] && lo[k] + extra[k] >= L (extra == null: 0), if L > 0.
__global__ void __launch_bounds__(1024) k_reach_mask(const int *__restrict__ lo, const int *__restrict__ extra,
                                                     const uint8_t *__restrict__ ok, const int *n_dev,
                                                     uint8_t *__restrict__ mask, int *__restrict__ n_mask,
                                                     int *__restrict__ list) {
  __shared__ int s_max[32];
  const int n = *n_dev;
  int mx = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (!ok || ok[k]) mx = max(mx, lo[k]);
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (int)(blockDim.x >> 5) ? s_max[threadIdx.x] : 0;
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (threadIdx.x == 0) s_max[0] = mx;
  }
  __syncthreads();
  mx = s_max[0];
  __shared__ int s_set;
  if (threadIdx.x == 0) s_set = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int up = lo[k] + (extra ? extra[k] : 0);
    const bool m = (!ok || ok[k]) && (mx == 0 ? extra != nullptr : up >= mx);
    mask[k] = m ? 1 : 0;
    // the set entries are also listed (in no particular order) for the kernels
    // that visit only them
    if (m && (list || n_mask)) {
      const int slot = atomicAdd(&s_set, 1);
      if (list) list[slot] = k;
    }
  }
  if (n_mask) {
    __syncthreads();
    if (threadIdx.x == 0) *n_mask = s_set;
  }
}

// One block: the K ok hypotheses with the largest lo + extra (ties to the
// smaller index), marked in sel (cleared first), by K rounds of block argmax.
__global__ void __launch_bounds__(1024) k_top_upper(const int *__restrict__ lo, const int *__restrict__ extra,
                                                    const uint8_t *__restrict__ ok, const int *n_dev, int K,
                                                    uint8_t *__restrict__ sel) {
  // key: upper bound in the high word, complemented index in the low word,
  // so keys are distinct and a larger key wins (ties to the smaller index).
  // The K-th largest key T is found by radix selection, eight bits at a time
  // from the top; the K keys >= T are then marked.
  __shared__ unsigned hist[256];
  __shared__ unsigned long long s_prefix, s_mask;
  __shared__ unsigned s_need, s_nok;
  const int n = *n_dev;
  auto key_of = [&](int k) {
    return ((unsigned long long)(unsigned)(lo[k] + extra[k]) << 32) | (unsigned)(0x7fffffff - k);
  };
  if (threadIdx.x == 0) s_nok = 0, s_prefix = 0ull, s_mask = 0ull, s_need = (unsigned)K;
  __syncthreads();
  unsigned mine = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) mine += (!ok || ok[k]) ? 1u : 0u;
  atomicAdd(&s_nok, mine);
  __syncthreads();
  if (s_nok <= (unsigned)K) {  // every candidate is selected
    for (int k = threadIdx.x; k < n; k += blockDim.x) sel[k] = (!ok || ok[k]) ? 1 : 0;
    return;
  }
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0u;
    __syncthreads();
    const unsigned long long prefix = s_prefix, mask = s_mask;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      if (ok && !ok[k]) continue;
      const unsigned long long key = key_of(k);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned need = s_need, above = 0u;
      int d = 255;
      for (; d > 0; --d) {
        if (above + hist[d] >= need) break;
        above += hist[d];
      }
      s_need = need - above;
      s_prefix = prefix | ((unsigned long long)d << shift);
      s_mask = mask | (255ull << shift);
    }
    __syncthreads();
  }
  const unsigned long long T = s_prefix;
  for (int k = threadIdx.x; k < n; k += blockDim.x) sel[k] = ((!ok || ok[k]) && key_of(k) >= T) ? 1 : 0;
}

// One block: C = the maximum exact count among sel; then
// rest[k] = ok[k] && !sel[k] && lo[k] + extra[k] >= C and all[k] = sel[k] | rest[k].
__global__ void __launch_bounds__(1024) k_reach_rest(const int *__restrict__ lo, const int *__restrict__ extra,
                                                     const int *__restrict__ exact, const uint8_t *__restrict__ sel,
                                                     const uint8_t *__restrict__ ok, const int *n_dev,
                                                     uint8_t *__restrict__ rest, uint8_t *__restrict__ all) {
  __shared__ int s_max[32];
  const int n = *n_dev;
  int mx = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (sel[k]) mx = max(mx, exact[k]);
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_max[w]);
    s_max[0] = m;
  }
  __syncthreads();
  mx = s_max[0];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const bool r = (!ok || ok[k]) && !sel[k] && lo[k] + extra[k] >= mx;
    rest[k] = r ? 1 : 0;
    all[k] = (r || sel[k]) ? 1 : 0;
  }
}

}  // namespace

cudaError_t launch_cls_build(const float *boxQ, float eps, const float4 *XQ, int nQ, ClsParams *cp, unsigned *in_bits,
                             unsigned *near_bits, cudaStream_t s) {
  LSR_CUDA_TRY(cudaMemsetAsync(in_bits, 0, sizeof(unsigned) * (size_t)kClsCapWords, s));
  LSR_CUDA_TRY(cudaMemsetAsync(near_bits, 0, sizeof(unsigned) * (size_t)kClsCapWords, s));
  LSR_LAUNCH(k_cls_params<<<1, 32, 0, s>>>(boxQ, eps, cp));
  LSR_LAUNCH(k_cls_splat<<<kSms * 16, 256, 0, s>>>(XQ, nQ, cp, in_bits, near_bits));
  return cudaGetLastError();
}

cudaError_t launch_consensus_count(const float4 *XP, int nP, const ClsParams *cp, const unsigned *in_bits,
                                   const unsigned *near_bits, const GridParams *ge, const int *start_e,
                                   const float4 *Xe, const float *pose, const uint8_t *ok, const int *n_dev,
                                   int n_host, float eps, int *count, cudaStream_t s) {
  LSR_LAUNCH(k_consensus_count<false><<<kSms * 8, kClsThreads, 0, s>>>(XP, nP, 1, cp, in_bits, near_bits, ge, start_e,
                                                                       Xe, pose, ok, n_dev, n_host, eps * eps, count,
                                                                       nullptr, nullptr, nullptr, nullptr, nullptr));
  return cudaGetLastError();
}

cudaError_t launch_consensus_count_bar(const float4 *XP, int nP, const ClsParams *cp, const unsigned *in_bits,
                                       const unsigned *near_bits, const GridParams *ge, const int *start_e,
                                       const float4 *Xe, const float *pose, const uint8_t *ok, const int *n_dev,
                                       float eps, int *count, const int *c0, const int *ub_lo, const int *ub_extra,
                                       unsigned long long *prog, cudaStream_t s) {
  LSR_LAUNCH(k_consensus_count<false><<<kSms * 8, kClsThreads, 0, s>>>(XP, nP, 1, cp, in_bits, near_bits, ge, start_e,
                                                                       Xe, pose, ok, n_dev, 0, eps * eps, count,
                                                                       nullptr, c0, prog, ub_lo, ub_extra));
  return cudaGetLastError();
}

cudaError_t launch_consensus_bounds(const float4 *XP, int nP, int stride, const ClsParams *cp,
                                    const unsigned *in_bits, const unsigned *near_bits, const float *pose,
                                    const uint8_t *ok, const int *n_dev, int *in_count, int *amb_count,
                                    const int *c0, unsigned long long *prog, cudaStream_t s) {
  LSR_LAUNCH(k_consensus_count<true><<<kSms * 8, kClsThreads, 0, s>>>(XP, nP, stride, cp, in_bits, near_bits, nullptr,
                                                                      nullptr, nullptr, pose, ok, n_dev, 0, 0.f,
                                                                      in_count, amb_count, c0, prog, nullptr, nullptr));
  if (c0) LSR_LAUNCH(k_bounds_finish<<<kSms * 2, 256, 0, s>>>(prog, ok, n_dev, nP, amb_count));
  return cudaGetLastError();
}

cudaError_t launch_sel_max(const int *exact, const uint8_t *sel, const int *n_dev, int *out, cudaStream_t s) {
  LSR_LAUNCH(k_sel_max<<<1, 1024, 0, s>>>(exact, sel, n_dev, out));
  return cudaGetLastError();
}

cudaError_t launch_top_upper(const int *lo, const int *extra, const uint8_t *ok, const int *n_dev, int K,
                             uint8_t *sel, cudaStream_t s) {
  LSR_LAUNCH(k_top_upper<<<1, 1024, 0, s>>>(lo, extra, ok, n_dev, K, sel));
  return cudaGetLastError();
}

cudaError_t launch_reach_rest(const int *lo, const int *extra, const int *exact, const uint8_t *sel, const uint8_t *ok,
                              const int *n_dev, uint8_t *rest, uint8_t *all, cudaStream_t s) {
  LSR_LAUNCH(k_reach_rest<<<1, 1024, 0, s>>>(lo, extra, exact, sel, ok, n_dev, rest, all));
  return cudaGetLastError();
}

cudaError_t launch_reach_mask(const int *lo, const int *extra, const uint8_t *ok, const int *n_dev, uint8_t *mask, int *n_mask,
                              int *list,
                              cudaStream_t s) {
  LSR_LAUNCH(k_reach_mask<<<1, 1024, 0, s>>>(lo, extra, ok, n_dev, mask, n_mask, list));
  return cudaGetLastError();
}

LSR_CHECK_READER(classify)

}  // namespace lsr
