// lsr_features.cu -- per-point normals, SPFH and FPFH (Algorithm 1, the FPFH
// computation; radii of Sec. IV).
//
// Normals and SPFH are warp-per-point: the 32 lanes of a warp stride over the
// contiguous sorted ranges of the neighbouring grid cells, so the neighbour
// loads of a warp are coalesced and the work per point is split evenly. FPFH
// is lane-per-point over candidates staged in shared memory (see k_fpfh).
#include <math_constants.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations in FP32. a[6]
// = (xx, xy, xz, yy, yz, zz). Returns the eigenvalues w[3] (unsorted) and the
// eigenvectors as the columns of v.
__device__ void sym3_eigen(const float a[6], float w[3], float v[3][3]) {
  float A[3][3] = {{a[0], a[1], a[2]}, {a[1], a[3], a[4]}, {a[2], a[4], a[5]}};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) v[r][c] = (r == c) ? 1.f : 0.f;
  for (int sweep = 0; sweep < 8; ++sweep) {
    float off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    float diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-14f * diag) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      float apq = A[p][q];
      if (apq == 0.f) continue;
      float theta = (A[q][q] - A[p][p]) / (2.f * apq);
      float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      float c = rsqrtf(t * t + 1.f), s = t * c;
      for (int k = 0; k < 3; ++k) {
        float akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - s * akq;
        A[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        float apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - s * aqk;
        A[q][k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        float vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
      }
    }
  }
  w[0] = A[0][0], w[1] = A[1][1], w[2] = A[2][2];
}

// Normal of each point: PCA of the points within r (inclusive, self included),
// accumulated about the query point (one pass), eigenvector of the smallest
// eigenvalue, turned toward the viewpoint; fewer than 3 points: invalid.
// A warp walks the neighbourhoods of 32 points one after another (the lanes
// over each point's candidates); lane k keeps point k's sums, and the 32
// eigen-decompositions then run at once, one per lane.
__global__ void __launch_bounds__(kThreads) k_normals(const float4 *__restrict__ X, int n, const GridParams *gnp,
                                                      const int *__restrict__ start, const float4 *__restrict__ Xn,
                                                      float r2, float3 vp, float4 *__restrict__ N,
                                                      int *__restrict__ count) {
  const GridParams g = *gnp;
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * kThreads + threadIdx.x) >> 5, nwarps = (gridDim.x * kThreads) >> 5;
  // this warp's points: base + k * nwarps for k = 0..31
  for (int base = warp; base < n; base += 32 * nwarps) {
    int mk = 0;
    float ms[3] = {0, 0, 0}, mss[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < 32; ++j) {
      const int i = base + j * nwarps;
      if (i >= n) break;
      float3 p = f3(X[i]);
      int k = 0;
      float s[3] = {0, 0, 0}, ss[6] = {0, 0, 0, 0, 0, 0};
      grid_ranges(g, start, p.x, p.y, p.z, [&](int b, int e) {
        for (int t = b + lane; t < e; t += 32) {
          float4 q = Xn[t];
          float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
          if (dx * dx + dy * dy + dz * dz <= r2) {
            ++k;
            s[0] += dx, s[1] += dy, s[2] += dz;
            ss[0] += dx * dx, ss[1] += dx * dy, ss[2] += dx * dz;
            ss[3] += dy * dy, ss[4] += dy * dz, ss[5] += dz * dz;
          }
        }
      });
      k = warp_sum(k);
      for (int d = 0; d < 3; ++d) s[d] = warp_sum(s[d]);
      for (int d = 0; d < 6; ++d) ss[d] = warp_sum(ss[d]);
      if (lane == j) {
        mk = k;
        for (int d = 0; d < 3; ++d) ms[d] = s[d];
        for (int d = 0; d < 6; ++d) mss[d] = ss[d];
      }
    }
    const int i = base + lane * nwarps;
    if (i >= n) continue;
    const float3 p = f3(X[i]);
    float4 out = make_float4(0.f, 0.f, 0.f, -1.f);
    if (mk >= 3) {
      float ik = 1.f / (float)mk;
      float m[3] = {ms[0] * ik, ms[1] * ik, ms[2] * ik};
      float C[6] = {mss[0] * ik - m[0] * m[0], mss[1] * ik - m[0] * m[1], mss[2] * ik - m[0] * m[2],
                    mss[3] * ik - m[1] * m[1], mss[4] * ik - m[1] * m[2], mss[5] * ik - m[2] * m[2]};
      float w[3], V[3][3];
      sym3_eigen(C, w, V);
      int jm = 0;
      if (w[1] < w[jm]) jm = 1;
      if (w[2] < w[jm]) jm = 2;
      float3 nrm = make_float3(V[0][jm], V[1][jm], V[2][jm]);
      float3 tv = make_float3(vp.x - p.x, vp.y - p.y, vp.z - p.z);
      if (dot3(nrm, tv) < 0.f) nrm = make_float3(-nrm.x, -nrm.y, -nrm.z);
      float sum = w[0] + w[1] + w[2];
      out = make_float4(nrm.x, nrm.y, nrm.z, sum > 0.f ? fmaxf(w[jm], 0.f) / sum : 0.f);
    }
    N[i] = out;
    if (count) count[i] = mk;
  }
}

// Darboux-frame pair features of FPFH (Rusu et al., ICRA 2009). The source is
// the point whose normal makes the smaller angle with the joining line (ties
// keep p); u = n_s, v = (u x e)/|u x e|, w = u x v; alpha = v.n_t, phi = u.e,
// theta = atan2(w.n_t, u.n_t). A pair without a frame (|u x e|^2 < 1e-12) is
// skipped. Bins: 11 per feature over [-1, 1], [-1, 1], [-pi, pi].
// tie (optional): set when the two angles are equal, the one case in which
// the features of (q, p) differ from those of (p, q).
__device__ __forceinline__ bool pair_bins(float3 p, float3 np, float3 q, float3 nq, float d2, int &ba, int &bp,
                                          int &bt, bool *tie = nullptr) {
  float id = rsqrtf(d2);
  float3 e = make_float3((q.x - p.x) * id, (q.y - p.y) * id, (q.z - p.z) * id);
  float cs = fabsf(dot3(np, e)), ct = fabsf(dot3(nq, e));
  if (tie) *tie = cs == ct;
  float3 u = np, nt = nq;
  if (cs < ct) {
    u = nq, nt = np;
    e = make_float3(-e.x, -e.y, -e.z);
  }
  float3 v = cross3(u, e);
  float vn2 = dot3(v, v);
  if (vn2 < 1e-12f) return false;
  float iv = rsqrtf(vn2);
  v = make_float3(v.x * iv, v.y * iv, v.z * iv);
  float3 w = cross3(u, v);
  float alpha = dot3(v, nt), phi = dot3(u, e), theta = atan2f(dot3(w, nt), dot3(u, nt));
  ba = min(max(__float2int_rd((alpha + 1.f) * 5.5f), 0), 10);
  bp = min(max(__float2int_rd((phi + 1.f) * 5.5f), 0), 10);
  bt = min(max(__float2int_rd((theta + CUDART_PI_F) * (11.f / (2.f * CUDART_PI_F))), 0), 10);
  return true;
}

// SPFH, each unordered pair once: the pair (p, t) with t after p in the grid
// order is evaluated by p's warp only. Its features are those of (t, p) as well
// (the source is the point whose normal makes the smaller angle with the
// line, whichever is named first; only an exact tie of the two angles makes
// them differ, and then (t, p) is evaluated too), so they count for both: into
// p's private per-lane column of a per-warp [bin][lane] histogram in shared
// memory (row stride 33 words, so both the lane-private updates and the
// per-bin column sums avoid bank conflicts), and into t's counts H (n x 36
// ints, the 33 bins) by atomic adds. p's own sums
// are added to H at the end of its warp; k_spfh_finish divides. Counts are
// integers, so the result does not depend on the order of the adds. The
// lanes test 32 candidates at a time against r; those within it are queued in
// shared memory and their pair features evaluated 32 at a time, a lane each,
// so that the feature arithmetic runs on full warps.
__global__ void __launch_bounds__(kThreads) k_spfh(const float4 *__restrict__ X, const float4 *__restrict__ N, int n,
                                                   const GridParams *gfp, const int *__restrict__ start, float r2,
                                                   int *__restrict__ H) {
  __shared__ int hist[kWarps][kD * 33];
  // candidates within r, queued until 32 can be evaluated at once (a lane
  // each), so that the pair features run on full warps
  __shared__ int qt_s[kWarps][64];
  __shared__ float qd_s[kWarps][64];
  const GridParams g = *gfp;
  int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  int warp = (blockIdx.x * kThreads + threadIdx.x) >> 5, nwarps = (gridDim.x * kThreads) >> 5;
  int *h = hist[wl];
  int *qt = qt_s[wl];
  float *qd = qd_s[wl];
  for (int i = warp; i < n; i += nwarps) {
    for (int b = 0; b < kD; ++b) h[b * 33 + lane] = 0;
    float3 p = f3(X[i]);
    float4 np4 = N[i];
    if (np4.w >= 0.f) {
      float3 np = f3(np4);
      // the pair (p, t) for the queued candidate of this lane (m lanes)
      auto evaluate = [&](int m) {
        if (lane >= m) return;
        const int t = qt[lane];
        const float d2 = qd[lane];
        const float4 q4 = X[t];
        const float4 nq4 = N[t];
        if (nq4.w < 0.f) return;
        const float dx = q4.x - p.x, dy = q4.y - p.y, dz = q4.z - p.z;
        int ba, bp, bt;
        bool tie = false;
        const bool ok = pair_bins(p, np, f3(q4), f3(nq4), d2, ba, bp, bt, &tie);
        if (ok) {
          h[ba * 33 + lane] += 1;
          h[(kNB + bp) * 33 + lane] += 1;
          h[(2 * kNB + bt) * 33 + lane] += 1;
        }
        int *ht = H + (size_t)t * kDS;
        if (tie) {
          // t's own view of the pair
          const float qx = -dx, qy = -dy, qz = -dz;
          if (!pair_bins(f3(q4), f3(nq4), p, np, qx * qx + qy * qy + qz * qz, ba, bp, bt)) return;
        } else if (!ok) {
          return;
        }
        atomicAdd(ht + ba, 1);
        atomicAdd(ht + kNB + bp, 1);
        atomicAdd(ht + 2 * kNB + bt, 1);
      };
      int cnt = 0;  // queued candidates (the same on every lane)
      grid_ranges(g, start, p.x, p.y, p.z, [&](int b, int e) {
        for (int t0 = b > i + 1 ? b : i + 1; t0 < e; t0 += 32) {
          const int t = t0 + lane;
          bool in = t < e;
          float d2 = 0.f;
          if (in) {
            const float4 q4 = X[t];
            const float dx = q4.x - p.x, dy = q4.y - p.y, dz = q4.z - p.z;
            d2 = dx * dx + dy * dy + dz * dz;
            in = !(d2 > r2 || d2 == 0.f);
          }
          const unsigned m = __ballot_sync(0xffffffffu, in);
          if (in) {
            const int k = cnt + __popc(m & ((1u << lane) - 1u));
            qt[k] = t;
            qd[k] = d2;
          }
          cnt += __popc(m);
          if (cnt >= 32) {
            __syncwarp();
            evaluate(32);
            __syncwarp();
            // move the rest (fewer than 32) to the front
            if (lane < cnt - 32) {
              qt[lane] = qt[32 + lane];
              qd[lane] = qd[32 + lane];
            }
            cnt -= 32;
            __syncwarp();
          }
        }
      });
      __syncwarp();
      evaluate(cnt);
    }
    __syncwarp();
    int *hi = H + (size_t)i * kDS;
    int c = 0;
    for (int l = 0; l < 32; ++l) c += h[lane * 33 + l];
    if (c) atomicAdd(hi + lane, c);
    if (lane == 0) {
      int c2 = 0;
      for (int l = 0; l < 32; ++l) c2 += h[32 * 33 + l];
      if (c2) atomicAdd(hi + 32, c2);
    }
    __syncwarp();
  }
}

// S = H / (pair count), one thread per (point, column); zeros in the padding;
// kout (optional): the pair counts. Every counted pair adds one to each of
// the three sub-histograms, so the count is the sum of the first one.
__global__ void k_spfh_finish(const int *__restrict__ H, int n, float *__restrict__ S, int *__restrict__ kout) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * kDS) return;
  const int i = (int)(t / kDS), b = (int)(t - (int64_t)i * kDS);
  int kk = 0;
#pragma unroll
  for (int k = 0; k < kNB; ++k) kk += H[(size_t)i * kDS + k];
  const float inv = kk > 0 ? 1.f / (float)kk : 0.f;
  S[t] = b < kD ? (float)H[t] * inv : 0.f;
  if (b == 0 && kout) kout[i] = kk;
}

// 16-byte global -> shared copy that completes asynchronously (cp.async).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// FPFH: one query per lane. A window of 32 consecutive points of the
// cell-sorted array is taken by kFpParts warps of one block; the lanes whose
// queries lie in the same grid cell (most of a window: a cell holds dozens of
// points) walk that cell's 3 x 3 x 3 neighbourhood together. The cell's
// candidate ranges are listed, cut into chunks of 32 candidates and dealt out
// to the window's warps round robin; a warp copies its next chunk's positions,
// normal flags and SPFH rows (contiguous in the sorted array) to shared memory
// with coalesced asynchronous copies while it sums the current one, every lane
// reading each candidate from there (a broadcast) and adding its row weighted
// by 1/d when the candidate is its neighbour (0 < d <= r, not itself, valid
// normal). A window spanning several cells walks once per distinct cell. The
// parts' sums are then added in part order (the window's warps meet at a named
// barrier of their own), SPFH(p) added and each lane's three sub-histograms
// rescaled. Every sum runs in a fixed order, so the result is deterministic.
constexpr int kFpParts = 3;                      // warps per window
constexpr int kFpWin = 2;                        // windows per block
constexpr int kFpThreads = 32 * kFpParts * kFpWin;
constexpr int kFpRowV = kDS / 4;                 // float4 per SPFH row
// one staging buffer: 32 rows, 32 positions, 32 normal flags (float4 units)
constexpr int kFpBufV = 32 * kFpRowV + 32 + 8;
constexpr int kFpWarpV = 2 * kFpBufV + 14;    // two buffers and the range list (27 pairs) a warp
constexpr int kFpSmem = kFpParts * kFpWin * kFpWarpV * 16;
static_assert(kFpRowV * 32 * 4 >= (kD + 1) * 32, "the staging buffer holds a part's sums");

// barrier of the kFpParts warps of one window (named barrier 1 + window slot)
__device__ __forceinline__ void window_sync(int wslot) {
  static_assert(kFpWin == 2, "one named barrier per window slot");
  if (wslot == 0)
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kFpParts) : "memory");
  else
    asm volatile("bar.sync 2, %0;" ::"n"(32 * kFpParts) : "memory");
}

__global__ void __launch_bounds__(kFpThreads, 3) k_fpfh(const float4 *__restrict__ X, const float4 *__restrict__ N,
                                                        const float *__restrict__ S, int n, const GridParams *gfp,
                                                        const int *__restrict__ start, float r2,
                                                        float *__restrict__ F) {
  extern __shared__ float4 fp_smem[];
  const GridParams g = *gfp;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int part = wl % kFpParts, wslot = wl / kFpParts;
  float4 *const wbuf = fp_smem + (size_t)wl * kFpWarpV;
  // stage candidates c0 .. c0 + m - 1 into buffer bi
  auto stage = [&](int c0, int m, int bi) {
    float4 *bb = wbuf + bi * kFpBufV;
    if (lane < m) {
      cp_async16(bb + 32 * kFpRowV + lane, X + c0 + lane);
      cp_async4(reinterpret_cast<float *>(bb + 32 * kFpRowV + 32) + lane, &N[c0 + lane].w);
    }
    const float4 *src = reinterpret_cast<const float4 *>(S + (size_t)c0 * kDS);
#pragma unroll
    for (int u = 0; u < kFpRowV; ++u) {
      const int k = lane + 32 * u;
      if (k < kFpRowV * m) cp_async16(bb + k, src + k);
    }
    cp_async_commit();
  };
  const int nwin = (n + 31) / 32;
  // the window's warps meet at its barrier twice a window (the trip count is
  // the same for the whole block)
  for (int wb = blockIdx.x * kFpWin; wb < nwin; wb += gridDim.x * kFpWin) {
    const int i0 = (wb + wslot) * 32;
    const int i = i0 + lane;
    const bool in = i < n;
    const float4 p4 = in ? X[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool valid = in && N[i].w >= 0.f;
    // the cell as the grid walk computes it (the grouping key)
    const int cx = __float2int_rd((p4.x - g.ox) * g.inv_cell), cy = __float2int_rd((p4.y - g.oy) * g.inv_cell),
              cz = __float2int_rd((p4.z - g.oz) * g.inv_cell);
    float acc[kD];
#pragma unroll
    for (int b = 0; b < kD; ++b) acc[b] = 0.f;
    int kk = 0;
    unsigned todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
      const int lead = __ffs(todo) - 1;
      const int lx = __shfl_sync(0xffffffffu, cx, lead), ly = __shfl_sync(0xffffffffu, cy, lead),
                lz = __shfl_sync(0xffffffffu, cz, lead);
      const bool mine = valid && cx == lx && cy == ly && cz == lz && ((todo >> lane) & 1u);
      todo &= ~__ballot_sync(0xffffffffu, mine);
      // the leader's position gives the cell's ranges (the same for every
      // lane of the group and every part); every lane runs the uniform loop
      const float px = __shfl_sync(0xffffffffu, p4.x, lead), py = __shfl_sync(0xffffffffu, p4.y, lead),
                  pz = __shfl_sync(0xffffffffu, p4.z, lead);
      // the cell's candidate ranges, listed first (uniform), then dealt out
      // to the window's warps 32 candidates at a time, round robin
      int *rl = reinterpret_cast<int *>(wbuf + 2 * kFpBufV);
      int nr = 0;
      grid_ranges(g, start, px, py, pz, [&](int b, int e) {
        if (b >= e) return;
        if (lane == 0) rl[2 * nr] = b, rl[2 * nr + 1] = e;
        ++nr;
      });
      __syncwarp();
      // (r, k): chunk k of range r; advance past the ends of ranges
      auto settle = [&](int &r, int &k) {
        while (r < nr) {
          const int nk = (rl[2 * r + 1] - rl[2 * r] + 31) >> 5;
          if (k < nk) break;
          k -= nk;
          ++r;
        }
      };
      auto chunk = [&](int r, int k, int &c0, int &m) {
        c0 = rl[2 * r] + 32 * k;
        m = rl[2 * r + 1] - c0 < 32 ? rl[2 * r + 1] - c0 : 32;
      };
      int r = 0, k = part;
      settle(r, k);
      int bi = 0;
      if (r < nr) {
        int c0, m;
        chunk(r, k, c0, m);
        stage(c0, m, 0);
      }
#pragma unroll 1
      while (r < nr) {
        int c0, m;
        chunk(r, k, c0, m);
        int rn = r, kn = k + kFpParts;
        settle(rn, kn);
        // the next chunk's copies run while this one is summed
        if (rn < nr) {
          int n0, nm;
          chunk(rn, kn, n0, nm);
          stage(n0, nm, bi ^ 1);
          cp_async_wait_group<1>();
        } else {
          cp_async_wait_group<0>();
        }
        __syncwarp();
        const float4 *rows = wbuf + bi * kFpBufV, *pos = rows + 32 * kFpRowV;
        const float *nw = reinterpret_cast<const float *>(pos + 32);
#pragma unroll 1
        for (int j = 0; j < m; ++j) {
          const float4 q4 = pos[j];
          const float dx = q4.x - p4.x, dy = q4.y - p4.y, dz = q4.z - p4.z;
          const float d2 = dx * dx + dy * dy + dz * dz;
          const bool acc_t = mine && c0 + j != i && d2 <= r2 && d2 != 0.f && nw[j] >= 0.f;
          if (!__any_sync(0xffffffffu, acc_t)) continue;
          const float w = acc_t ? rsqrtf(d2) : 0.f;
          kk += acc_t ? 1 : 0;
          const float4 *rj = rows + kFpRowV * j;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 v = rj[q];
            acc[4 * q + 0] += w * v.x;
            acc[4 * q + 1] += w * v.y;
            acc[4 * q + 2] += w * v.z;
            acc[4 * q + 3] += w * v.w;
          }
          acc[32] += w * rj[8].x;
        }
        __syncwarp();  // this buffer is refilled two chunks on
        r = rn, k = kn, bi ^= 1;
      }
    }
    // the parts' sums meet in the staging buffers ([bin][lane], then counts)
    float *cb = reinterpret_cast<float *>(wbuf);
#pragma unroll
    for (int b = 0; b < kD; ++b) cb[b * 32 + lane] = acc[b];
    cb[kD * 32 + lane] = __int_as_float(kk);
    window_sync(wslot);
    if (part == 0 && in) {
      kk = 0;
#pragma unroll
      for (int b = 0; b < kD; ++b) acc[b] = 0.f;
      for (int pp = 0; pp < kFpParts; ++pp) {
        const float *ob = reinterpret_cast<const float *>(fp_smem + (size_t)(wslot * kFpParts + pp) * kFpWarpV);
#pragma unroll
        for (int b = 0; b < kD; ++b) acc[b] += ob[b * 32 + lane];
        kk += __float_as_int(ob[kD * 32 + lane]);
      }
      float f[kD];
      const float ik = kk > 0 ? 1.f / (float)kk : 0.f;
      const float *srow_i = S + (size_t)i * kDS;
#pragma unroll
      for (int b = 0; b < kD; ++b) f[b] = valid ? srow_i[b] + acc[b] * ik : 0.f;
      // sub-histograms: bins 0..10, 11..21, 22..32
      float gs[3];
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        float t = 0.f;
#pragma unroll
        for (int b = 0; b < kNB; ++b) t += f[h * kNB + b];
        gs[h] = t;
      }
      float *row = F + (size_t)i * kDS;
#pragma unroll
      for (int b = 0; b < kD; ++b) row[b] = gs[b / kNB] > 0.f ? f[b] / gs[b / kNB] : 0.f;
#pragma unroll
      for (int b = kD; b < kDS; ++b) row[b] = 0.f;
    }
    window_sync(wslot);  // the buffers are reused by the next window
  }
}

inline int blocks_for_warps(int n) {
  int b = (int)lsr_div_up(n, kWarps);
  return b < 1 ? 1 : (b > kSms * 64 ? kSms * 64 : b);
}

}  // namespace

cudaError_t launch_normals(const float4 *X, int n, const GridParams *gn, const int *start_n, const float4 *Xn, float r,
                           float3 vp, float4 *N, int *count, cudaStream_t s) {
  // about 32 points a warp (the eigen-decompositions run a lane each)
  const int64_t nb = lsr_div_up(lsr_div_up(n > 0 ? n : 1, 32), kWarps);
  LSR_LAUNCH(k_normals<<<(int)(nb < kSms * 64 ? nb : kSms * 64), kThreads, 0, s>>>(X, n, gn, start_n, Xn, r * r, vp, N,
                                                                                   count));
  return cudaGetLastError();
}

cudaError_t launch_spfh(const float4 *X, const float4 *N, int n, const GridParams *gf, const int *start_f, float r,
                        float *spfh, int *k, void *scratch, cudaStream_t s) {
  int *H = static_cast<int *>(scratch);
  LSR_CUDA_TRY(cudaMemsetAsync(H, 0, sizeof(int) * kDS * (size_t)n, s));
  LSR_LAUNCH(k_spfh<<<blocks_for_warps(n), kThreads, 0, s>>>(X, N, n, gf, start_f, r * r, H));
  LSR_LAUNCH(k_spfh_finish<<<(int)lsr_div_up((int64_t)n * kDS, 256), 256, 0, s>>>(H, n, spfh, k));
  return cudaGetLastError();
}

cudaError_t launch_fpfh(const float4 *X, const float4 *N, const float *spfh, int n, const GridParams *gf,
                        const int *start_f, float r, float *fpfh, cudaStream_t s) {
  const int64_t nb = lsr_div_up(lsr_div_up(n > 0 ? n : 1, 32), kFpWin);
  // dynamic shared memory above the default 48 KB
  LSR_CUDA_TRY(cudaFuncSetAttribute(k_fpfh, cudaFuncAttributeMaxDynamicSharedMemorySize, kFpSmem));
  LSR_LAUNCH(k_fpfh<<<(int)(nb < kSms * 64 ? nb : kSms * 64), kFpThreads, kFpSmem, s>>>(X, N, spfh, n, gf, start_f,
                                                                                        r * r, fpfh));
  return cudaGetLastError();
}

LSR_CHECK_READER(features)

}  // namespace lsr
