// lsr_nn.cu -- the nearest-neighbour modes of the consensus and the variant
// consensus kernels.
//
// Exact mode (the default everywhere): the nearest Q point within the radius
// over every cell of the uniform grid of eq. (1) that the ball overlaps.
//
// Single-cell mode (the paper's O(1) lookup, Sec. IV after eq. (1)): Q is
// binned into cells of edge `cell` on a lattice anchored at Q's centroid c,
// cell index = floor((x - c) / cell) per axis, and a query looks only in its
// own cell. It is approximate -- a neighbour across a cell face is missed --
// and can only lose inliers, never add one. The lattice origin is moved to
// the first lattice plane below the bounding box (c + k cell, k integer), so
// the dense cell range starts at 0; when the box holds more cells than the
// storage, cells wrap and a query keeps only candidates whose own cell
// coordinates equal its own.
//
// Variant consensus (lsr_params.nn_mode, normal_mode): per (hypothesis, chunk
// of P) a block counts the points whose nearest Q point (exact or single
// cell) is closer than eps and, with the per-inlier normal check, whose normal
// agrees with the point's rotated normal (cos >= cos_normal); distance sums in
// 2^-40 fixed point, as the exact consensus kernel.
#include <float.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kNnThreads = 256;
constexpr int kVarChunk = 2048;

// Grid parameters of the single-cell lattice: cell exact (no rounding margin),
// origin on the lattice through the centroid (box[8..10]).
__global__ void k_cell_grid_params(const float *box, float cell, int npts, int cap, GridParams *g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  GridParams q;
  q.cell = cell;
  q.inv_cell = 1.0f / cell;
  const float c[3] = {box[8], box[9], box[10]};
  float o[3];
  int nn[3];
  for (int d = 0; d < 3; ++d) {
    const double k = floor(((double)box[d] - (double)c[d]) / (double)cell);
    o[d] = (float)((double)c[d] + k * (double)cell);
    float e = (box[3 + d] - o[d]) * q.inv_cell;
    if (!(e >= 0.f)) e = 0.f;
    if (e > 1073741824.f) e = 1073741824.f;
    nn[d] = (int)floorf(e) + 1;
  }
  q.ox = o[0], q.oy = o[1], q.oz = o[2];
  q.nx = nn[0], q.ny = nn[1], q.nz = nn[2];
  long long wx = nn[0], wy = nn[1], wz = nn[2];
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

// Nearest point of (x, y, z)'s own cell: (index into Xs or -1, squared distance).
__device__ __forceinline__ int single_cell_nn(const GridParams &g, const int *__restrict__ start,
                                              const float4 *__restrict__ Xs, float x, float y, float z, float &best) {
  best = FLT_MAX;
  const float fx = (x - g.ox) * g.inv_cell, fy = (y - g.oy) * g.inv_cell, fz = (z - g.oz) * g.inv_cell;
  if (!(fx >= 0.f && fx < (float)g.nx && fy >= 0.f && fy < (float)g.ny && fz >= 0.f && fz < (float)g.nz)) return -1;
  const int cx = __float2int_rd(fx), cy = __float2int_rd(fy), cz = __float2int_rd(fz);
  if (cx >= g.nx || cy >= g.ny || cz >= g.nz) return -1;
  const bool wrapped = (g.wx != g.nx) | (g.wy != g.ny) | (g.wz != g.nz);
  const int slot = ((cz % g.wz) * g.wy + (cy % g.wy)) * g.wx + (cx % g.wx);
  if (!LSR_IN_BOUNDS(slot + 1, g.ncells + 1, kSiteGridSlot)) return -1;
  const int b = start[slot], e = start[slot + 1];
  int bt = -1, bidx = 0x7fffffff;
  for (int t = b; t < e; ++t) {
    if (!LSR_IN_BOUNDS(t, g.npts, kSiteGridPoint)) break;
    const float4 q = Xs[t];
    if (wrapped && (__float2int_rd((q.x - g.ox) * g.inv_cell) != cx || __float2int_rd((q.y - g.oy) * g.inv_cell) != cy ||
                    __float2int_rd((q.z - g.oz) * g.inv_cell) != cz))
      continue;
    const float d2 = dist2(q, x, y, z);
    const int qi = __float_as_int(q.w);
    if (d2 < best || (d2 == best && qi < bidx)) best = d2, bt = t, bidx = qi;
  }
  return bt;
}

// Stage kernel: nearest Q point of every query (caller-order xyz) in either
// mode; nn = the carried index (caller order of Q) or -1, d2 = its squared
// distance or +inf.
template <int G>
__global__ void __launch_bounds__(kNnThreads) k_nn_stage(const float *__restrict__ X, int nX, const GridParams *gp,
                                                         const int *__restrict__ start, const float4 *__restrict__ Xs,
                                                         float r2, int single, int *__restrict__ nn,
                                                         float *__restrict__ d2) {
  const GridParams g = *gp;
  constexpr int GPB = kNnThreads / G;
  const int grp = threadIdx.x / G, sub = threadIdx.x & (G - 1);
  for (int r0 = blockIdx.x * GPB; r0 < nX; r0 += gridDim.x * GPB) {
    const int i = r0 + grp;
    const bool valid = i < nX;
    const float x = valid ? X[3 * i] : __int_as_float(0x7fc00000), y = valid ? X[3 * i + 1] : 0.f,
                z = valid ? X[3 * i + 2] : 0.f;
    float best;
    int bt;
    if (single) {
      bt = single_cell_nn(g, start, Xs, x, y, z, best);
    } else {
      int bidx;
      group_nn<G>(g, start, Xs, x, y, z, r2, best, bt, bidx);
    }
    if (!valid || sub != 0) continue;
    nn[i] = bt >= 0 ? __float_as_int(Xs[bt].w) : -1;
    d2[i] = bt >= 0 ? best : __int_as_float(0x7f800000);
  }
}

// Variant consensus over the ok hypotheses (see the file comment). XP: P in
// any order with w = its internal index (rows of NP); Xs: the grid's sorted Q
// points with w = Q's internal index (rows of NQ).
template <int G, bool kSingle, bool kNormals>
__global__ void __launch_bounds__(kNnThreads) k_consensus_var(const float4 *__restrict__ XP, int nP,
                                                              const float4 *__restrict__ NP, const GridParams *gp,
                                                              const int *__restrict__ start,
                                                              const float4 *__restrict__ Xs,
                                                              const float4 *__restrict__ NQ, int nQ,
                                                              const float *__restrict__ pose,
                                                              const uint8_t *__restrict__ ok, const int *n_dev,
                                                              float eps2, float cos_normal, int *count,
                                                              unsigned long long *sum) {
  constexpr int GPB = kNnThreads / G;
  const GridParams g = *gp;
  const int nh = *n_dev;
  const int chunks = (nP + kVarChunk - 1) / kVarChunk;
  const int64_t items = (int64_t)nh * chunks;
  const int grp = threadIdx.x / G, sub = threadIdx.x & (G - 1);
  __shared__ int s_cnt[kNnThreads / 32];
  __shared__ unsigned long long s_sum[kNnThreads / 32];
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int s = (int)(item / chunks), c = (int)(item - (int64_t)s * chunks);
    if (ok && !ok[s]) continue;
    Rigid12 T;
    T.load(pose + (size_t)s * 12);
    int cnt = 0;
    unsigned long long acc = 0ull;
    const int i0 = c * kVarChunk, i1 = min(nP, (c + 1) * kVarChunk);
    for (int r = i0; r < i1; r += GPB) {  // block-uniform trip count
      const int i = r + grp;
      const bool valid = i < i1;
      const float4 p = valid ? XP[i] : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
      float x, y, z;
      T.apply(p, x, y, z);
      float best;
      int bt;
      if (kSingle) {
        bt = single_cell_nn(g, start, Xs, x, y, z, best);
      } else {
        int bidx;
        group_nn<G>(g, start, Xs, x, y, z, eps2, best, bt, bidx);
      }
      if (!valid || sub != 0 || bt < 0 || !(best < eps2)) continue;
      if (kNormals) {
        const int ip = __float_as_int(p.w), iq = __float_as_int(Xs[bt].w);
        if (!LSR_IN_BOUNDS(ip, nP, kSiteGridPoint) || !LSR_IN_BOUNDS(iq, nQ, kSiteGridPoint)) continue;
        const float4 np = NP[ip], nq = NQ[iq];
        if (np.w < 0.f || nq.w < 0.f) continue;
        const float rx = fmaf(T.r0, np.x, fmaf(T.r1, np.y, T.r2 * np.z));
        const float ry = fmaf(T.r3, np.x, fmaf(T.r4, np.y, T.r5 * np.z));
        const float rz = fmaf(T.r6, np.x, fmaf(T.r7, np.y, T.r8 * np.z));
        if (!(fmaf(rx, nq.x, fmaf(ry, nq.y, rz * nq.z)) >= cos_normal)) continue;
      }
      ++cnt;
      acc += (unsigned long long)__double2ll_rn((double)best * kFixScale);
    }
    cnt = warp_sum(cnt);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_cnt[w] = cnt, s_sum[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tc = 0;
      unsigned long long ts = 0ull;
      for (int k = 0; k < kNnThreads / 32; ++k) tc += s_cnt[k], ts += s_sum[k];
      if (tc) {
        atomicAdd(&count[s], tc);
        atomicAdd(&sum[s], ts);
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_cell_grid_params(const float *box, float cell, int npts, int cap_cells, GridParams *g,
                                    cudaStream_t s) {
  LSR_LAUNCH(k_cell_grid_params<<<1, 32, 0, s>>>(box, cell, npts, cap_cells, g));
  return cudaGetLastError();
}

cudaError_t launch_nn_stage(const float *X, int nX, const GridParams *g, const int *start, const float4 *Xs, float r,
                            int single, int *nn, float *d2, cudaStream_t s) {
  int64_t b = lsr_div_up((int64_t)(nX > 0 ? nX : 1) * (single ? 1 : 4), kNnThreads);
  const int nb = (int)(b > kSms * 16 ? kSms * 16 : b);
  if (single)
    LSR_LAUNCH(k_nn_stage<1><<<nb, kNnThreads, 0, s>>>(X, nX, g, start, Xs, r * r, 1, nn, d2));
  else
    LSR_LAUNCH(k_nn_stage<4><<<nb, kNnThreads, 0, s>>>(X, nX, g, start, Xs, r * r, 0, nn, d2));
  return cudaGetLastError();
}

cudaError_t launch_consensus_variant(const float4 *XP, int nP, const float4 *NP, const GridParams *g,
                                     const int *start, const float4 *Xs, const float4 *NQ, int nQ, const float *pose,
                                     const uint8_t *ok, const int *n_dev, float eps, bool single, bool normals,
                                     float cos_normal, int *count, unsigned long long *sum, cudaStream_t s) {
  const float e2 = eps * eps;
#define LSR_VAR(G, S, N)                                                                                     \
  LSR_LAUNCH(k_consensus_var<G, S, N><<<kSms * 8, kNnThreads, 0, s>>>(XP, nP, NP, g, start, Xs, NQ, nQ, pose, ok, \
                                                                      n_dev, e2, cos_normal, count, sum))
  if (single && normals)
    LSR_VAR(1, true, true);
  else if (single)
    LSR_VAR(1, true, false);
  else if (normals)
    LSR_VAR(4, false, true);
  else
    LSR_VAR(4, false, false);
#undef LSR_VAR
  return cudaGetLastError();
}

LSR_CHECK_READER(nn)

}  // namespace lsr
