// lsr_refine.cu -- robust pose refinement and the robust alignment objective.
//
// The cost is the line-process objective of eq. (3)-(4) with the line process
// eliminated: for a residual r, min_l l r^2 + mu (sqrt(l) - 1)^2 is reached at
// l* = (mu / (mu + r^2))^2 and equals the Geman-McClure rho(r^2) = mu r^2 /
// (mu + r^2). Refinement iterates reweighted Gauss-Newton with the Jacobian
// G_p = [-[p]_x | I] of eq. (5), taken about a linearisation centre c (the
// weighted centroid of the current correspondences, so that FP32 stays exact
// to the micrometre whatever the clouds' offset): FP32 per-thread and
// per-block sums, then one launch-closing block sums the block partials in
// FP64 in a fixed order, solves the 6x6 system (Schur complement of its
// translation block, then a 3x3 adjugate) and updates the
// FP64 pose -- one kernel launch per iteration, no host round trip.
#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kRefThreads = 256;
constexpr int kRefG = 4;   // lanes per nearest-neighbour query in refinement (4 measured fastest of 4/8/16)
constexpr int kRefBlocksPerSm = 4;  // resident refinement blocks per SM (64 registers a thread; 3 measured slower)
constexpr int kRefMaxBlocks = kSms * kRefBlocksPerSm;  // refine_blocks' cap
constexpr int kRefGroup = 16;                           // blocks per first-level closing sum
constexpr int kRefMaxGroups = (kRefMaxBlocks + kRefGroup - 1) / kRefGroup;
constexpr int kObjG = 8;   // lanes per query in the objective
// 21 (upper triangle of A) + 6 (b) + count + sum w + sum w x (3)
constexpr int kNAcc = kRefAcc;
static_assert(kNAcc == 32, "refinement partial layout");

template <int N>
__device__ __forceinline__ void block_reduce_to(float (&v)[N], double *out) {
  __shared__ float sm[kRefThreads / 32][N];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) sm[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x < N) {
    double s = 0.0;
    for (int k = 0; k < kRefThreads / 32; ++k) s += (double)sm[k][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// Per-step sums of the IRLS normal equations. With J = [-[xc]_x | I] (xc the
// moved point about the step's centre c), w the line-process weight of eq. (4)
// and r the residual, J^T W J and J^T W r need only these 17 sums:
//   [0] count  [1] sum w  [2..4] sum w xc  [5..10] sum w xc_a xc_b (00 01 02 11 12 22)
//   [11..16] b = sum w J^T r = (sum w xc x r, sum w r)
constexpr int kNSum = 17;
static_assert(kNSum <= kNAcc, "refinement partial layout");

// The state one step reads, copied to shared memory by the closing block
// while it sums the partials (its loads then overlap instead of queueing
// behind each other in the single solving thread).
struct StepState {
  double T[12];
  double center[3];
  int iters_done;
  int level_iters;
};

// 1 / x in FP64 for a positive x: the FP32 reciprocal refined by two Newton-
// Raphson steps r <- r + r (1 - x r) (each doubles the correct bits: 24 ->
// 48 -> 96, so the result is within an ulp of 1 / x); outside the FP32 range
// the FP64 division. A division costs far more FP64 latency on this part
// than the four fused multiply-adds.
__device__ __forceinline__ double recip_pos(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// Solve A d = -b in FP64 from the summed partials and left-multiply the pose
// by the update about the centre c used for this step: x' = Exp(d_w)(x - c) +
// c + d_v. The next step's centre is the weighted centroid of this step's
// correspondences. Reads the state from ss, writes it to st.
//
// With J = [-[xc]_x | I], A = [[M, [s]_x], [[s]_x^T, sw I]] where M is the
// rotation block, s = sum w xc and sw = sum w. The translation block is a
// multiple of I, so it is eliminated in closed form (Schur complement):
//   M' = M - [s]_x [s]_x^T / sw = M - (|s|^2 I - s s^T) / sw,
//   M' d_w = -b_w + (s x b_v) / sw,   d_v = -(b_v - s x d_w) / sw,
// and the 3x3 system is solved by its adjugate (one reciprocal). A is
// positive definite iff sw > 0 and M' is (its leading minors m00, m00 m11 -
// m01^2 and det M' positive). This is the same solution as a 6x6 Cholesky in
// exact arithmetic with a far shorter chain of dependent FP64 operations,
// whose latency is long on this part.
//
// Run by warps 0 and 1 of the closing block (every thread of the block
// reaches its barrier): the solve, the Exp coefficients and the twelve pose
// entries (lanes 0..11) on warp 0; the next centre on warp 1 meanwhile, and
// the step length and the state on warp 1 after the pose. Each value is
// computed by one lane in a fixed order, so the result is deterministic.
__device__ void refine_solve(const double *S, const StepState &ss, RansacState *st, int max_iters, double tol) {
  __shared__ double sd[6], scoef[2], scn[3];
  __shared__ int spd;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double *xx = S + 5, *b = S + 11;
  const double sw = S[1], sx0 = S[2], sx1 = S[3], sx2 = S[4];
  bool pd = S[0] >= 3.0 && sw > 0.0;
  if (warp == 1 && lane == 0 && sw > 0.0) {
    const double iw = recip_pos(sw);
    const double *c = ss.center;
    scn[0] = c[0] + sx0 * iw, scn[1] = c[1] + sx1 * iw, scn[2] = c[2] + sx2 * iw;
  }
  if (warp == 0) {
    if (lane == 0 && pd) {
      const double iw = recip_pos(sw);
      const double ss2 = sx0 * sx0 + sx1 * sx1 + sx2 * sx2;
      // M' (symmetric; M from the weighted second moments of xc)
      const double m00 = xx[3] + xx[5] - (ss2 - sx0 * sx0) * iw;
      const double m11 = xx[0] + xx[5] - (ss2 - sx1 * sx1) * iw;
      const double m22 = xx[0] + xx[3] - (ss2 - sx2 * sx2) * iw;
      const double m01 = -xx[1] + sx0 * sx1 * iw;
      const double m02 = -xx[2] + sx0 * sx2 * iw;
      const double m12 = -xx[4] + sx1 * sx2 * iw;
      // right-hand side -b_w + (s x b_v) / sw
      const double r0 = -b[0] + (sx1 * b[5] - sx2 * b[4]) * iw;
      const double r1 = -b[1] + (sx2 * b[3] - sx0 * b[5]) * iw;
      const double r2 = -b[2] + (sx0 * b[4] - sx1 * b[3]) * iw;
      // adjugate (cofactors) and determinant
      const double c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
      const double c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
      const double det = m00 * c00 + m01 * c01 + m02 * c02;
      pd = m00 > 0.0 && c22 > 0.0 && det > 0.0;
      if (pd) {
        const double idet = recip_pos(det);
        const double w0 = (c00 * r0 + c01 * r1 + c02 * r2) * idet;
        const double w1 = (c01 * r0 + c11 * r1 + c12 * r2) * idet;
        const double w2 = (c02 * r0 + c12 * r1 + c22 * r2) * idet;
        sd[0] = w0, sd[1] = w1, sd[2] = w2;
        // d_v = -(b_v - s x d_w) / sw
        sd[3] = -(b[3] - (sx1 * w2 - sx2 * w1)) * iw;
        sd[4] = -(b[4] - (sx2 * w0 - sx0 * w2)) * iw;
        sd[5] = -(b[5] - (sx0 * w1 - sx1 * w0)) * iw;
      }
    }
    pd = __shfl_sync(0xffffffffu, pd, 0);
    __syncwarp();
    if (pd && lane == 0) {
      // Exp of the rotation part: the series of sin(t)/t and (1 - cos t)/t^2 to
      // the t^8 term below t = 0.01 (the next term is below 1e-21; the
      // coefficients' reciprocals are FP64 constants), else sin/cos
      const double th2 = sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2];
      if (th2 < 1e-4) {
        scoef[0] = 1.0 - th2 * (1.0 / 6.0) * (1.0 - th2 * (1.0 / 20.0) * (1.0 - th2 * (1.0 / 42.0) * (1.0 - th2 * (1.0 / 72.0))));
        scoef[1] = 0.5 * (1.0 - th2 * (1.0 / 12.0) * (1.0 - th2 * (1.0 / 30.0) * (1.0 - th2 * (1.0 / 56.0) * (1.0 - th2 * (1.0 / 90.0)))));
      } else {
        const double th = sqrt(th2);
        scoef[0] = sin(th) / th;
        scoef[1] = (1.0 - cos(th)) / th2;
      }
    }
    if (lane == 0) spd = pd;
    __syncwarp();
  }
  __syncthreads();  // spd, sd, scoef (warp 0) and scn (warp 1)
  pd = spd != 0;
  if (warp == 1 && lane == 0) {
    if (!pd) {
      st->active = 0;
      return;
    }
    if (sw > 0.0)
      for (int r = 0; r < 3; ++r) st->center[r] = scn[r];
    double nd2 = 0.0;
    for (int i = 0; i < 6; ++i) nd2 += sd[i] * sd[i];
    st->last_step = sqrt(nd2);
    st->iters_done = ss.iters_done + 1;
    st->level_iters = ss.level_iters + 1;
    if (nd2 < tol * tol || ss.level_iters + 1 >= max_iters) st->active = 0;
  }
  if (warp != 0 || !pd) return;
  if (lane < 12) {
    // pose entry (r, q): row r of Rd (its three entries), then row r of Rd T
    const int r = lane >> 2, q = lane & 3;
    const double *d = sd;
    const double a = scoef[0], bb = scoef[1];
    const double K[9] = {0, -d[2], d[1], d[2], 0, -d[0], -d[1], d[0], 0};
    double Rd[3];
    for (int cc = 0; cc < 3; ++cc) {
      const double k2 = K[3 * r] * K[cc] + K[3 * r + 1] * K[3 + cc] + K[3 * r + 2] * K[6 + cc];
      Rd[cc] = (r == cc ? 1.0 : 0.0) + a * K[3 * r + cc] + bb * k2;
    }
    const double *c = ss.center;
    const double vr = c[r] - (Rd[0] * c[0] + Rd[1] * c[1] + Rd[2] * c[2]) + d[3 + r];
    st->T[lane] = Rd[0] * ss.T[q] + Rd[1] * ss.T[4 + q] + Rd[2] * ss.T[8 + q] + (q == 3 ? vr : 0.0);
  }
}

// One IRLS step. Every block accumulates its points; the last block to
// finish (atomic ticket, no waiting) sums all block partials and solves.
__global__ void __launch_bounds__(kRefThreads, kRefBlocksPerSm) k_refine_step(const float4 *__restrict__ XP, int nP, int strideP,
                                                             const GridParams *gep, const int *__restrict__ start,
                                                             const float4 *__restrict__ Xe, float eps2, float mu,
                                                             RansacState *st, double *partials, int max_iters,
                                                             double tol, int *__restrict__ seeds) {
  __shared__ int s_last;
  __shared__ double tot[kNSum];
  // the next step may be scheduled now (launched as a programmatic dependent,
  // it waits below for this one to finish); this step reads the pose, the
  // state and the seeds the previous step wrote
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (!st->active) return;
  const GridParams g = *gep;
  const double *T = st->T;
  float R[9], tc[3], c[3];
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) R[3 * r + k] = (float)T[4 * r + k];
    c[r] = (float)st->center[r];
    tc[r] = (float)(T[4 * r + 3] - st->center[r]);
  }
  constexpr int G = kRefG, GPB = kRefThreads / G;
  const int grp = threadIdx.x / G, sub = threadIdx.x & (G - 1);
  float acc[kNSum];
#pragma unroll
  for (int u = 0; u < kNSum; ++u) acc[u] = 0.f;
  // block-uniform trip count: every lane reaches the group shuffles
  for (int r0 = blockIdx.x * GPB; r0 < nP; r0 += gridDim.x * GPB) {
    int i = r0 + grp;
    bool valid = i < nP;
    float4 p = valid ? XP[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid && strideP > 1 && __float_as_int(p.w) % strideP != 0) valid = false;
    if (!valid) p.x = __int_as_float(0x7fc00000);  // NaN: the query visits no cell
    const float xc0 = fmaf(R[0], p.x, fmaf(R[1], p.y, fmaf(R[2], p.z, tc[0])));
    const float xc1 = fmaf(R[3], p.x, fmaf(R[4], p.y, fmaf(R[5], p.z, tc[1])));
    const float xc2 = fmaf(R[6], p.x, fmaf(R[7], p.y, fmaf(R[8], p.z, tc[2])));
    const float x = xc0 + c[0], y = xc1 + c[1], z = xc2 + c[2];
    float best;
    int bt, bidx;
    // the previous step's neighbour of this point starts the search (an exact
    // search either way)
    const int seed = valid ? seeds[i] : -1;
    group_nn<G>(g, start, Xe, x, y, z, eps2, best, bt, bidx, seed);
    if (valid && sub == 0) seeds[i] = bt;
    if (!valid || bt < 0 || sub != 0) continue;
    const float4 q = Xe[bt];
    const float e0 = x - q.x, e1 = y - q.y, e2 = z - q.z;  // the residual
    const float s = e0 * e0 + e1 * e1 + e2 * e2;
    const float l = mu / (mu + s);
    const float w = l * l;
    const float w0 = w * xc0, w1 = w * xc1, w2 = w * xc2;
    acc[0] += 1.f;
    acc[1] += w;
    acc[2] += w0, acc[3] += w1, acc[4] += w2;
    acc[5] += w0 * xc0, acc[6] += w0 * xc1, acc[7] += w0 * xc2;
    acc[8] += w1 * xc1, acc[9] += w1 * xc2, acc[10] += w2 * xc2;
    acc[11] += w * (xc1 * e2 - xc2 * e1);
    acc[12] += w * (xc2 * e0 - xc0 * e2);
    acc[13] += w * (xc0 * e1 - xc1 * e0);
    acc[14] += w * e0, acc[15] += w * e1, acc[16] += w * e2;
  }
  {
    __shared__ float sm[kRefThreads / 32][kNSum];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int u = 0; u < kNSum; ++u) {
      const float v = warp_sum(acc[u]);
      if (lane == 0) sm[wp][u] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNSum) {
      double t = 0.0;
      for (int k = 0; k < kRefThreads / 32; ++k) t += (double)sm[k][threadIdx.x];
      partials[(size_t)blockIdx.x * kNAcc + threadIdx.x] = t;
    }
  }
  // Two-level close: the last block of each group of kRefGroup blocks sums its
  // group's partials in block order; the last group to close sums the group
  // sums and solves (fewer dependent loads on the closing path).
  double *gpart = partials + (size_t)kRefMaxBlocks * kNAcc;
  unsigned *gticket = reinterpret_cast<unsigned *>(gpart + (size_t)kRefMaxGroups * kNAcc);
  const unsigned cgrp = blockIdx.x / kRefGroup, ng = (gridDim.x + kRefGroup - 1) / kRefGroup;
  const unsigned g0 = cgrp * kRefGroup, gsz = min((unsigned)kRefGroup, gridDim.x - g0);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(gticket + cgrp, 1u) == gsz - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < kNSum) {
    double v[kRefGroup];
#pragma unroll
    for (int u = 0; u < kRefGroup; ++u)
      v[u] = (unsigned)u < gsz ? __ldcg(partials + (size_t)(g0 + u) * kNAcc + threadIdx.x) : 0.0;
    double t = 0.0;
#pragma unroll
    for (int u = 0; u < kRefGroup; ++u) t += v[u];
    gpart[(size_t)cgrp * kNAcc + threadIdx.x] = t;
  }
  if (threadIdx.x == 0) gticket[cgrp] = 0u;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->ticket, 1u) == ng - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ StepState ss;
  if (threadIdx.x < 12) ss.T[threadIdx.x] = __ldcg(st->T + threadIdx.x);
  else if (threadIdx.x < 15) ss.center[threadIdx.x - 12] = __ldcg(st->center + threadIdx.x - 12);
  else if (threadIdx.x == 15) ss.iters_done = __ldcg(&st->iters_done);
  else if (threadIdx.x == 16) ss.level_iters = __ldcg(&st->level_iters);
  {
    // sum k = t % 17 over the groups t / 17, t / 17 + 15, ..., then the 15
    // segments in order (a fixed order: the sums are deterministic)
    constexpr int kSeg = kRefThreads / kNSum;
    __shared__ double seg[kSeg][kNSum];
    const int k = threadIdx.x % kNSum, sg = threadIdx.x / kNSum;
    if (sg < kSeg) {
      double sum = 0.0;
      for (unsigned b = sg; b < ng; b += kSeg) sum += __ldcg(gpart + (size_t)b * kNAcc + k);
      seg[sg][k] = sum;
    }
    __syncthreads();
    if (threadIdx.x < kNSum) {
      double t = 0.0;
      for (int q = 0; q < kSeg; ++q) t += seg[q][threadIdx.x];
      tot[threadIdx.x] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) st->ticket = 0u;
  refine_solve(tot, ss, st, max_iters, tol);
}

__global__ void k_refine_level_begin(RansacState *st) {
  if (threadIdx.x == 0) {
    st->active = st->status == 0 ? 1 : 0;
    st->level_iters = 0;
    st->ticket = 0u;
  }
}

__global__ void k_subsample(const float *xyz, int n, int stride, float4 *out) {
  int m_n = (n + stride - 1) / stride;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < m_n; m += gridDim.x * blockDim.x) {
    int i = m * stride;
    out[m] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __int_as_float(m));
  }
}

// Starting pose (T_in, or the selected hypothesis already in st) and the
// first linearisation centre: the centroid of P moved by that pose.
__global__ void k_refine_init(RansacState *st, const float *boxP, const double *T_in) {
  if (threadIdx.x != 0) return;
  if (T_in) {
    for (int i = 0; i < 16; ++i) st->T[i] = st->T_hyp[i] = T_in[i];
    st->active = 1;
    st->status = 0;
    st->iters_done = 0;
  }
  const double *T = st->T;
  double m[3] = {boxP[8], boxP[9], boxP[10]};
  for (int r = 0; r < 3; ++r) st->center[r] = T[4 * r] * m[0] + T[4 * r + 1] * m[1] + T[4 * r + 2] * m[2] + T[4 * r + 3];
  st->ticket = 0u;
}

__global__ void k_final_pose(const RansacState *st, float *pose) {
  if (threadIdx.x < 12) {
    int r = threadIdx.x / 4, c = threadIdx.x % 4;
    pose[threadIdx.x] = (float)st->T[4 * r + c];
  }
}

__global__ void k_final_count(const int *count, const unsigned long long *sum, RansacState *st) {
  if (threadIdx.x == 0) {
    st->final_count = count[0];
    st->final_sumd2 = (double)sum[0] / kFixScale;
  }
}

// ---------------------------------------------------------------- information matrix
// Loop verification (eq. (5)-(6)): Lambda = sum over K of G_p^T G_p with
// G_p = [-[p]_x | I], K the moved points p = R p' + t whose nearest Q point
// lies within eps. Written out, G_p^T G_p = [[|p|^2 I - p p^T, [p]_x],
// [-[p]_x, I]], so Lambda needs only |K|, sum p and sum p p^T. Each group of
// kRefG lanes searches one point; its first lane adds 1, d and d d^T with
// d = p - c (c: the centre of Q's box, which keeps the FP32 sums small) to ten
// per-thread sums; blocks reduce them to FP64 partials, and one thread adds
// the partials in block order and expands them about c.
struct InfoArgs {
  float R[9], t[3];
  float eps2;
};

__global__ void __launch_bounds__(kRefThreads) k_info_sums(const float *__restrict__ P, int nP, const GridParams *gep,
                                                           const int *__restrict__ start, const float4 *__restrict__ Xe,
                                                           const float *__restrict__ boxQ, InfoArgs a,
                                                           double *__restrict__ partials) {
  constexpr int G = kRefG, GPB = kRefThreads / G;
  const GridParams g = *gep;
  const float c0 = 0.5f * (boxQ[0] + boxQ[3]), c1 = 0.5f * (boxQ[1] + boxQ[4]), c2 = 0.5f * (boxQ[2] + boxQ[5]);
  const int grp = threadIdx.x / G, sub = threadIdx.x & (G - 1);
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  // block-uniform trip count: every lane reaches the group shuffles
  for (int r0 = blockIdx.x * GPB; r0 < nP; r0 += gridDim.x * GPB) {
    const int i = r0 + grp;
    const bool valid = i < nP;
    float px = valid ? P[3 * i] : __int_as_float(0x7fc00000), py = valid ? P[3 * i + 1] : 0.f,
          pz = valid ? P[3 * i + 2] : 0.f;  // NaN: the query visits no cell
    const float x = fmaf(a.R[0], px, fmaf(a.R[1], py, fmaf(a.R[2], pz, a.t[0])));
    const float y = fmaf(a.R[3], px, fmaf(a.R[4], py, fmaf(a.R[5], pz, a.t[1])));
    const float z = fmaf(a.R[6], px, fmaf(a.R[7], py, fmaf(a.R[8], pz, a.t[2])));
    float best;
    int bt, bidx;
    group_nn<G>(g, start, Xe, x, y, z, a.eps2, best, bt, bidx);
    if (!valid || bt < 0 || sub != 0) continue;
    const float dx = x - c0, dy = y - c1, dz = z - c2;
    acc[0] += 1.f;
    acc[1] += dx, acc[2] += dy, acc[3] += dz;
    acc[4] += dx * dx, acc[5] += dx * dy, acc[6] += dx * dz;
    acc[7] += dy * dy, acc[8] += dy * dz, acc[9] += dz * dz;
  }
  block_reduce_to<10>(acc, partials + (size_t)blockIdx.x * 10);
}

__global__ void k_info_final(const double *__restrict__ partials, int nb, const float *__restrict__ boxQ,
                             double *__restrict__ out) {
  __shared__ double seg[256], tot[10];
  block_sum_partials(partials, nb, 10, 10, seg, tot);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double S[10];
  for (int k = 0; k < 10; ++k) S[k] = tot[k];
  const double c[3] = {0.5 * ((double)boxQ[0] + (double)boxQ[3]), 0.5 * ((double)boxQ[1] + (double)boxQ[4]),
                       0.5 * ((double)boxQ[2] + (double)boxQ[5])};
  const double n = S[0];
  // sum p = sum d + n c; sum p p^T = sum d d^T + c (sum d)^T + (sum d) c^T + n c c^T
  double sp[3], spp[3][3];
  const double sdd[3][3] = {{S[4], S[5], S[6]}, {S[5], S[7], S[8]}, {S[6], S[8], S[9]}};
  for (int r = 0; r < 3; ++r) sp[r] = S[1 + r] + n * c[r];
  for (int r = 0; r < 3; ++r)
    for (int q = r; q < 3; ++q)  // upper triangle, mirrored: Lambda is exactly symmetric
      spp[r][q] = spp[q][r] = sdd[r][q] + c[r] * S[1 + q] + S[1 + r] * c[q] + n * c[r] * c[q];
  const double tr = spp[0][0] + spp[1][1] + spp[2][2];
  // [sp]_x
  const double K[3][3] = {{0.0, -sp[2], sp[1]}, {sp[2], 0.0, -sp[0]}, {-sp[1], sp[0], 0.0}};
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      out[6 * r + q] = (r == q ? tr : 0.0) - spp[r][q];
      out[6 * r + 3 + q] = K[r][q];
      out[6 * (3 + r) + q] = -K[r][q];
      out[6 * (3 + r) + 3 + q] = r == q ? n : 0.0;
    }
  out[36] = n;
}

// ---------------------------------------------------------------- objective
// E = sum_i rho(s_i) - rho(eps^2) over points with an NN closer than eps.
// Forward and backward share this kernel; the backward also writes
// dP_i = 2 rho'(s) R^T r_i, scatters dQ_j -= 2 rho'(s) r_i, and reduces
// g_v = sum 2 rho' r_i and g_w = sum z_i x (2 rho' r_i) with z_i = x_i - v.
// dxi = (J_l(w)^T g_w, g_v) is finished on the host. The nearest neighbour is
// found in FP32 (the pose rounded to FP32); the residual of the pair, the
// terms and their sums are evaluated in FP64 from the FP32 coordinates: a
// residual of a few millimetres between points metres from the origin would
// otherwise carry the 2^-24 rounding of the coordinates (about 1e-7 m).
struct ObjArgs {
  float Rf[9], tf[3];    // the pose in FP32, for the neighbour search
  double R[9], t[3], v[3];
  float eps2;
  double mu, rho_eps, scale;
};

__device__ __forceinline__ double warp_sum_dbl(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(kRefThreads) k_objective(const float *__restrict__ P, int nP, const GridParams *gep,
                                                           const int *__restrict__ start,
                                                           const float4 *__restrict__ Xe, ObjArgs a, int want_grad,
                                                           double *partials, float *__restrict__ dP,
                                                           float *__restrict__ dQ) {
  const GridParams g = *gep;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};  // E, g_v (3), g_w (3)
  constexpr int G = kObjG, GPB = kRefThreads / G;
  int grp = threadIdx.x / G, sub = threadIdx.x & (G - 1);
  for (int rb = blockIdx.x * GPB; rb < nP; rb += gridDim.x * GPB) {
    int i = rb + grp;
    bool valid = i < nP;
    float px = valid ? P[3 * i] : __int_as_float(0x7fc00000), py = valid ? P[3 * i + 1] : 0.f,
          pz = valid ? P[3 * i + 2] : 0.f;
    float x = fmaf(a.Rf[0], px, fmaf(a.Rf[1], py, fmaf(a.Rf[2], pz, a.tf[0])));
    float y = fmaf(a.Rf[3], px, fmaf(a.Rf[4], py, fmaf(a.Rf[5], pz, a.tf[1])));
    float z = fmaf(a.Rf[6], px, fmaf(a.Rf[7], py, fmaf(a.Rf[8], pz, a.tf[2])));
    float best;
    int bt, bidx;
    group_nn<G>(g, start, Xe, x, y, z, a.eps2, best, bt, bidx);
    if (!valid || sub != 0) continue;
    if (bt < 0) {
      if (want_grad) dP[3 * i] = dP[3 * i + 1] = dP[3 * i + 2] = 0.f;
      continue;
    }
    const float4 q = Xe[bt];
    const double p[3] = {px, py, pz};
    double zd[3], r[3];
    for (int k = 0; k < 3; ++k) {
      zd[k] = a.R[3 * k] * p[0] + a.R[3 * k + 1] * p[1] + a.R[3 * k + 2] * p[2] + a.t[k];
      r[k] = zd[k] - (double)(k == 0 ? q.x : (k == 1 ? q.y : q.z));
    }
    const double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double den = a.mu + s;
    acc[0] += a.mu * s / den - a.rho_eps;
    if (want_grad) {
      const double k2 = 2.0 * a.mu * a.mu / (den * den);
      const double g0 = k2 * r[0], g1 = k2 * r[1], g2 = k2 * r[2];
      dP[3 * i + 0] = (float)(a.scale * (a.R[0] * g0 + a.R[3] * g1 + a.R[6] * g2));
      dP[3 * i + 1] = (float)(a.scale * (a.R[1] * g0 + a.R[4] * g1 + a.R[7] * g2));
      dP[3 * i + 2] = (float)(a.scale * (a.R[2] * g0 + a.R[5] * g1 + a.R[8] * g2));
      const int j = __float_as_int(q.w);
      atomicAdd(&dQ[3 * j + 0], (float)(-a.scale * g0));
      atomicAdd(&dQ[3 * j + 1], (float)(-a.scale * g1));
      atomicAdd(&dQ[3 * j + 2], (float)(-a.scale * g2));
      const double zx = zd[0] - a.v[0], zy = zd[1] - a.v[1], zz = zd[2] - a.v[2];
      acc[1] += g0, acc[2] += g1, acc[3] += g2;
      acc[4] += zy * g2 - zz * g1;
      acc[5] += zz * g0 - zx * g2;
      acc[6] += zx * g1 - zy * g0;
    }
  }
  __shared__ double sm[kRefThreads / 32][7];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double v = warp_sum_dbl(acc[k]);
    if (lane == 0) sm[wp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double t = 0.0;
    for (int k = 0; k < kRefThreads / 32; ++k) t += sm[k][threadIdx.x];
    partials[(size_t)blockIdx.x * 7 + threadIdx.x] = t;
  }
}

__global__ void k_objective_sum(const double *partials, int nblocks, double *out) {
  __shared__ double seg[256], tot[7];
  block_sum_partials(partials, nblocks, 7, 7, seg, tot);
  if (threadIdx.x < 7) out[threadIdx.x] = tot[threadIdx.x];
}

}  // namespace

// One query per group of kRefG lanes per round; at most two blocks per SM so
// that the launch-closing block sums few partials.
int64_t refine_partial_doubles() { return (int64_t)kNAcc * (kRefMaxBlocks + kRefMaxGroups) + kRefMaxGroups; }

cudaError_t refine_reset_tickets(double *partials, cudaStream_t s) {
  return cudaMemsetAsync(partials + (size_t)kNAcc * (kRefMaxBlocks + kRefMaxGroups), 0,
                         sizeof(unsigned) * kRefMaxGroups, s);
}

int refine_blocks(int nP) {
  int64_t b = lsr_div_up((int64_t)(nP > 0 ? nP : 1) * kRefG, kRefThreads);
  return (int)(b < 1 ? 1 : (b > kSms * kRefBlocksPerSm ? kSms * kRefBlocksPerSm : b));  // all blocks resident
}

int gnc_stride(int64_t n, int level, int levels) {
  int64_t f = 1;
  for (int k = 0; k < levels - 1 - level; ++k) f *= 4;
  int64_t cap = n / 4096;
  if (f > cap) f = cap;
  return (int)(f < 1 ? 1 : f);
}

cudaError_t launch_refine_init(RansacState *st, const float *boxP, const double *T_in, cudaStream_t s) {
  LSR_LAUNCH(k_refine_init<<<1, 32, 0, s>>>(st, boxP, T_in));
  return cudaGetLastError();
}

cudaError_t launch_refine_level_begin(RansacState *st, cudaStream_t s) {
  LSR_LAUNCH(k_refine_level_begin<<<1, 32, 0, s>>>(st));
  return cudaGetLastError();
}

cudaError_t launch_subsample(const float *xyz, int n, int stride, float4 *out, cudaStream_t s) {
  int m = (n + stride - 1) / stride;
  int b = (int)lsr_div_up(m > 0 ? m : 1, 256);
  LSR_LAUNCH(k_subsample<<<b < 4096 ? b : 4096, 256, 0, s>>>(xyz, n, stride, out));
  return cudaGetLastError();
}

cudaError_t launch_refine_step(const float4 *XP, int nP, int strideP, const GridParams *ge, const int *start_e,
                               const float4 *Xe, float eps_r, float mu, int max_iters, RansacState *st,
                               double *partials, int *seeds, bool chained, cudaStream_t s) {
  int nb = refine_blocks((int)lsr_div_up(nP, strideP));
  if (chained) {
    // directly after the previous step: scheduled while it closes
    cudaError_t e = cudaSuccess;
    LSR_LAUNCH(e = pdl_launch(k_refine_step, dim3(nb), dim3(kRefThreads), s, XP, nP, strideP, ge, start_e, Xe,
                              eps_r * eps_r, mu, st, partials, max_iters, 1e-6, seeds));
    LSR_CUDA_TRY(e);
  } else {
    LSR_LAUNCH(k_refine_step<<<nb, kRefThreads, 0, s>>>(XP, nP, strideP, ge, start_e, Xe, eps_r * eps_r, mu, st,
                                                        partials, max_iters, 1e-6, seeds));
  }
  return cudaGetLastError();
}

cudaError_t launch_final_pose(RansacState *st, float *pose, cudaStream_t s) {
  LSR_LAUNCH(k_final_pose<<<1, 32, 0, s>>>(st, pose));
  return cudaGetLastError();
}

cudaError_t launch_final_count(const int *count, const unsigned long long *sum, RansacState *st, cudaStream_t s) {
  LSR_LAUNCH(k_final_count<<<1, 32, 0, s>>>(count, sum, st));
  return cudaGetLastError();
}

int information_blocks(int nP) {
  int64_t b = lsr_div_up((int64_t)(nP > 0 ? nP : 1) * kRefG, kRefThreads);
  return (int)(b < 1 ? 1 : (b > kSms * 4 ? kSms * 4 : b));
}

cudaError_t launch_information(const float *P, int nP, const GridParams *ge, const int *start_e, const float4 *Xe,
                               const float *boxQ, const float R[9], const float t[3], float eps, double *partials,
                               double *out, cudaStream_t s) {
  InfoArgs a;
  for (int k = 0; k < 9; ++k) a.R[k] = R[k];
  for (int k = 0; k < 3; ++k) a.t[k] = t[k];
  a.eps2 = eps * eps;
  const int nb = information_blocks(nP);
  LSR_LAUNCH(k_info_sums<<<nb, kRefThreads, 0, s>>>(P, nP, ge, start_e, Xe, boxQ, a, partials));
  LSR_LAUNCH(k_info_final<<<1, 256, 0, s>>>(partials, nb, boxQ, out));
  return cudaGetLastError();
}

int objective_blocks(int nP) {
  int64_t b = lsr_div_up((int64_t)(nP > 0 ? nP : 1) * kObjG, kRefThreads);
  return (int)(b < 1 ? 1 : (b > kSms * 2 ? kSms * 2 : b));
}

cudaError_t launch_objective(const float *P, int nP, const GridParams *ge, const int *start_e, const float4 *Xe,
                             const double T[16], const double v[3], float eps, float mu, double scale,
                             int want_grad, double *partials, double *out7, float *dP, float *dQ, cudaStream_t s) {
  ObjArgs a;
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) a.R[3 * r + q] = T[4 * r + q], a.Rf[3 * r + q] = (float)T[4 * r + q];
    a.t[r] = T[4 * r + 3], a.tf[r] = (float)T[4 * r + 3], a.v[r] = v[r];
  }
  a.eps2 = eps * eps;
  a.mu = mu;
  const double e2 = (double)eps * (double)eps;
  a.rho_eps = a.mu * e2 / (a.mu + e2);
  a.scale = scale;
  int nb = objective_blocks(nP);
  LSR_LAUNCH(k_objective<<<nb, kRefThreads, 0, s>>>(P, nP, ge, start_e, Xe, a, want_grad, partials, dP, dQ));
  LSR_LAUNCH(k_objective_sum<<<1, 256, 0, s>>>(partials, nb, out7));
  return cudaGetLastError();
}

LSR_CHECK_READER(refine)

}  // namespace lsr
