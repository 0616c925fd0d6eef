// lsr_ransac.cu -- hypothesis sampling, polygon pre-rejection, stream
// compaction, per-hypothesis rigid transform, consensus on the 3D grid and
// selection (Algorithm 1 of the paper, after the pre-matching cache).
#include <float.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

// ---------------------------------------------------------------- Philox
// Philox-4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies words 0 and 2 by the round multipliers, mixes the high halves
// with words 1 and 3 and the key, and the key is bumped by the Weyl constants.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0, c[1] = lo1, c[2] = n2, c[3] = lo0;
    k0 += W0, k1 += W1;
  }
}

// The 4 caller-order sample indices of hypothesis h: floor(word_k * n / 2^64).
__device__ __forceinline__ void sample4(uint64_t seed, uint64_t pair, uint32_t h, int n, int idx[4]) {
  uint64_t c[4] = {(uint64_t)h, 0ull, 0ull, 0ull};
  philox4x64_10(c, seed, pair);
#pragma unroll
  for (int k = 0; k < 4; ++k) idx[k] = (int)__umul64hi(c[k], (uint64_t)(unsigned)n);
}

__device__ __forceinline__ float d2f(float4 a, float4 b) {
  float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return dx * dx + dy * dy + dz * dz;
}

struct HypIn {
  const float4 *XP;
  const int *invP;
  const float4 *NP;
  int nP;
  const float4 *XQ;
  const float4 *NQ;
  int nQ;
  const int *nn;
  uint64_t seed, pair;
  float tau2;
};

// Pre-rejection test of one hypothesis (Alg. 1): distinct valid samples,
// non-degenerate cyclic edges, and every edge pair within the tau similarity.
__device__ __forceinline__ bool hyp_pass(const HypIn &in, uint32_t h, int ii[4], int jj[4]) {
  int idx[4];
  sample4(in.seed, in.pair, h, in.nP, idx);
  if (idx[0] == idx[1] || idx[0] == idx[2] || idx[0] == idx[3] || idx[1] == idx[2] || idx[1] == idx[3] ||
      idx[2] == idx[3])
    return false;
  float4 p[4], q[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!LSR_IN_BOUNDS(idx[k], in.nP, kSiteHypSample)) return false;
    ii[k] = in.invP[idx[k]];
    if (!LSR_IN_BOUNDS(ii[k], in.nP, kSiteHypSample)) return false;
    if (in.NP[ii[k]].w < 0.f) return false;
    jj[k] = in.nn[ii[k]];
    if (jj[k] < 0 || jj[k] >= in.nQ) return false;
    if (in.NQ[jj[k]].w < 0.f) return false;
    p[k] = in.XP[ii[k]];
    q[k] = in.XQ[jj[k]];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int b = (a + 1) & 3;
    float ep = d2f(p[a], p[b]), eq = d2f(q[a], q[b]);
    if (ep < 1e-12f || eq < 1e-12f) return false;
    if (ep < in.tau2 * eq || eq < in.tau2 * ep) return false;
  }
  return true;
}

constexpr int kHypThreads = 256;
constexpr int kHypIters = 16;
constexpr int kHypPerBlock = kHypThreads * kHypIters;

#ifdef LSR_CHECKED
// Test probe (lsr_debug_inject LSR_INJECT_CHECK): when armed, the first
// thread of the next hypothesis count asks one out-of-range index question of
// the check machinery -- no memory access follows it -- and disarms.
static __device__ int g_check_probe;
#endif

// Survivors of each block of kHypPerBlock hypotheses: counted into
// block_counts and written in increasing hypothesis id (warp ballots and a
// block prefix per iteration) to the block's own region of local
// (kHypPerBlock ints a block), so that one gather after the scan places them
// in order without testing the hypotheses again.
__global__ void __launch_bounds__(kHypThreads) k_hyp_count(HypIn in, int64_t H, int *block_counts, int *local) {
#ifdef LSR_CHECKED
  if (blockIdx.x == 0 && threadIdx.x == 0 && g_check_probe) {
    g_check_probe = 0;
    (void)LSR_IN_BOUNDS(in.nP, in.nP, kSiteProbe);
  }
#endif
  __shared__ int warp_cnt[kHypThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int *mine = local + (size_t)blockIdx.x * kHypPerBlock;
  int pos = 0;
  int64_t base = (int64_t)blockIdx.x * kHypPerBlock;
  for (int it = 0; it < kHypIters; ++it) {
    int64_t h = base + it * kHypThreads + threadIdx.x;
    int ii[4], jj[4];
    const bool ok = h < H && hyp_pass(in, (uint32_t)h, ii, jj);
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) warp_cnt[w] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int k = 0; k < kHypThreads / 32; ++k) {
      const int c = warp_cnt[k];
      before += (k < w) ? c : 0;
      total += c;
    }
    if (ok) mine[pos + before + __popc(m & ((1u << lane) - 1u))] = (int)h;
    pos += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) block_counts[blockIdx.x] = pos;
}

// Block b's survivors from its region of local to their scanned offset.
__global__ void __launch_bounds__(kHypThreads) k_hyp_gather(const int *__restrict__ local,
                                                            const int *__restrict__ block_counts,
                                                            const int *__restrict__ block_offsets, int *surv,
                                                            int cap) {
  const int n = block_counts[blockIdx.x], off = block_offsets[blockIdx.x];
  const int *mine = local + (size_t)blockIdx.x * kHypPerBlock;
  for (int j = threadIdx.x; j < n; j += kHypThreads)
    if (off + j < cap) surv[off + j] = mine[j];
}

__global__ void k_set_int(int *p, int v) {
  if (threadIdx.x == 0) *p = v;
}

__global__ void k_hyp_finish(const int *offsets, int nb, int cap, RansacState *st) {
  if (threadIdx.x == 0) {
    int total = offsets[nb];
    st->n_surv_total = total;
    st->n_surv = total < cap ? total : cap;
  }
}

// ---------------------------------------------------------------- rigid fit
// Horn's closed-form absolute orientation (J. Opt. Soc. Am. A, 1987): the
// rotation is the unit quaternion of the largest eigenvalue of the symmetric
// 4x4 matrix built from the cross-covariance S = sum (p - pm)(q - qm)^T;
// eigenvector by cyclic Jacobi in FP32.
__device__ void horn4(const float3 p[4], const float3 q[4], float R[9], float t[3]) {
  float3 pm = make_float3(0, 0, 0), qm = make_float3(0, 0, 0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    pm.x += p[k].x, pm.y += p[k].y, pm.z += p[k].z;
    qm.x += q[k].x, qm.y += q[k].y, qm.z += q[k].z;
  }
  pm.x *= 0.25f, pm.y *= 0.25f, pm.z *= 0.25f;
  qm.x *= 0.25f, qm.y *= 0.25f, qm.z *= 0.25f;
  float S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float a[3] = {p[k].x - pm.x, p[k].y - pm.y, p[k].z - pm.z};
    float b[3] = {q[k].x - qm.x, q[k].y - qm.y, q[k].z - qm.z};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) S[r][c] += a[r] * b[c];
  }
  float Sxx = S[0][0], Sxy = S[0][1], Sxz = S[0][2], Syx = S[1][0], Syy = S[1][1], Syz = S[1][2], Szx = S[2][0],
        Szy = S[2][1], Szz = S[2][2];
  float A[4][4] = {{Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
                   {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
                   {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
                   {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
  float V[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) V[r][c] = r == c ? 1.f : 0.f;
  for (int sweep = 0; sweep < 10; ++sweep) {
    float off = 0.f, dg = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      dg += A[r][r] * A[r][r];
#pragma unroll
      for (int c = r + 1; c < 4; ++c) off += A[r][c] * A[r][c];
    }
    if (off <= 1e-14f * dg) break;
#pragma unroll
    for (int pp = 0; pp < 3; ++pp)
#pragma unroll
      for (int qq = pp + 1; qq < 4; ++qq) {
        float apq = A[pp][qq];
        if (apq == 0.f) continue;
        float th = (A[qq][qq] - A[pp][pp]) / (2.f * apq);
        float tt = copysignf(1.f, th) / (fabsf(th) + sqrtf(th * th + 1.f));
        float c = rsqrtf(tt * tt + 1.f), s = tt * c;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float akp = A[k][pp], akq = A[k][qq];
          A[k][pp] = c * akp - s * akq;
          A[k][qq] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float apk = A[pp][k], aqk = A[qq][k];
          A[pp][k] = c * apk - s * aqk;
          A[qq][k] = s * apk + c * aqk;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float vkp = V[k][pp], vkq = V[k][qq];
          V[k][pp] = c * vkp - s * vkq;
          V[k][qq] = s * vkp + c * vkq;
        }
      }
  }
  int j = 0;
#pragma unroll
  for (int k = 1; k < 4; ++k)
    if (A[k][k] > A[j][j]) j = k;
  float w = V[0][j], x = V[1][j], y = V[2][j], z = V[3][j];
  float inv = rsqrtf(w * w + x * x + y * y + z * z);
  w *= inv, x *= inv, y *= inv, z *= inv;
  R[0] = 1.f - 2.f * (y * y + z * z), R[1] = 2.f * (x * y - z * w), R[2] = 2.f * (x * z + y * w);
  R[3] = 2.f * (x * y + z * w), R[4] = 1.f - 2.f * (x * x + z * z), R[5] = 2.f * (y * z - x * w);
  R[6] = 2.f * (x * z - y * w), R[7] = 2.f * (y * z + x * w), R[8] = 1.f - 2.f * (x * x + y * y);
  t[0] = qm.x - (R[0] * pm.x + R[1] * pm.y + R[2] * pm.z);
  t[1] = qm.y - (R[3] * pm.x + R[4] * pm.y + R[5] * pm.z);
  t[2] = qm.z - (R[6] * pm.x + R[7] * pm.y + R[8] * pm.z);
}

// Pose of every survivor (Alg. 1, "Estimate transformation") and the normal
// check moved into hypothesis testing (Sec. IV): rejected if any sampled pair
// has cos(R n_p, n_q) < cos_normal.
__global__ void k_rigid_survivors(HypIn in, const int *surv, const RansacState *st, float cos_normal, float *pose,
                                  uint8_t *ok, int *n_ok) {
  int S = st->n_surv;
  int cnt = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    int ii[4], jj[4];
    uint32_t h = (uint32_t)surv[s];
    bool pass = hyp_pass(in, h, ii, jj);  // recomputes the sample; always true for survivors
    float3 p[4], q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 a = in.XP[ii[k]], b = in.XQ[jj[k]];
      p[k] = make_float3(a.x, a.y, a.z);
      q[k] = make_float3(b.x, b.y, b.z);
    }
    float R[9], t[3];
    horn4(p, q, R, t);
    bool good = pass;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 np = in.NP[ii[k]], nq = in.NQ[jj[k]];
      float rx = R[0] * np.x + R[1] * np.y + R[2] * np.z;
      float ry = R[3] * np.x + R[4] * np.y + R[5] * np.z;
      float rz = R[6] * np.x + R[7] * np.y + R[8] * np.z;
      if (rx * nq.x + ry * nq.y + rz * nq.z < cos_normal) good = false;
    }
    float *o = pose + (size_t)s * 12;
    o[0] = R[0], o[1] = R[1], o[2] = R[2], o[3] = t[0];
    o[4] = R[3], o[5] = R[4], o[6] = R[5], o[7] = t[1];
    o[8] = R[6], o[9] = R[7], o[10] = R[8], o[11] = t[2];
    ok[s] = good ? 1 : 0;
    cnt += good;
  }
  cnt = warp_sum(cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_ok, cnt);
}

__global__ void k_rigid4(const float *ps, const float *qs, int nh, float *pose) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nh; s += gridDim.x * blockDim.x) {
    float3 p[4], q[4];
    for (int k = 0; k < 4; ++k) {
      p[k] = make_float3(ps[12 * s + 3 * k], ps[12 * s + 3 * k + 1], ps[12 * s + 3 * k + 2]);
      q[k] = make_float3(qs[12 * s + 3 * k], qs[12 * s + 3 * k + 1], qs[12 * s + 3 * k + 2]);
    }
    float R[9], t[3];
    horn4(p, q, R, t);
    float *o = pose + (size_t)s * 12;
    o[0] = R[0], o[1] = R[1], o[2] = R[2], o[3] = t[0];
    o[4] = R[3], o[5] = R[4], o[6] = R[5], o[7] = t[1];
    o[8] = R[6], o[9] = R[7], o[10] = R[8], o[11] = t[2];
  }
}

// ---------------------------------------------------------------- consensus
// Hypothesis testing (Alg. 1, "Find all inliers", Sec. IV: one thread block
// per (hypothesis, chunk of P), block reductions): every point of P is
// transformed and its nearest Q point found exactly in the eps grid (eq. (1),
// all cells overlapping the eps ball). Inlier iff d^2 < eps^2. The squared
// distances are summed in 2^-40 fixed point so the totals do not depend on
// the order of the atomic adds.
constexpr int kConsThreads = 256;
constexpr int kConsChunk = 2048;


// Minimum squared distance below eps2 by a group of G lanes (no index needed).
template <int G>
__device__ __forceinline__ float group_min_d2(const GridParams &g, const int *__restrict__ start,
                                              const float4 *__restrict__ Xe, float x, float y, float z, float eps2) {
  int sub = threadIdx.x & (G - 1);
  float best = eps2;
  int next = sub, base = 0;
  grid_ranges(g, start, x, y, z, [&](int b, int e) {
    int len = e - b;
    // four independent loads in flight per lane, then the remainder
    for (; next + 3 * G < base + len; next += 4 * G) {
      int t = b + next - base;
      float4 q0 = Xe[t], q1 = Xe[t + G], q2 = Xe[t + 2 * G], q3 = Xe[t + 3 * G];
      float d0 = dist2(q0, x, y, z), d1 = dist2(q1, x, y, z), d2 = dist2(q2, x, y, z), d3 = dist2(q3, x, y, z);
      best = fminf(best, fminf(fminf(d0, d1), fminf(d2, d3)));
    }
    for (; next < base + len; next += G) best = fminf(best, dist2(Xe[b + next - base], x, y, z));
    base += len;
  });
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, off));
  return best;
}

template <int G>
__global__ void __launch_bounds__(kConsThreads) k_consensus(const float4 *__restrict__ XP, int nP, const GridParams *gep,
                                                            const int *__restrict__ start,
                                                            const float4 *__restrict__ Xe, const float *__restrict__ pose,
                                                            const uint8_t *__restrict__ ok, const int *n_dev, int n_host,
                                                            float eps2, int *count, unsigned long long *sum,
                                                            const int *list) {
  constexpr int GPB = kConsThreads / G;
  const GridParams g = *gep;
  int nh = n_dev ? *n_dev : n_host;
  // few poses (the top ties, the refined pose): smaller chunks of P so that
  // every block of the grid gets work (the counts and fixed-point sums do not
  // depend on the split)
  int chunk = kConsChunk;
  while (chunk > 256 && (int64_t)nh * ((nP + chunk - 1) / chunk) < (int64_t)gridDim.x) chunk >>= 1;
  int chunks = (nP + chunk - 1) / chunk;
  int64_t items = (int64_t)nh * chunks;
  int grp = threadIdx.x / G, sub = threadIdx.x & (G - 1);
  __shared__ int s_cnt[kConsThreads / 32];
  __shared__ unsigned long long s_sum[kConsThreads / 32];
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    int s = (int)(item / chunks), c = (int)(item - (int64_t)s * chunks);
    if (list) {
      s = list[s];
    } else if (ok && !ok[s]) {
      continue;
    }
    Rigid12 T;
    T.load(pose + (size_t)s * 12);
    int cnt = 0;
    unsigned long long acc = 0ull;
    int i0 = c * chunk, i1 = (c + 1) * chunk < nP ? (c + 1) * chunk : nP;
    // block-uniform trip count: every lane reaches the group shuffles
    for (int r = i0; r < i1; r += GPB) {
      int i = r + grp;
      bool valid = i < i1;
      float4 p = valid ? XP[i] : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
      float x, y, z;
      T.apply(p, x, y, z);
      float best = group_min_d2<G>(g, start, Xe, x, y, z, eps2);
      if (valid && sub == 0 && best < eps2) {
        ++cnt;
        acc += (unsigned long long)__double2ll_rn((double)best * kFixScale);
      }
    }
    cnt = warp_sum(cnt);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_cnt[w] = cnt, s_sum[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tc = 0;
      unsigned long long ts = 0ull;
      for (int k = 0; k < kConsThreads / 32; ++k) tc += s_cnt[k], ts += s_sum[k];
      if (tc) {
        atomicAdd(&count[s], tc);
        atomicAdd(&sum[s], ts);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- selection
// Alg. 1, "Find the hypothesis that has max inlier ratio and fitness score
// passing minimum threshold": the largest inlier count wins, then the smaller
// mean squared inlier distance, then the smaller hypothesis id. Accepted if
// count >= min_ratio * |P|.
__device__ __forceinline__ bool better(int c, double f, int h, int bc, double bf, int bh) {
  if (c != bc) return c > bc;
  if (f != bf) return f < bf;
  return h < bh;
}

__global__ void __launch_bounds__(1024) k_select(const int *surv, const int *count, const unsigned long long *sum,
                                                 const uint8_t *ok, const float *pose, int nP, float min_ratio,
                                                 RansacState *st) {
  __shared__ int sc[1024], sh[1024], ss[1024];
  __shared__ double sf[1024];
  int S = st->n_surv;
  int bc = -1, bh = 0x7fffffff, bs = -1;
  double bf = DBL_MAX;
  for (int s = threadIdx.x; s < S; s += 1024) {
    if (!ok[s]) continue;
    int c = count[s];
    double f = c > 0 ? (double)sum[s] / kFixScale / (double)c : DBL_MAX;
    int h = surv[s];
    if (bs < 0 || better(c, f, h, bc, bf, bh)) bc = c, bf = f, bh = h, bs = s;
  }
  sc[threadIdx.x] = bc, sf[threadIdx.x] = bf, sh[threadIdx.x] = bh, ss[threadIdx.x] = bs;
  __syncthreads();
  for (int half = 512; half > 0; half >>= 1) {
    if (threadIdx.x < half) {
      int o = threadIdx.x + half;
      if (ss[o] >= 0 && (ss[threadIdx.x] < 0 || better(sc[o], sf[o], sh[o], sc[threadIdx.x], sf[threadIdx.x],
                                                        sh[threadIdx.x]))) {
        sc[threadIdx.x] = sc[o], sf[threadIdx.x] = sf[o], sh[threadIdx.x] = sh[o], ss[threadIdx.x] = ss[o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int best = ss[0];
    st->best = best;
    st->best_h = best >= 0 ? sh[0] : -1;
    st->best_count = best >= 0 ? sc[0] : 0;
    st->best_fit = best >= 0 && sc[0] > 0 ? (float)sf[0] : 0.f;
    bool accept = best >= 0 && (double)sc[0] >= (double)min_ratio * (double)nP;
    st->status = accept ? 0 : 1;
    st->active = accept ? 1 : 0;
    st->iters_done = 0;
    for (int i = 0; i < 16; ++i) st->T[i] = st->T_hyp[i] = (i % 5 == 0) ? 1.0 : 0.0;
    if (accept) {
      const float *T = pose + (size_t)best * 12;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) st->T_hyp[4 * r + c] = st->T[4 * r + c] = (double)T[4 * r + c];
    }
  }
}

}  // namespace

int hyp_blocks(int64_t H) { return (int)lsr_div_up(H > 0 ? H : 1, kHypPerBlock); }

int64_t hyp_local_ints(int64_t H) { return (int64_t)hyp_blocks(H) * kHypPerBlock; }

cudaError_t launch_hypotheses(const float4 *XP, const int *invP, const float4 *NP, int nP, const float4 *XQ,
                              const float4 *NQ, int nQ, const int *nn, const uint8_t *, const uint8_t *, int64_t H,
                              uint64_t seed, uint64_t pair, float tau, int *block_counts, int *block_offsets,
                              int *scan_scratch, int *surv, int surv_cap, RansacState *st, int *local,
                              cudaStream_t s) {
  HypIn in{XP, invP, NP, nP, XQ, NQ, nQ, nn, seed, pair, tau * tau};
  int nb = hyp_blocks(H);
  LSR_LAUNCH(k_hyp_count<<<nb, kHypThreads, 0, s>>>(in, H, block_counts, local));
  int *nb_dev = block_counts + nb;  // one spare int after the counts holds nb
  LSR_LAUNCH(k_set_int<<<1, 32, 0, s>>>(nb_dev, nb));
  LSR_CUDA_TRY(scan_exclusive(block_counts, block_offsets, nb_dev, nb, scan_scratch, s));
  LSR_LAUNCH(k_hyp_gather<<<nb, kHypThreads, 0, s>>>(local, block_counts, block_offsets, surv, surv_cap));
  LSR_LAUNCH(k_hyp_finish<<<1, 32, 0, s>>>(block_offsets, nb, surv_cap, st));
  return cudaGetLastError();
}

cudaError_t launch_rigid_survivors(const float4 *XP, const int *invP, const float4 *NP, int nP, const float4 *XQ,
                                   const float4 *NQ, const int *nn, const int *surv, const RansacState *st,
                                   uint64_t seed, uint64_t pair, float cos_normal, float *pose, uint8_t *ok,
                                   int *n_normal_ok, cudaStream_t s) {
  HypIn in{XP, invP, NP, nP, XQ, NQ, 0x7fffffff, nn, seed, pair, 0.f};
  LSR_LAUNCH(k_rigid_survivors<<<kSms * 4, 256, 0, s>>>(in, surv, st, cos_normal, pose, ok, n_normal_ok));
  return cudaGetLastError();
}

cudaError_t launch_rigid4(const float *ps, const float *qs, int nh, float *pose, cudaStream_t s) {
  int b = (int)lsr_div_up(nh > 0 ? nh : 1, 256);
  LSR_LAUNCH(k_rigid4<<<b, 256, 0, s>>>(ps, qs, nh, pose));
  return cudaGetLastError();
}

cudaError_t launch_consensus(const float4 *XP, int nP, const GridParams *ge, const int *start_e, const float4 *Xe,
                             const float *pose, const uint8_t *ok, const int *n_dev, int n_host, float eps, int *count,
                             unsigned long long *sum, cudaStream_t s, int lanes, const int *list) {
  float e2 = eps * eps;
#define LSR_CONS(G)                                                                                            \
  LSR_LAUNCH(k_consensus<G><<<kSms * 8, kConsThreads, 0, s>>>(XP, nP, ge, start_e, Xe, pose, ok, n_dev, n_host, e2, \
                                                             count, sum, list))
  switch (lanes) {
    case 2: LSR_CONS(2); break;
    case 4: LSR_CONS(4); break;
    case 8: LSR_CONS(8); break;
    case 16: LSR_CONS(16); break;
    default: LSR_CONS(1); break;
  }
#undef LSR_CONS
  return cudaGetLastError();
}

cudaError_t launch_select(const int *surv, const int *count, const unsigned long long *sum, const uint8_t *ok,
                          const float *pose, int nP, float min_ratio, RansacState *st, cudaStream_t s) {
  LSR_LAUNCH(k_select<<<1, 1024, 0, s>>>(surv, count, sum, ok, pose, nP, min_ratio, st));
  return cudaGetLastError();
}

// Arms the test probe on stream s (checked builds; else cudaErrorNotSupported).
cudaError_t check_probe_arm(cudaStream_t s) {
#ifdef LSR_CHECKED
  static const int one = 1;
  return cudaMemcpyToSymbolAsync(g_check_probe, &one, sizeof(int), 0, cudaMemcpyHostToDevice, s);
#else
  (void)s;
  return cudaErrorNotSupported;
#endif
}

LSR_CHECK_READER(ransac)

}  // namespace lsr
