// lsr_match.cu -- feature pre-matching cache on the FP32 cores (Algorithm 1,
// "Parallel FPFH feature pre-matching": nn[i] = NN of F(p_i) in F(Q)).
//
// Exact brute force: nn[i] = argmin_j sum_k (a_k - b_k)^2 with ties to the
// smallest j. Each thread keeps two query descriptors in registers; tiles of
// database descriptors are staged in shared memory and read as broadcasts,
// so one shared load feeds two distance accumulations.
#include <float.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kMT = 128;   // threads per block
constexpr int kQPT = 2;    // queries per thread
constexpr int kTile = 64;  // database rows per shared-memory tile

__global__ void __launch_bounds__(kMT) k_match_fp32(const float *__restrict__ FP, int nP, const float *__restrict__ FQ,
                                                    int nQ, int *__restrict__ nn, float *__restrict__ d1) {
  __shared__ float4 tile[kTile][9];
  float a[kQPT][kD];
  int qi[kQPT];
#pragma unroll
  for (int u = 0; u < kQPT; ++u) {
    qi[u] = blockIdx.x * (kMT * kQPT) + u * kMT + threadIdx.x;
    const float *row = FP + (size_t)(qi[u] < nP ? qi[u] : 0) * kDS;
#pragma unroll
    for (int k = 0; k < kD; ++k) a[u][k] = row[k];
  }
  float best[kQPT];
  int bj[kQPT];
#pragma unroll
  for (int u = 0; u < kQPT; ++u) best[u] = FLT_MAX, bj[u] = -1;
  for (int base = 0; base < nQ; base += kTile) {
    __syncthreads();
    for (int k = threadIdx.x; k < kTile * 9; k += kMT) {
      int r = k / 9, c = k - 9 * r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (base + r < nQ) v = reinterpret_cast<const float4 *>(FQ + (size_t)(base + r) * kDS)[c];
      tile[r][c] = v;
    }
    __syncthreads();
    int m = nQ - base < kTile ? nQ - base : kTile;
    for (int j = 0; j < m; ++j) {
      float s[kQPT];
#pragma unroll
      for (int u = 0; u < kQPT; ++u) s[u] = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float4 b = tile[j][c];
#pragma unroll
        for (int u = 0; u < kQPT; ++u) {
          float t0 = a[u][4 * c] - b.x, t1 = a[u][4 * c + 1] - b.y, t2 = a[u][4 * c + 2] - b.z,
                t3 = a[u][4 * c + 3] - b.w;
          s[u] = fmaf(t0, t0, s[u]);
          s[u] = fmaf(t1, t1, s[u]);
          s[u] = fmaf(t2, t2, s[u]);
          s[u] = fmaf(t3, t3, s[u]);
        }
      }
      float b32 = tile[j][8].x;
#pragma unroll
      for (int u = 0; u < kQPT; ++u) {
        float t = a[u][32] - b32;
        s[u] = fmaf(t, t, s[u]);
        if (s[u] < best[u]) best[u] = s[u], bj[u] = base + j;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kQPT; ++u)
    if (qi[u] < nP) {
      nn[qi[u]] = bj[u];
      if (d1) d1[qi[u]] = best[u];
    }
}

}  // namespace

cudaError_t launch_match_fp32(const float *FP, int nP, const float *FQ, int nQ, int *nn, float *d1, cudaStream_t s) {
  int blocks = (int)lsr_div_up(nP, kMT * kQPT);
  if (blocks < 1) blocks = 1;
  LSR_LAUNCH(k_match_fp32<<<blocks, kMT, 0, s>>>(FP, nP, FQ, nQ, nn, d1));
  return cudaGetLastError();
}

}  // namespace lsr
