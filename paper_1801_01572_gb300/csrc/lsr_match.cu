// lsr_match.cu -- feature pre-matching cache on the FP32 cores (Algorithm 1,
// "Parallel FPFH feature pre-matching": nn[i] = NN of F(p_i) in F(Q)).
//
// Exact brute force: nn[i] = argmin_j sum_k (a_k - b_k)^2 with ties to the
// smallest j, accumulated as s = fma(t, t, s) over k = 0..32. Each thread keeps
// two query descriptors in registers; tiles of database descriptors are
// staged in shared memory and read as broadcasts, so one shared load feeds two
// distance accumulations. The partial sums only grow (t^2 >= 0 and rounding is
// monotone), so a row whose partial sum already exceeds every query's current
// best in the warp can neither win nor tie: after 8, 16 and 24 components the
// warp tests that and skips the rest of the row (same result).
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
        if (c % 2 == 0 && c > 0) {
          bool past = true;
#pragma unroll
          for (int u = 0; u < kQPT; ++u) past &= s[u] > best[u];
          if (__all_sync(0xffffffffu, past)) break;
        }
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
        if (c == 7) {
          float b32 = tile[j][8].x;
#pragma unroll
          for (int u = 0; u < kQPT; ++u) {
            float t = a[u][32] - b32;
            s[u] = fmaf(t, t, s[u]);
            if (s[u] < best[u]) best[u] = s[u], bj[u] = base + j;
          }
        }
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
  for (int t0 = blockIdx.x; t0 * (kMT * kQPT) < nq; t0 += gridDim.x) {
    float a[kQPT][kD];
    int slot[kQPT];
#pragma unroll
    for (int u = 0; u < kQPT; ++u) {
      int q = t0 * (kMT * kQPT) + u * kMT + threadIdx.x;
      slot[u] = q < nq ? q : -1;
      int qi = q < nq ? rows[q] : 0;
      const float *row = FP + (size_t)(qi < nP ? qi : 0) * kDS;
#pragma unroll
      for (int k = 0; k < kD; ++k) a[u][k] = row[k];
    }
    float best[kQPT];
    int bj[kQPT];
#pragma unroll
    for (int u = 0; u < kQPT; ++u) best[u] = FLT_MAX, bj[u] = -1;
    for (int base = j0; base < j1; base += kTile) {
      __syncthreads();
      for (int k = threadIdx.x; k < kTile * 9; k += kMT) {
        int r = k / 9, c = k - 9 * r;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (base + r < j1) v = reinterpret_cast<const float4 *>(FQ + (size_t)(base + r) * kDS)[c];
        tile[r][c] = v;
      }
      __syncthreads();
      int m = j1 - base < kTile ? j1 - base : kTile;
      for (int j = 0; j < m; ++j) {
        float s[kQPT];
#pragma unroll
        for (int u = 0; u < kQPT; ++u) s[u] = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c % 2 == 0 && c > 0) {
            bool past = true;
#pragma unroll
            for (int u = 0; u < kQPT; ++u) past &= s[u] > best[u];
            if (__all_sync(0xffffffffu, past)) break;
          }
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
          if (c == 7) {
            float b32 = tile[j][8].x;
#pragma unroll
            for (int u = 0; u < kQPT; ++u) {
              float t = a[u][32] - b32;
              s[u] = fmaf(t, t, s[u]);
              if (s[u] < best[u]) best[u] = s[u], bj[u] = base + j;
            }
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kQPT; ++u)
      if (slot[u] >= 0 && bj[u] >= 0)
        atomicMin(packed + slot[u], ((unsigned long long)__float_as_uint(best[u]) << 32) | (unsigned)bj[u]);
    __syncthreads();
  }
}

__global__ void k_rows_init(const int *nrows, unsigned long long *packed) {
  const int nq = *nrows;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) packed[q] = ~0ull;
}

__global__ void k_rows_finish(const int *rows, const int *nrows, const unsigned long long *packed, int *nn,
                              float *d1) {
  const int nq = *nrows;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    unsigned long long v = packed[q];
    int r = rows[q];
    bool none = v == ~0ull;
    nn[r] = none ? -1 : (int)(unsigned)(v & 0xFFFFFFFFu);
    if (d1) d1[r] = none ? FLT_MAX : __uint_as_float((unsigned)(v >> 32));
  }
}

}  // namespace

cudaError_t launch_match_fp32(const float *FP, int nP, const float *FQ, int nQ, int *nn, float *d1, cudaStream_t s) {
  int blocks = (int)lsr_div_up(nP, kMT * kQPT);
  if (blocks < 1) blocks = 1;
  LSR_LAUNCH(k_match_fp32<<<blocks, kMT, 0, s>>>(FP, nP, FQ, nQ, nn, d1));
  return cudaGetLastError();
}

cudaError_t launch_match_fp32_rows(const float *FP, int nP, const float *FQ, int nQ, const int *rows,
                                   const int *nrows, unsigned long long *packed, int *nn, float *d1,
                                   cudaStream_t s) {
  constexpr int kChunks = 64;
  int chunk = (int)lsr_div_up(lsr_div_up(nQ, kChunks), kTile) * kTile;
  int ny = (int)lsr_div_up(nQ, chunk);
  int nx = (int)lsr_div_up(nP, kMT * kQPT);
  nx = nx < 1 ? 1 : (nx > 10 ? 10 : nx);
  int fin = (int)lsr_div_up(nP, 256);
  fin = fin < 1 ? 1 : (fin > 1216 ? 1216 : fin);
  LSR_LAUNCH(k_rows_init<<<fin, 256, 0, s>>>(nrows, packed));
  LSR_LAUNCH(k_match_rows_chunked<<<dim3(nx, ny), kMT, 0, s>>>(FP, nP, FQ, nQ, chunk, rows, nrows, packed));
  LSR_LAUNCH(k_rows_finish<<<fin, 256, 0, s>>>(rows, nrows, packed, nn, d1));
  return cudaGetLastError();
}

}  // namespace lsr
