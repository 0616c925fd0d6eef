// lsr_voxel.cu -- voxel downsampling (Algorithm 1, first line: "Downsample P
// and Q").
//
// One point per occupied voxel of edge leaf, the mean of the points in it.
// Voxels are aligned to the coordinate origin: key = floor(x / leaf) per axis,
// computed in FP64 so that every point lands in the voxel its exact
// coordinates say. The voxels of the keys' bounding box are numbered with x
// fastest; per voxel the kernel adds 1 to a count and the point's offset from
// the voxel corner, in units of leaf / 2^36, to three 64-bit integer sums --
// integer atomics, so the sums and hence the means do not depend on the order
// the points arrive in. Occupied voxels are numbered by a scan and written in
// voxel order (z slowest, then y, then x).
#include <float.h>

#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr double kVoxFix = 68719476736.0;  // 2^36: up to 2^28 points a voxel in 64 bits

__device__ __forceinline__ void vox_key(const float *P, int64_t i, double inv_leaf, int &kx, int &ky, int &kz) {
  kx = (int)floor((double)P[3 * i] * inv_leaf);
  ky = (int)floor((double)P[3 * i + 1] * inv_leaf);
  kz = (int)floor((double)P[3 * i + 2] * inv_leaf);
}

// Key bounding box: kb[0..2] minima, kb[3..5] maxima (initialised to +/- INT_MAX).
__global__ void k_vox_bounds(const float *__restrict__ P, int64_t n, double inv_leaf, int *__restrict__ kb) {
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int k[3];
    vox_key(P, i, inv_leaf, k[0], k[1], k[2]);
    for (int d = 0; d < 3; ++d) lo[d] = min(lo[d], k[d]), hi[d] = max(hi[d], k[d]);
  }
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
    if ((threadIdx.x & 31) == 0) atomicMin(kb + d, lo[d]), atomicMax(kb + 3 + d, hi[d]);
  }
}

__global__ void k_vox_accum(const float *__restrict__ P, int64_t n, double leaf, double inv_leaf,
                            const int *__restrict__ kb, int *__restrict__ cnt, unsigned long long *__restrict__ sums) {
  const int64_t nx = (int64_t)kb[3] - kb[0] + 1, ny = (int64_t)kb[4] - kb[1] + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int k[3];
    vox_key(P, i, inv_leaf, k[0], k[1], k[2]);
    const int64_t c = ((int64_t)(k[2] - kb[2]) * ny + (k[1] - kb[1])) * nx + (k[0] - kb[0]);
    atomicAdd(cnt + c, 1);
    for (int d = 0; d < 3; ++d) {
      // offset from the voxel corner in [0, leaf), as a 36-bit fraction of leaf
      const double f = ((double)P[3 * i + d] - (double)k[d] * leaf) * inv_leaf;
      const double q = fmin(fmax(f, 0.0), 1.0) * kVoxFix;
      atomicAdd(sums + 3 * c + d, (unsigned long long)q);
    }
  }
}

__global__ void k_vox_flags(const int *__restrict__ cnt, const int *ncells, int *__restrict__ flag) {
  const int64_t nc = *ncells;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
    flag[c] = cnt[c] > 0 ? 1 : 0;
}

__global__ void k_vox_emit(const int *__restrict__ kb, const int *ncells, double leaf, const int *__restrict__ cnt,
                           const unsigned long long *__restrict__ sums, const int *__restrict__ pos,
                           float *__restrict__ out, int64_t cap, int64_t *__restrict__ n_out) {
  const int64_t nc = *ncells;
  const int64_t nx = (int64_t)kb[3] - kb[0] + 1, ny = (int64_t)kb[4] - kb[1] + 1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const int k = cnt[c];
    if (k == 0 || pos[c] >= cap) continue;
    const int64_t key[3] = {kb[0] + c % nx, kb[1] + (c / nx) % ny, kb[2] + c / (nx * ny)};
    for (int d = 0; d < 3; ++d)
      out[3 * (int64_t)pos[c] + d] =
          (float)(((double)key[d] + (double)sums[3 * c + d] / (kVoxFix * (double)k)) * leaf);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = pos[nc];
}

}  // namespace

cudaError_t launch_vox_bounds(const float *P, int64_t n, float leaf, int *kb, cudaStream_t s) {
  const int init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
  LSR_CUDA_TRY(cudaMemcpyAsync(kb, init, sizeof(init), cudaMemcpyHostToDevice, s));
  const int64_t nb = lsr_div_up(n, 256);
  LSR_LAUNCH(k_vox_bounds<<<(int)(nb < 1216 ? nb : 1216), 256, 0, s>>>(P, n, 1.0 / (double)leaf, kb));
  return cudaGetLastError();
}

cudaError_t launch_vox_cells(const float *P, int64_t n, float leaf, const int *kb, int64_t ncells,
                             const int *ncells_dev, int *cnt, unsigned long long *sums, int *flag, int *pos,
                             int *scan, float *out, int64_t cap, int64_t *n_out, cudaStream_t s) {
  LSR_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)ncells, s));
  LSR_CUDA_TRY(cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * 3 * (size_t)ncells, s));
  const int64_t nb = lsr_div_up(n, 256), cb = lsr_div_up(ncells, 256);
  LSR_LAUNCH(k_vox_accum<<<(int)(nb < 1216 ? nb : 1216), 256, 0, s>>>(P, n, (double)leaf, 1.0 / (double)leaf, kb, cnt,
                                                                    sums));
  LSR_LAUNCH(k_vox_flags<<<(int)(cb < 1216 ? cb : 1216), 256, 0, s>>>(cnt, ncells_dev, flag));
  LSR_CUDA_TRY(scan_exclusive(flag, pos, ncells_dev, (int)ncells, scan, s));
  LSR_LAUNCH(k_vox_emit<<<(int)(cb < 1216 ? cb : 1216), 256, 0, s>>>(kb, ncells_dev, (double)leaf, cnt, sums, pos, out,
                                                                   cap, n_out));
  return cudaGetLastError();
}

}  // namespace lsr
