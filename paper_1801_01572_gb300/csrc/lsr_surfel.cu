// lsr_surfel.cu -- dense model correction after a loop closure (eq. (7)).
//
// Every surfel moves with the keyframes that observe it: with F the keyframes
// f whose time stamp lies strictly between the surfel's initialisation and
// last-update stamps and whose camera (before the correction) sees the
// surfel -- in front of it, no farther than the maximum depth, projecting
// inside the image --
//   p' = (1/k) sum_f T_f_new T_f_old^-1 p,   n' = normalize(sum_f R_f_new R_f_old^-1 n),
// k = |F|; a surfel no keyframe observes is removed. Surfels do not interact:
// one thread per surfel, the keyframes' two 3 x 4 transforms (precomputed on
// the host in FP64, stored in FP32) read through the read-only cache, the
// time window found by binary search over the sorted keyframe stamps.
#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kSurfThreads = 256;

__device__ __forceinline__ void xf34(const float *__restrict__ T, float x, float y, float z, float &ox, float &oy,
                                     float &oz) {
  ox = fmaf(__ldg(T + 0), x, fmaf(__ldg(T + 1), y, fmaf(__ldg(T + 2), z, __ldg(T + 3))));
  oy = fmaf(__ldg(T + 4), x, fmaf(__ldg(T + 5), y, fmaf(__ldg(T + 6), z, __ldg(T + 7))));
  oz = fmaf(__ldg(T + 8), x, fmaf(__ldg(T + 9), y, fmaf(__ldg(T + 10), z, __ldg(T + 11))));
}

__global__ void __launch_bounds__(kSurfThreads) k_surfel_correct(int64_t n, const float *__restrict__ pos,
                                                                 const float *__restrict__ nrm,
                                                                 const float *__restrict__ t0,
                                                                 const float *__restrict__ tu, int m,
                                                                 const KfPose *__restrict__ kf,
                                                                 const float *__restrict__ t_kf, SurfelCam cam,
                                                                 float *__restrict__ pos_out,
                                                                 float *__restrict__ nrm_out,
                                                                 uint8_t *__restrict__ keep,
                                                                 unsigned long long *__restrict__ n_keep) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    const float nx = nrm[3 * i], ny = nrm[3 * i + 1], nz = nrm[3 * i + 2];
    const float a = t0[i], b = tu[i];
    // first keyframe with t_f > t0
    int lo = 0, hi = m;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(t_kf + mid) > a) hi = mid; else lo = mid + 1;
    }
    int k = 0;
    float sx = 0.f, sy = 0.f, sz = 0.f, qx = 0.f, qy = 0.f, qz = 0.f;
    for (int f = lo; f < m && __ldg(t_kf + f) < b; ++f) {
      float cx, cy, cz;
      xf34(kf[f].A, px, py, pz, cx, cy, cz);
      if (!(cz > 0.f && cz <= cam.dmax)) continue;
      const float u = cam.fx * cx / cz + cam.cx, v = cam.fy * cy / cz + cam.cy;
      if (!(u >= 0.f && u < cam.w && v >= 0.f && v < cam.h)) continue;
      float ox, oy, oz;
      xf34(kf[f].M, px, py, pz, ox, oy, oz);
      sx += ox, sy += oy, sz += oz;
      const float *R = kf[f].M;
      qx += fmaf(__ldg(R + 0), nx, fmaf(__ldg(R + 1), ny, __ldg(R + 2) * nz));
      qy += fmaf(__ldg(R + 4), nx, fmaf(__ldg(R + 5), ny, __ldg(R + 6) * nz));
      qz += fmaf(__ldg(R + 8), nx, fmaf(__ldg(R + 9), ny, __ldg(R + 10) * nz));
      ++k;
    }
    const bool kept = k > 0;
    float op[3] = {px, py, pz}, on[3] = {nx, ny, nz};
    if (kept) {
      const float ik = 1.f / (float)k;
      op[0] = sx * ik, op[1] = sy * ik, op[2] = sz * ik;
      const float il = rsqrtf(fmaxf(qx * qx + qy * qy + qz * qz, 1e-30f));
      on[0] = qx * il, on[1] = qy * il, on[2] = qz * il;
    }
    for (int d = 0; d < 3; ++d) pos_out[3 * i + d] = op[d], nrm_out[3 * i + d] = on[d];
    keep[i] = kept ? 1 : 0;
    const unsigned ballot = __ballot_sync(__activemask(), kept);
    if (ballot && (threadIdx.x & 31) == __ffs(__activemask()) - 1) atomicAdd(n_keep, (unsigned long long)__popc(ballot));
  }
}

}  // namespace

cudaError_t launch_surfel_correct(int64_t n, const float *pos, const float *nrm, const float *t0, const float *tu,
                                  int m, const KfPose *kf, const float *t_kf, const SurfelCam &cam, float *pos_out,
                                  float *nrm_out, uint8_t *keep, unsigned long long *n_keep, cudaStream_t s) {
  LSR_CUDA_TRY(cudaMemsetAsync(n_keep, 0, sizeof(unsigned long long), s));
  const int64_t nb = lsr_div_up(n, kSurfThreads);
  const int blocks = (int)(nb < 1 ? 1 : (nb > kSms * 16 ? kSms * 16 : nb));
  LSR_LAUNCH(k_surfel_correct<<<blocks, kSurfThreads, 0, s>>>(n, pos, nrm, t0, tu, m, kf, t_kf, cam, pos_out, nrm_out,
                                                               keep, n_keep));
  return cudaGetLastError();
}

}  // namespace lsr
