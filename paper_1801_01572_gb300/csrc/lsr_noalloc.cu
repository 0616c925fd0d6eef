// lsr_noalloc.cu -- pose scoring that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need to
// score candidate poses: a SLAM back end that re-checks loop candidates inside
// a real-time loop with a hard latency budget, a process whose device memory
// is owned by another framework's pool, or code that must not change the
// device's allocation state between two points in time. For them,
// lsr_consensus_static scores poses against a fragment pair exactly like
// lsr_stage_consensus, but takes its scratch space from one fixed array that
// lives in the library's device image instead of from a context workspace.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (kStaticScratchBytes) until the process exits. Host code
// cannot use the array's name as a device address: on the first call on each
// device the entry point asks the runtime for the array's device address
// (cudaGetSymbolAddress, with that device current) and caches it; every later
// call on that device reuses the cached address. The cached address does not
// survive a reset of the device. Every call synchronises its stream before
// returning.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/lsr.h"
#include "lsr_internal.cuh"

namespace lsr {

namespace {

// Fixed limits of the allocation-free entry point.
constexpr int64_t kStaticMaxP = 65536;
constexpr int64_t kStaticMaxQ = 65536;
constexpr int64_t kStaticMaxPoses = 4096;
constexpr int kStaticCapCells = 1 << 20;  // eps-grid cells (wraps beyond)
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;

// The scratch array itself: shared by every call on a device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
int static_scratch(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LSR_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return LSR_E_ARG;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return LSR_E_CUDA;
    }
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return LSR_OK;
}

// Carves aligned pieces out of the fixed array; fails instead of growing.
struct StaticCarve {
  char *base;
  size_t off = 0, cap;
  bool ok = true;
  template <class T>
  T *take(size_t n) {
    off = (off + 255) / 256 * 256;
    size_t bytes = sizeof(T) * (n > 0 ? n : 1);
    if (off + bytes > cap) {
      ok = false;
      return nullptr;
    }
    T *p = reinterpret_cast<T *>(base + off);
    off += bytes;
    return p;
  }
};

__global__ void k_pack_static(const float *xyz, int n, float4 *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __int_as_float(i));
}

__global__ void k_fix_to_double(const unsigned long long *s, int n, double *d) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    d[k] = (double)s[k] / kFixScale;
}

int blocks_for(int64_t n) { return (int)(n < 1 ? 1 : ((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096)); }

}  // namespace
}  // namespace lsr

using namespace lsr;

extern "C" int lsr_consensus_static(const float *P, int64_t nP, const float *Q, int64_t nQ, const float *Rt,
                                    int64_t nh, float eps, int32_t *count, double *sumd2, void *cuda_stream) {
  if (!P || !Q || !Rt || !count || !sumd2 || nP < 1 || nQ < 1 || nh < 1 || !(eps > 0.f && eps <= 10.f))
    return LSR_E_ARG;
  if (nP > kStaticMaxP || nQ > kStaticMaxQ || nh > kStaticMaxPoses) return LSR_E_TOO_LARGE;
  void *base = nullptr;
  int rc = static_scratch(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;

  StaticCarve a{(char *)base, 0, kStaticScratchBytes};
  float *p = a.take<float>(3 * nP);
  float *q = a.take<float>(3 * nQ);
  float4 *XP = a.take<float4>(nP);
  float *box = a.take<float>(kBox);
  double *box_part = a.take<double>((size_t)kBoxPart * bbox_blocks((int)nQ));
  GridParams *ge = a.take<GridParams>(1);
  int *start = a.take<int>((size_t)kStaticCapCells + 1);
  float4 *Xe = a.take<float4>(nQ);
  int *inv = a.take<int>(nQ);
  unsigned *mask = a.take<unsigned>((size_t)nbmask_words(kStaticCapCells));
  GridScratch sc;
  sc.slot = a.take<int>(nQ);
  sc.tmp = a.take<int>(nQ);
  sc.counts = a.take<int>((size_t)kStaticCapCells + 1);
  sc.scan = a.take<int>((size_t)scan_scratch_ints(kStaticCapCells));
  float *pose = a.take<float>(12 * nh);
  int *cnt = a.take<int>(nh);
  unsigned long long *sum = a.take<unsigned long long>(nh);
  double *sd = a.take<double>(nh);
  if (!a.ok) return LSR_E_TOO_LARGE;  // cannot happen within the limits above

#define LSR_STATIC_TRY(call)            \
  do {                                  \
    if ((call) != cudaSuccess) {        \
      cudaGetLastError();               \
      return LSR_E_CUDA;                \
    }                                   \
  } while (0)
  // inputs (device or host) into the fixed array; no allocation anywhere
  LSR_STATIC_TRY(cudaMemcpyAsync(p, P, sizeof(float) * 3 * nP, cudaMemcpyDefault, s));
  LSR_STATIC_TRY(cudaMemcpyAsync(q, Q, sizeof(float) * 3 * nQ, cudaMemcpyDefault, s));
  LSR_STATIC_TRY(cudaMemcpyAsync(pose, Rt, sizeof(float) * 12 * nh, cudaMemcpyDefault, s));
  LSR_LAUNCH(k_pack_static<<<blocks_for(nP), 256, 0, s>>>(p, (int)nP, XP));
  // the eps grid of Q (the array keeps the previous call's contents: every
  // piece below is fully rewritten, and the sums are cleared)
  LSR_STATIC_TRY(launch_bbox_xyz(q, (int)nQ, box_part, bbox_blocks((int)nQ), box, s));
  LSR_STATIC_TRY(launch_grid_params(box, eps, (int)nQ, kStaticCapCells, ge, s));
  LSR_STATIC_TRY(build_grid_xyz(q, (int)nQ, ge, kStaticCapCells, start, Xe, inv, sc, s));
  LSR_STATIC_TRY(build_nbmask(ge, start, kStaticCapCells, mask, s));
  LSR_STATIC_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * nh, s));
  LSR_STATIC_TRY(cudaMemsetAsync(sum, 0, sizeof(unsigned long long) * nh, s));
  LSR_STATIC_TRY(launch_consensus(XP, (int)nP, ge, start, Xe, pose, nullptr, nullptr, (int)nh, eps, cnt, sum, s));
  LSR_LAUNCH(k_fix_to_double<<<blocks_for(nh), 256, 0, s>>>(sum, (int)nh, sd));
  LSR_STATIC_TRY(cudaGetLastError());
  LSR_STATIC_TRY(cudaMemcpyAsync(count, cnt, sizeof(int) * nh, cudaMemcpyDefault, s));
  LSR_STATIC_TRY(cudaMemcpyAsync(sumd2, sd, sizeof(double) * nh, cudaMemcpyDefault, s));
  LSR_STATIC_TRY(cudaStreamSynchronize(s));
#undef LSR_STATIC_TRY
  return LSR_OK;
}
