// lsr_api.cu -- the C ABI (include/lsr.h): context, device workspace, and the
// host-side orchestration of the registration pipeline of Algorithm 1.
//
// Every stage runs on the context's stream without host round trips: counts
// that decide launch sizes (survivors, selected hypothesis, convergence) live
// in device memory and are read by persistent-grid kernels, so a whole
// registration is one stream of launches followed by a single device-to-host
// copy of the result and one synchronisation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "../../include/lsr.h"
#include "lsr_internal.cuh"

using namespace lsr;

namespace lsr {
unsigned long long g_launches = 0;

// Per-kernel timing: events from a reusable pool bracket the matching
// launches; after the call has synchronised, their elapsed times are added to
// a table keyed by kernel name (the launch expression up to its <<<).
struct KernelTimer {
  cudaStream_t stream = nullptr;
  std::string filter;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Open {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Open> open;
  cudaEvent_t pending_start = nullptr;
  bool failed = false;
  struct Entry {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0;
  };
  std::vector<Entry> table;

  cudaEvent_t take() {
    if (used == pool.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        failed = true;
        return nullptr;
      }
      pool.push_back(e);
    }
    return pool[used++];
  }
  // After the stream has synchronised: fold the bracketed launches into the table.
  void collect() {
    for (const Open &o : open) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, o.a, o.b) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      Entry *e = nullptr;
      for (Entry &x : table)
        if (x.name == o.name) e = &x;
      if (!e) {
        table.push_back(Entry{o.name});
        e = &table.back();
      }
      e->launches += 1;
      e->ms += ms;
    }
    open.clear();
    used = 0;
  }
  ~KernelTimer() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

thread_local KernelTimer *g_ktimer = nullptr;

static std::string kernel_name_of(const char *expr) {
  const char *p = expr;
  // a programmatic-dependent launch: pdl_launch(kernel, ...)
  if (const char *k = strstr(p, "pdl_launch(")) {
    p = k + strlen("pdl_launch(");
    const char *q = strchr(p, ',');
    std::string out;
    for (const char *c = p; *c && c != q; ++c)
      if (*c != ' ' && *c != '\n') out.push_back(*c);
    return out;
  }
  while (*p == ' ' || *p == '(' || *p == '\n') ++p;
  const char *q = strstr(p, "<<<");
  std::string n = q ? std::string(p, q) : std::string(p);
  std::string out;
  for (char ch : n)
    if (ch != ' ' && ch != '\n') out.push_back(ch);
  return out;
}

void ktimer_mark(const char *launch_expr, bool after) {
  KernelTimer *t = g_ktimer;
  if (!t || t->failed) return;
  if (!after) {
    t->pending_start = nullptr;
    std::string name = kernel_name_of(launch_expr);
    if (name.compare(0, t->filter.size(), t->filter) != 0) return;
    cudaEvent_t a = t->take();
    if (!a || cudaEventRecord(a, t->stream) != cudaSuccess) {
      cudaGetLastError();
      t->failed = true;
      return;
    }
    t->pending_start = a;
    t->open.push_back(KernelTimer::Open{name, a, nullptr});
  } else {
    if (!t->pending_start) return;
    cudaEvent_t b = t->take();
    if (!b || cudaEventRecord(b, t->stream) != cudaSuccess) {
      cudaGetLastError();
      t->failed = true;
      t->open.pop_back();
      return;
    }
    t->open.back().b = b;
    t->pending_start = nullptr;
  }
}
}  // namespace lsr

struct lsr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  lsr_params prm{};
  bool profiling = false;
  char *ws = nullptr;
  size_t ws_cap = 0;
  RansacState *st_host = nullptr;  // pinned, one per batch slot
  int st_host_cap = 0;
  float *box_host = nullptr;       // pinned, 2 x 8 floats per slot
  cudaEvent_t ev[9] = {};
  std::string last_error;
  bool broken = false;
  // consensus tuning: lanes per nearest-neighbour query (2 measured fastest
  // on the 150k-point room pair among 1..16; LSR_CONSENSUS_LANES overrides)
  int cons_lanes = 2;
  // concurrent batches: worker streams, each with its own workspace
  std::vector<cudaStream_t> lanes;
  std::vector<char *> lane_ws;
  std::vector<size_t> lane_cap;
  std::vector<cudaEvent_t> lane_done;
  cudaEvent_t fork = nullptr;
  // the last captured batch graph, its signature and its kernel count
  cudaGraphExec_t gexec = nullptr;
  std::string gkey;
  unsigned long long glaunches = 0;
  // autotuner choices: matcher tile shape per size bucket (ceil log2 of the
  // query count; 0 = not tuned yet) and the number of batch streams
  int tile_choice[32] = {};
  int streams_choice = 0;
  // test-only fault injection (lsr_debug_inject): device workspace
  // allocations to fail, tensor-core matcher launches to stall
  int inject_alloc = 0;
  int inject_stall = 0;
  // per-kernel event timing (lsr_set_kernel_timing); null when off
  KernelTimer *ktimer = nullptr;
};

namespace {

constexpr size_t kAlign = 256;

// Bump allocator over the workspace; with base == nullptr it only measures.
struct Arena {
  char *base;
  size_t off = 0;
  explicit Arena(char *b) : base(b) {}
  template <class T>
  T *take(size_t n) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += sizeof(T) * (n > 0 ? n : 1);
    return p;
  }
};

int cap_cells_for(int n) { return std::max(8 * n, 1 << 20); }

// Consensus: clouds of P from this size on take the estimate pre-pass (every
// kConsensusPrepassStride-th point) before the full bounds pass.
constexpr int kConsensusPrepassMin = 16384;
constexpr int kConsensusPrepassStride = 16;

struct CloudLayout {
  int n = 0, cap_f = 0, cap_n = 0, cap_e = 0;
  float *src = nullptr;  // staged copy of host input (or null)
  float *box = nullptr;  // 8 floats: bbox (6) + non-finite flag + pad
  double *box_part = nullptr;
  GridParams *gf = nullptr, *gn = nullptr, *ge = nullptr;
  int *start_f = nullptr, *start_n = nullptr, *start_e = nullptr;
  float4 *X = nullptr, *Xn = nullptr, *Xe = nullptr, *N = nullptr;
  int *inv = nullptr;
  float *S = nullptr, *F = nullptr;
  unsigned *mask_e = nullptr;
};

struct ScratchLayout {
  int n_max = 0, cap_max = 0;
  GridScratch g{};
};

void plan_cloud(Arena &a, int n, bool stage_src, bool features, bool eps_grid, CloudLayout &c) {
  c.n = n;
  c.cap_f = cap_cells_for(n);
  c.cap_n = cap_cells_for(n);
  c.cap_e = cap_cells_for(n);
  c.src = stage_src ? a.take<float>((size_t)3 * n) : nullptr;
  c.box = a.take<float>(kBox);
  c.box_part = a.take<double>((size_t)kBoxPart * bbox_blocks(n));
  c.gf = a.take<GridParams>(1);
  c.gn = a.take<GridParams>(1);
  c.ge = a.take<GridParams>(1);
  c.start_f = a.take<int>((size_t)c.cap_f + 1);
  c.X = a.take<float4>(n);
  c.inv = a.take<int>(n);
  if (features) {
    c.start_n = a.take<int>((size_t)c.cap_n + 1);
    c.Xn = a.take<float4>(n);
    c.N = a.take<float4>(n);
    c.S = a.take<float>((size_t)n * kDS);
    c.F = a.take<float>((size_t)n * kDS);
  }
  if (eps_grid) {
    c.start_e = a.take<int>((size_t)c.cap_e + 1);
    c.Xe = a.take<float4>(n);
    c.mask_e = a.take<unsigned>((size_t)nbmask_words(c.cap_e));
  }
}

void plan_scratch(Arena &a, int n_max, int cap_max, ScratchLayout &s) {
  s.n_max = n_max;
  s.cap_max = cap_max;
  s.g.slot = a.take<int>(n_max);
  s.g.tmp = a.take<int>(n_max);
  s.g.counts = a.take<int>((size_t)cap_max + 1);
  s.g.scan = a.take<int>((size_t)scan_scratch_ints(cap_max));
}

// Coarse levels of the graduated refinement: subsampled copies of Q and their
// grids (the finest level uses Q's eps grid).
struct LevelLayout {
  int levels = 0;
  int sQ[kMaxLevels] = {}, nsub[kMaxLevels] = {}, cap[kMaxLevels] = {};
  int sP[kMaxLevels] = {}, nsubP[kMaxLevels] = {};
  float4 *Qsub[kMaxLevels] = {}, *Xs[kMaxLevels] = {}, *Psub[kMaxLevels] = {};
  int *start[kMaxLevels] = {};
  unsigned *mask[kMaxLevels] = {};
  GridParams *g[kMaxLevels] = {};
};

void plan_levels(Arena &a, int nP, int nQ, int levels, LevelLayout &V) {
  V.levels = levels;
  for (int l = 0; l < levels; ++l) {
    V.sP[l] = gnc_stride(nP, l, levels);
    V.nsubP[l] = (int)lsr_div_up(nP, V.sP[l]);
    if (V.sP[l] > 1) V.Psub[l] = a.take<float4>(V.nsubP[l]);
  }
  for (int l = 0; l + 1 < levels; ++l) {
    V.sQ[l] = gnc_stride(nQ, l, levels);
    V.nsub[l] = (int)lsr_div_up(nQ, V.sQ[l]);
    V.cap[l] = cap_cells_for(V.nsub[l]);
    V.Qsub[l] = a.take<float4>(V.nsub[l]);
    V.Xs[l] = a.take<float4>(V.nsub[l]);
    V.start[l] = a.take<int>((size_t)V.cap[l] + 1);
    V.mask[l] = a.take<unsigned>((size_t)nbmask_words(V.cap[l]));
    V.g[l] = a.take<GridParams>(1);
  }
}

struct PairLayout {
  CloudLayout P, Q;
  LevelLayout lv;
  ScratchLayout sc;
  int *nn = nullptr;
  float *d1 = nullptr;
  int nb = 0;
  int *blk_cnt = nullptr, *blk_off = nullptr, *blk_scan = nullptr;
  int *hyp_local = nullptr;  // per hypothesis block: its survivors, before they are placed
  int surv_cap = 0;
  int *surv = nullptr;
  float *pose = nullptr;
  uint8_t *ok = nullptr;
  int *count = nullptr;
  unsigned long long *sum = nullptr;
  double *ref_part = nullptr;
  int *seeds = nullptr;      // refinement: each point's neighbour of the previous step
  float *fpose = nullptr;
  int *fcount = nullptr;
  unsigned long long *fsum = nullptr;
  RansacState *st = nullptr;
  char *tc_ws = nullptr;  // matcher workspace (tile bounds for FP32, operands and lists for BF16)
  ClsParams *cls = nullptr;  // consensus voxel classification of Q
  unsigned *in_bits = nullptr, *near_bits = nullptr;
  uint8_t *sel = nullptr;    // the hypotheses with the largest count upper bounds
  uint8_t *rest = nullptr;   // the others whose upper bound reaches their best count
  uint8_t *reach = nullptr;  // sel | rest: the hypotheses counted exactly
  uint8_t *tie = nullptr;    // those tied at the maximum exact count
  int *amb = nullptr;        // points in undecided voxels per hypothesis
  int *count2 = nullptr;     // exact counts of the reaching hypotheses
  int *tie_list = nullptr;   // the survivor slots tied at the top
  unsigned long long *prog = nullptr;  // per survivor: bounds progress (points done << 32 | IN + undecided)
  int *c0 = nullptr;         // an exact count reached by some survivor (the bounds pass's bar)
  // single-cell lattice of Q (lsr_params.nn_mode = LSR_NN_SINGLE_CELL)
  int cap_s = 0;
  GridParams *gs = nullptr;
  int *start_s = nullptr;
  float4 *Xs = nullptr;
};

int surv_cap_for(int64_t H) { return (int)std::min<int64_t>(H, (int64_t)1 << 22); }

void plan_pair(Arena &a, int nP, int nQ, bool stP, bool stQ, int64_t H, int levels, int precision,
               PairLayout &L) {
  plan_cloud(a, nP, stP, true, false, L.P);
  plan_cloud(a, nQ, stQ, true, true, L.Q);
  plan_levels(a, nP, nQ, levels, L.lv);
  plan_scratch(a, std::max(nP, nQ), std::max(L.P.cap_f, L.Q.cap_f), L.sc);
  L.nn = a.take<int>(nP);
  L.d1 = a.take<float>(nP);
  L.nb = hyp_blocks(H);
  L.blk_cnt = a.take<int>((size_t)L.nb + 2);
  L.blk_off = a.take<int>((size_t)L.nb + 2);
  L.blk_scan = a.take<int>((size_t)scan_scratch_ints(L.nb));
  L.hyp_local = a.take<int>((size_t)hyp_local_ints(H));
  L.surv_cap = surv_cap_for(H);
  L.surv = a.take<int>(L.surv_cap);
  L.pose = a.take<float>((size_t)12 * L.surv_cap);
  L.ok = a.take<uint8_t>(L.surv_cap);
  L.count = a.take<int>(L.surv_cap);
  L.sum = a.take<unsigned long long>(L.surv_cap);
  L.ref_part = a.take<double>((size_t)refine_partial_doubles());
  L.seeds = a.take<int>(nP);
  L.fpose = a.take<float>(12);
  L.fcount = a.take<int>(1);
  L.fsum = a.take<unsigned long long>(1);
  L.st = a.take<RansacState>(1);
  L.cls = a.take<ClsParams>(1);
  L.in_bits = a.take<unsigned>(kClsCapWords);
  L.near_bits = a.take<unsigned>(kClsCapWords);
  L.sel = a.take<uint8_t>(L.surv_cap);
  L.rest = a.take<uint8_t>(L.surv_cap);
  L.reach = a.take<uint8_t>(L.surv_cap);
  L.tie = a.take<uint8_t>(L.surv_cap);
  L.amb = a.take<int>(L.surv_cap);
  L.count2 = a.take<int>(L.surv_cap);
  L.tie_list = a.take<int>(L.surv_cap);
  L.prog = a.take<unsigned long long>(L.surv_cap);
  L.c0 = a.take<int>(1);
  L.tc_ws = a.take<char>(precision != LSR_MATCH_FP32 ? tc_workspace_bytes(nP, nQ, precision == LSR_MATCH_BF16)
                                                      : fp32_workspace_bytes(nP, nQ));
  L.cap_s = L.Q.cap_e;
  L.gs = a.take<GridParams>(1);
  L.start_s = a.take<int>((size_t)L.cap_s + 1);
  L.Xs = a.take<float4>(nQ);
}

int set_err(lsr_ctx *c, int code, const char *msg) {
  if (c) c->last_error = msg ? msg : lsr_error_string(code);
  return code;
}

int cuda_err(lsr_ctx *c, cudaError_t e, const char *where) {
  if (e == cudaSuccess) return LSR_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  if (c) {
    c->last_error = buf;
    if (e == cudaErrorIllegalAddress || e == cudaErrorLaunchFailure || e == cudaErrorIllegalInstruction ||
        e == cudaErrorMisalignedAddress || e == cudaErrorHardwareStackError)
      c->broken = true;
  }
  return e == cudaErrorMemoryAllocation ? LSR_E_OOM : LSR_E_CUDA;
}

#define TRY_CUDA(ctx, call, where)                       \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return cuda_err(ctx, e__, where); \
  } while (0)

// Checked build: the first bounds-check violation recorded by any unit since
// the last report becomes LSR_E_CHECK; the normal build's readers report none.
int check_report(lsr_ctx *c) {
  static cudaError_t (*const readers[])(CheckReport *) = {check_read_features, check_read_match,
                                                          check_read_match_tc, check_read_ransac,
                                                          check_read_classify, check_read_refine,
                                                          check_read_nn,       check_read_implicit};
  static const char *const units[] = {"features", "match", "match_tc", "ransac",
                                      "classify", "refine", "nn",       "implicit"};
  constexpr int kUnits = (int)(sizeof(units) / sizeof(units[0]));
  static const char *const sites[] = {"?", "grid row", "grid cell", "grid point", "hypothesis sample",
                                      "hypothesis match", "matcher row", "matcher query", "probe"};
  int rc = LSR_OK;
  for (int u = 0; u < kUnits; ++u) {
    CheckReport r{0, 0, 0};
    cudaError_t e = readers[u](&r);
    if (e != cudaSuccess) return cuda_err(c, e, "check words");
    if (r.site && rc == LSR_OK) {
      char buf[200];
      snprintf(buf, sizeof(buf), "bounds check failed in %s at the %s index: %lld outside [0, %lld)", units[u],
               r.site < 9 ? sites[r.site] : "?", r.index, r.bound);
      rc = set_err(c, LSR_E_CHECK, buf);
    }
  }
  return rc;
}

#define SYNC_CHECKED(ctx, stream)                                     \
  do {                                                                \
    TRY_CUDA(ctx, cudaStreamSynchronize(stream), "sync");             \
    int rc_chk__ = check_report(ctx);                                 \
    if (rc_chk__) return rc_chk__;                                    \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Page-locked host memory: copies from it can be captured into a CUDA graph.
bool is_pinned_host_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeHost;
}

// Injected allocation failure (test hook): consumes one pending failure.
bool injected_alloc_failure(lsr_ctx *c) {
  if (c->inject_alloc <= 0) return false;
  --c->inject_alloc;
  return true;
}

// The matcher's fault settings: a pending injected stall (20 ms wait limit,
// the producer issues nothing), else the defaults.
TcFault take_tc_fault(lsr_ctx *c) {
  TcFault f;
  if (c->inject_stall > 0) {
    --c->inject_stall;
    f.wait_ns = 20000000ull;
    f.stall = 1;
  }
  return f;
}

int ensure_ws(lsr_ctx *c, size_t bytes) {
  if (bytes <= c->ws_cap) return LSR_OK;
  if (injected_alloc_failure(c)) return set_err(c, LSR_E_OOM, "device workspace allocation failed (injected)");
  TRY_CUDA(c, cudaStreamSynchronize(c->stream), "workspace sync");
  if (c->ws) cudaFree(c->ws);
  c->ws = nullptr;
  c->ws_cap = 0;
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&c->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->ws = nullptr;
    return set_err(c, LSR_E_OOM, "device workspace allocation failed");
  }
  c->ws_cap = want;
  return LSR_OK;
}

int ensure_host_slots(lsr_ctx *c, int n) {
  if (n <= c->st_host_cap) return LSR_OK;
  c->gkey.clear();  // a captured batch copies its results into the old slots
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->box_host) cudaFreeHost(c->box_host);
  c->st_host = nullptr;
  c->box_host = nullptr;
  c->st_host_cap = 0;
  if (cudaMallocHost(&c->st_host, sizeof(RansacState) * n) != cudaSuccess ||
      cudaMallocHost(&c->box_host, sizeof(float) * 2 * kBox * n) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, LSR_E_OOM, "pinned host allocation failed");
  }
  c->st_host_cap = n;
  return LSR_OK;
}

bool valid_precision(int p) { return p == LSR_MATCH_FP32 || p == LSR_MATCH_BF16 || p == LSR_MATCH_BF16_PLAIN; }

int check_params(const lsr_params *p) {
  if (!(p->r_normal > 0.f && p->r_feature > 0.f && p->eps_inlier > 0.f && p->tau > 0.f && p->tau <= 1.f &&
        p->cos_normal >= -1.f && p->cos_normal <= 1.f && p->min_inlier_ratio >= 0.f && p->mu_scale > 0.f &&
        p->refine_iters >= 0 && p->refine_iters <= 10000 && p->refine_levels >= 1 &&
        p->refine_levels <= kMaxLevels && p->n_hypotheses >= 1 &&
        p->n_hypotheses <= 2147483647LL && valid_precision(p->match_precision)))
    return LSR_E_ARG;
  if (p->eps_inlier > 10.f) return LSR_E_ARG;  // fixed-point inlier sums assume eps^2 * |P| << 2^23
  if (p->batch_streams < 0 || p->batch_streams > 16 || (p->batch_graph != 0 && p->batch_graph != 1) ||
      p->match_tile < 0 || p->match_tile > 2)
    return LSR_E_ARG;
  if ((p->nn_mode != LSR_NN_EXACT && p->nn_mode != LSR_NN_SINGLE_CELL) ||
      (p->normal_mode != LSR_NORMALS_SAMPLES && p->normal_mode != LSR_NORMALS_INLIERS))
    return LSR_E_ARG;
  return LSR_OK;
}

constexpr int64_t kMaxPoints = (int64_t)1 << 26;

// ---------------------------------------------------------------- small kernels
__global__ void k_pack(const float *xyz, int n, float4 *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __int_as_float(i));
}
__global__ void k_iota(int *p, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}
// internal-order normals from caller-order normals (zero normal = invalid)
__global__ void k_gather_normals(const float *nrm, const float4 *X, int n, float4 *N) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int o = __float_as_int(X[k].w);
    float a = nrm[3 * o], b = nrm[3 * o + 1], c = nrm[3 * o + 2];
    N[k] = make_float4(a, b, c, (a == 0.f && b == 0.f && c == 0.f) ? -1.f : 0.f);
  }
}
__global__ void k_valid_normals(const uint8_t *valid, int n, float4 *N) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    N[k] = make_float4(0.f, 0.f, 1.f, valid[k] ? 0.f : -1.f);
}
__global__ void k_gather_rows(const float *src, int src_stride, const float4 *X, int n, float *dst) {
  // dst (internal, stride kDS) <- src (caller order, stride src_stride, 33 used)
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * kDS;
       t += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(t / kDS), b = (int)(t - (int64_t)k * kDS);
    int o = X ? __float_as_int(X[k].w) : k;
    dst[t] = b < kD ? src[(size_t)o * src_stride + b] : 0.f;
  }
}
__global__ void k_scatter_rows(const float *src, const float4 *X, int n, float *dst) {
  // dst (caller order, stride 33) <- src (internal, stride kDS)
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * kD;
       t += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(t / kD), b = (int)(t - (int64_t)k * kD);
    int o = __float_as_int(X[k].w);
    dst[(size_t)o * kD + b] = src[(size_t)k * kDS + b];
  }
}
__global__ void k_scatter_normals(const float4 *N, const int *cnt, const float4 *X, int n, float *nrm, int32_t *count,
                                  float *curv) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int o = __float_as_int(X[k].w);
    float4 v = N[k];
    if (nrm) nrm[3 * o] = v.x, nrm[3 * o + 1] = v.y, nrm[3 * o + 2] = v.z;
    if (count) count[o] = cnt[k];
    if (curv) curv[o] = v.w;
  }
}
__global__ void k_scatter_int(const int *src, const float4 *X, int n, int32_t *dst) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    dst[__float_as_int(X[k].w)] = src[k];
}
__global__ void k_sum_to_double(const unsigned long long *s, int n, double *d) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) d[k] = (double)s[k] / kFixScale;
}
int nblk(int64_t n, int t = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, kSms * 32)); }

// Build the feature-radius grid (internal order) and, optionally, the
// normal-radius and eps grids of one cloud.
cudaError_t build_cloud(const float *xyz, CloudLayout &c, float r_f, float r_n, float eps, bool normal_grid,
                        bool eps_grid, const ScratchLayout &sc, cudaStream_t s) {
  LSR_CUDA_TRY(launch_bbox_xyz(xyz, c.n, c.box_part, bbox_blocks(c.n), c.box, s));
  LSR_CUDA_TRY(launch_grid_params(c.box, r_f, c.n, c.cap_f, c.gf, s));
  LSR_CUDA_TRY(build_grid_xyz(xyz, c.n, c.gf, c.cap_f, c.start_f, c.X, c.inv, sc.g, s));
  if (normal_grid) {
    LSR_CUDA_TRY(launch_grid_params(c.box, r_n, c.n, c.cap_n, c.gn, s));
    LSR_CUDA_TRY(build_grid_f4(c.X, c.n, c.gn, c.cap_n, c.start_n, c.Xn, sc.g, s));
  }
  if (eps_grid) {
    LSR_CUDA_TRY(launch_grid_params(c.box, eps, c.n, c.cap_e, c.ge, s));
    LSR_CUDA_TRY(build_grid_f4(c.X, c.n, c.ge, c.cap_e, c.start_e, c.Xe, sc.g, s));
    LSR_CUDA_TRY(build_nbmask(c.ge, c.start_e, c.cap_e, c.mask_e, s));
  }
  return cudaSuccess;
}

// Graduated refinement (levels l = 0..L-1, radius eps * 2^(L-1-l)) from the
// pose in st. XP: P in internal order with caller indices in w; Q: caller-order
// xyz on the device; (ge, start_e, Xe): Q's eps grid for the finest level.
cudaError_t enqueue_refine(const float4 *XP, const float *P, int nP, const float *Q, int nQ, const float *boxQ,
                           const GridParams *ge, const int *start_e, const float4 *Xe, const LevelLayout &V, float eps,
                           float mu_scale, int iters, RansacState *st, double *part, int *seeds,
                           const ScratchLayout &sc, cudaStream_t s, bool chain) {
  int L = V.levels;
  LSR_CUDA_TRY(refine_reset_tickets(part, s));
  for (int l = 0; l < L; ++l) {
    float e = eps * (float)(1 << (L - 1 - l));
    float mu = mu_scale * e * e;
    // P at this level: every sP-th caller point, compacted (or all of X)
    const float4 *xp = XP;
    int np = nP;
    if (V.sP[l] > 1) {
      LSR_CUDA_TRY(launch_subsample(P, nP, V.sP[l], V.Psub[l], s));
      xp = V.Psub[l], np = V.nsubP[l];
    }
    const GridParams *g = ge;
    const int *st0 = start_e;
    const float4 *xs = Xe;
    if (l + 1 < L) {
      LSR_CUDA_TRY(launch_subsample(Q, nQ, V.sQ[l], V.Qsub[l], s));
      LSR_CUDA_TRY(launch_grid_params(boxQ, e, V.nsub[l], V.cap[l], V.g[l], s));
      LSR_CUDA_TRY(build_grid_f4(V.Qsub[l], V.nsub[l], V.g[l], V.cap[l], V.start[l], V.Xs[l], sc.g, s));
      LSR_CUDA_TRY(build_nbmask(V.g[l], V.start[l], V.cap[l], V.mask[l], s));
      g = V.g[l], st0 = V.start[l], xs = V.Xs[l];
    }
    LSR_CUDA_TRY(launch_refine_level_begin(st, s));
    LSR_CUDA_TRY(cudaMemsetAsync(seeds, 0xff, sizeof(int) * (size_t)np, s));  // no neighbour yet at this level
    for (int it = 0; it < iters; ++it)
      LSR_CUDA_TRY(launch_refine_step(xp, np, 1, g, st0, xs, e, mu, iters, st, part, seeds, chain && it > 0, s));
  }
  return cudaSuccess;
}

struct Timer {
  lsr_ctx *c;
  int k = 0;
  void mark() {
    if (c->profiling && k < 9) cudaEventRecord(c->ev[k++], c->stream);
  }
};

int size_bucket(int n) {
  int b = 0;
  while (b < 31 && (1 << b) < n) ++b;
  return b;
}

// Tensor-core matcher tile shape for nP queries: the parameter, else the
// autotuner's choice for the size bucket, else the static default.
int match_tile_for(const lsr_ctx *c, int nP) {
  if (c->prm.match_tile) return c->prm.match_tile;
  int t = c->tile_choice[size_bucket(nP)];
  return t ? t : tc_default_tile(nP);
}

// The registration of one pair, enqueued on stream s. Results stay in L.st.
// chain: refinement steps as programmatic dependent launches (one stream at a
// time only: with pairs on concurrent streams, steps waiting for their
// predecessor would hold SM slots the other streams need).
int enqueue_pair(lsr_ctx *c, const PairLayout &L, const float *P, const float *Q, const float *vpP, const float *vpQ,
                 uint64_t pair_id, Timer &tm, cudaStream_t s, bool chain) {
  const lsr_params &p = c->prm;
  int nP = L.P.n, nQ = L.Q.n;
  tm.mark();
  TRY_CUDA(c, cudaMemsetAsync(L.st, 0, sizeof(RansacState), s), "memset state");
  CloudLayout Pc = L.P, Qc = L.Q;
  TRY_CUDA(c, build_cloud(P, Pc, p.r_feature, p.r_normal, p.eps_inlier, true, false, L.sc, s), "grids P");
  TRY_CUDA(c, build_cloud(Q, Qc, p.r_feature, p.r_normal, p.eps_inlier, true, true, L.sc, s), "grids Q");
  tm.mark();
  float3 vp_p = vpP ? make_float3(vpP[0], vpP[1], vpP[2]) : make_float3(0.f, 0.f, 0.f);
  float3 vp_q = vpQ ? make_float3(vpQ[0], vpQ[1], vpQ[2]) : make_float3(0.f, 0.f, 0.f);
  TRY_CUDA(c, launch_normals(Pc.X, nP, Pc.gn, Pc.start_n, Pc.Xn, p.r_normal, vp_p, Pc.N, nullptr, s), "normals P");
  TRY_CUDA(c, launch_normals(Qc.X, nQ, Qc.gn, Qc.start_n, Qc.Xn, p.r_normal, vp_q, Qc.N, nullptr, s), "normals Q");
  tm.mark();
  TRY_CUDA(c, launch_spfh(Pc.X, Pc.N, nP, Pc.gf, Pc.start_f, p.r_feature, Pc.S, nullptr, Pc.F, s), "spfh P");
  TRY_CUDA(c, launch_spfh(Qc.X, Qc.N, nQ, Qc.gf, Qc.start_f, p.r_feature, Qc.S, nullptr, Qc.F, s), "spfh Q");
  TRY_CUDA(c, launch_fpfh(Pc.X, Pc.N, Pc.S, nP, Pc.gf, Pc.start_f, p.r_feature, Pc.F, s), "fpfh P");
  TRY_CUDA(c, launch_fpfh(Qc.X, Qc.N, Qc.S, nQ, Qc.gf, Qc.start_f, p.r_feature, Qc.F, s), "fpfh Q");
  tm.mark();
  if (p.match_precision != LSR_MATCH_FP32)
    TRY_CUDA(c,
             launch_match_bf16(Pc.F, nP, Qc.F, nQ, p.match_precision == LSR_MATCH_BF16, match_tile_for(c, nP), L.tc_ws,
                               L.nn, L.d1,
                               &L.st->match_fallbacks, &L.st->match_err, nullptr, s, take_tc_fault(c)),
             "match");
  else
    TRY_CUDA(c,
             launch_match_fp32(Pc.F, nP, Qc.F, nQ, L.tc_ws, L.nn, L.d1, s,
                               c->profiling ? &L.st->match_terms : nullptr),
             "match");
  tm.mark();
  TRY_CUDA(c,
           launch_hypotheses(Pc.X, Pc.inv, Pc.N, nP, Qc.X, Qc.N, nQ, L.nn, nullptr, nullptr, p.n_hypotheses, p.seed,
                             pair_id, p.tau, L.blk_cnt, L.blk_off, L.blk_scan, L.surv, L.surv_cap, L.st,
                             L.hyp_local, s),
           "hypotheses");
  tm.mark();
  // with the per-inlier normal check the sampled pairs are not checked (a
  // cosine threshold below -1 passes every hypothesis)
  const bool inlier_normals = p.normal_mode == LSR_NORMALS_INLIERS;
  TRY_CUDA(c,
           launch_rigid_survivors(Pc.X, Pc.inv, Pc.N, nP, Qc.X, Qc.N, L.nn, L.surv, L.st, p.seed, pair_id,
                                  inlier_normals ? -2.f : p.cos_normal, L.pose, L.ok, &L.st->n_normal_ok, s),
           "rigid");
  if (p.nn_mode != LSR_NN_EXACT || inlier_normals) {
    // variant consensus: every ok survivor counted with the single-cell lookup
    // and/or the per-inlier normal check (no classification bounds)
    const bool single = p.nn_mode == LSR_NN_SINGLE_CELL;
    const GridParams *g = Qc.ge;
    const int *gstart = Qc.start_e;
    const float4 *gx = Qc.Xe;
    if (single) {
      TRY_CUDA(c, launch_cell_grid_params(Qc.box, p.eps_inlier, nQ, L.cap_s, L.gs, s), "single-cell grid");
      TRY_CUDA(c, build_grid_f4(Qc.X, nQ, L.gs, L.cap_s, L.start_s, L.Xs, L.sc.g, s), "single-cell grid");
      g = L.gs, gstart = L.start_s, gx = L.Xs;
    }
    TRY_CUDA(c, cudaMemsetAsync(L.count, 0, sizeof(int) * L.surv_cap, s), "memset count");
    TRY_CUDA(c, cudaMemsetAsync(L.sum, 0, sizeof(unsigned long long) * L.surv_cap, s), "memset sum");
    TRY_CUDA(c,
             launch_consensus_variant(Pc.Xn, nP, Pc.N, g, gstart, gx, Qc.N, nQ, L.pose, L.ok, &L.st->n_surv,
                                      p.eps_inlier, single, inlier_normals, p.cos_normal, L.count, L.sum, s),
             "consensus variant");
    tm.mark();
    TRY_CUDA(c, launch_select(L.surv, L.count, L.sum, L.ok, L.pose, nP, p.min_inlier_ratio, L.st, s), "select");
  } else {
    // Inlier-count bounds of every survivor from the voxel classification of Q;
    // exact counts of the 32 largest upper bounds (on a subsample of P for a
    // large P) give C; exact counts of the others whose upper bound reaches C;
    // distance sums of the top ties. No survivor left out can be selected. P is read in normal-grid order (5 cm
    // cells): the counts and fixed-point sums do not depend on the order, and
    // a warp's points then land on fewer table words.
    TRY_CUDA(c, launch_cls_build(Qc.box, p.eps_inlier, Qc.X, nQ, L.cls, L.in_bits, L.near_bits, s), "classify");
    TRY_CUDA(c, cudaMemsetAsync(L.count, 0, sizeof(int) * L.surv_cap, s), "memset count");
    TRY_CUDA(c, cudaMemsetAsync(L.amb, 0, sizeof(int) * L.surv_cap, s), "memset count");
    TRY_CUDA(c, cudaMemsetAsync(L.count2, 0, sizeof(int) * L.surv_cap, s), "memset count");
    TRY_CUDA(c, cudaMemsetAsync(L.sum, 0, sizeof(unsigned long long) * L.surv_cap, s), "memset sum");
    // Large P: the 32 largest upper bounds on every 16th point pick the
    // hypotheses counted exactly first; their best count c0 then lets the
    // full bounds pass leave out every hypothesis whose upper bound falls
    // below c0 part-way (it can neither win nor tie).
    const bool prepass = nP >= kConsensusPrepassMin;
    if (prepass) {
      TRY_CUDA(c,
               launch_consensus_bounds(Pc.Xn, nP, kConsensusPrepassStride, L.cls, L.in_bits, L.near_bits, L.pose, L.ok,
                                       &L.st->n_surv, L.count, L.amb, nullptr, nullptr, s),
               "consensus estimate");
      TRY_CUDA(c, launch_top_upper(L.count, L.amb, L.ok, &L.st->n_surv, 32, L.sel, s), "top");
      TRY_CUDA(c,
               launch_consensus_count(Pc.Xn, nP, L.cls, L.in_bits, L.near_bits, Qc.ge, Qc.start_e, Qc.Xe, L.pose,
                                      L.sel, &L.st->n_surv, 0, p.eps_inlier, L.count2, s),
               "consensus top");
      TRY_CUDA(c, launch_sel_max(L.count2, L.sel, &L.st->n_surv, L.c0, s), "consensus bar");
      TRY_CUDA(c, cudaMemsetAsync(L.count, 0, sizeof(int) * L.surv_cap, s), "memset count");
      TRY_CUDA(c, cudaMemsetAsync(L.amb, 0, sizeof(int) * L.surv_cap, s), "memset count");
      TRY_CUDA(c, cudaMemsetAsync(L.prog, 0, sizeof(unsigned long long) * L.surv_cap, s), "memset count");
    }
    TRY_CUDA(c,
             launch_consensus_bounds(Pc.Xn, nP, 1, L.cls, L.in_bits, L.near_bits, L.pose, L.ok, &L.st->n_surv, L.count,
                                     L.amb, prepass ? L.c0 : nullptr, prepass ? L.prog : nullptr, s),
             "consensus bounds");
    if (!prepass) {
      TRY_CUDA(c, launch_top_upper(L.count, L.amb, L.ok, &L.st->n_surv, 32, L.sel, s), "top");
      TRY_CUDA(c,
               launch_consensus_count(Pc.Xn, nP, L.cls, L.in_bits, L.near_bits, Qc.ge, Qc.start_e, Qc.Xe, L.pose,
                                      L.sel, &L.st->n_surv, 0, p.eps_inlier, L.count2, s),
               "consensus top");
      TRY_CUDA(c, launch_sel_max(L.count2, L.sel, &L.st->n_surv, L.c0, s), "consensus bar");
    }
    TRY_CUDA(c, launch_reach_rest(L.count, L.amb, L.count2, L.sel, L.ok, &L.st->n_surv, L.rest, L.reach, s), "reach");
    // the others that may reach c0, each given up on once it no longer can
    TRY_CUDA(c, cudaMemsetAsync(L.prog, 0, sizeof(unsigned long long) * L.surv_cap, s), "memset count");
    TRY_CUDA(c,
             launch_consensus_count_bar(Pc.Xn, nP, L.cls, L.in_bits, L.near_bits, Qc.ge, Qc.start_e, Qc.Xe, L.pose,
                                        L.rest, &L.st->n_surv, p.eps_inlier, L.count2, L.c0, L.count, L.amb, L.prog,
                                        s),
             "consensus reach");
    TRY_CUDA(c, launch_reach_mask(L.count2, nullptr, L.reach, &L.st->n_surv, L.tie, &L.st->n_tie, L.tie_list, s),
             "ties");
    // (the exact kernel adds its counts too: into amb, no longer needed)
    TRY_CUDA(c,
             launch_consensus(Pc.Xn, nP, Qc.ge, Qc.start_e, Qc.Xe, L.pose, nullptr, &L.st->n_tie, 0, p.eps_inlier,
                              L.amb, L.sum, s, c->cons_lanes, L.tie_list),
             "consensus sums");
    tm.mark();
    TRY_CUDA(c, launch_select(L.surv, L.count2, L.sum, L.reach, L.pose, nP, p.min_inlier_ratio, L.st, s), "select");
  }
  TRY_CUDA(c, launch_refine_init(L.st, Pc.box, nullptr, s), "refine init");
  float eps = p.eps_inlier;
  TRY_CUDA(c,
           enqueue_refine(Pc.X, P, nP, Q, nQ, Qc.box, Qc.ge, Qc.start_e, Qc.Xe, L.lv, eps, p.mu_scale, p.refine_iters,
                          L.st, L.ref_part, L.seeds, L.sc, s, chain),
           "refine");
  TRY_CUDA(c, launch_final_pose(L.st, L.fpose, s), "final pose");
  TRY_CUDA(c, cudaMemsetAsync(L.fcount, 0, sizeof(int), s), "memset fcount");
  TRY_CUDA(c, cudaMemsetAsync(L.fsum, 0, sizeof(unsigned long long), s), "memset fsum");
  TRY_CUDA(c,
           launch_consensus(Pc.X, nP, Qc.ge, Qc.start_e, Qc.Xe, L.fpose, nullptr, nullptr, 1, eps, L.fcount, L.fsum, s,
                            c->cons_lanes),
           "final count");
  TRY_CUDA(c, launch_final_count(L.fcount, L.fsum, L.st, s), "final count");
  tm.mark();
  return LSR_OK;
}

void fill_result(const RansacState &st, const float *boxP, const float *boxQ, lsr_result *r) {
  memset(r, 0, sizeof(*r));
  bool ok = st.status == 0;
  for (int i = 0; i < 16; ++i) {
    r->T[i] = ok ? st.T[i] : (i % 5 == 0 ? 1.0 : 0.0);
    r->T_hyp[i] = ok ? st.T_hyp[i] : (i % 5 == 0 ? 1.0 : 0.0);
  }
  r->inliers = st.final_count;
  r->hyp_inliers = st.best_count;
  r->survivors = st.n_surv_total;
  r->n_normal_ok = st.n_normal_ok;
  r->best_h = st.best >= 0 ? st.best_h : -1;
  r->match_fallbacks = st.match_fallbacks;
  r->match_terms = (int64_t)st.match_terms;
  r->fitness = st.final_count > 0 ? (float)(st.final_sumd2 / st.final_count) : 0.f;
  r->hyp_fitness = st.best_fit;
  r->status = ok ? LSR_STATUS_ALIGNED : LSR_STATUS_NO_ALIGNMENT;
  r->refine_iters_done = st.iters_done;
  (void)boxP;
  (void)boxQ;
}

// Stage a cloud to the device if it lives in host memory.
int stage_input(lsr_ctx *c, const float *src, int64_t n, float *dst, const float **out, cudaStream_t s = nullptr) {
  if (is_device_ptr(src)) {
    *out = src;
    return LSR_OK;
  }
  TRY_CUDA(c, cudaMemcpyAsync(dst, src, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s ? s : c->stream), "H2D");
  *out = dst;
  return LSR_OK;
}

int guard(lsr_ctx *c) {
  if (!c) return LSR_E_STATE;
  if (c->broken) return set_err(c, LSR_E_STATE, "context unusable after a device fault");
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, LSR_E_CUDA, "cudaSetDevice failed");
  }
  return LSR_OK;
}

// Generic copy of a result array to a caller pointer (device or host).
int copy_out(lsr_ctx *c, void *dst, const void *src, size_t bytes) {
  TRY_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream), "copy out");
  return LSR_OK;
}

// ---------------------------------------------------------------- batches
// A batch of pairs (lsr_register_batch). Pairs run on S worker streams, each
// with its own workspace, assigned longest-first to the least loaded stream;
// the context stream forks to the workers and joins them. The same enqueue
// can be captured into one CUDA graph and replayed.
struct BatchIn {
  int n;
  const float *const *P;
  const int64_t *nP;
  const float *const *Q;
  const int64_t *nQ;
  const float *vp;
  uint64_t pair0;
};

size_t pair_bytes(const lsr_ctx *c, int64_t nP, int64_t nQ) {
  Arena m(nullptr);
  PairLayout L;
  plan_pair(m, (int)nP, (int)nQ, true, true, c->prm.n_hypotheses, c->prm.refine_levels, c->prm.match_precision, L);
  return m.off;
}

int ensure_lanes(lsr_ctx *c, int S, size_t bytes) {
  while ((int)c->lanes.size() < S) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, LSR_E_CUDA, "stream creation failed");
    }
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamDestroy(st);
      return set_err(c, LSR_E_CUDA, "event creation failed");
    }
    c->lanes.push_back(st);
    c->lane_done.push_back(ev);
    c->lane_ws.push_back(nullptr);
    c->lane_cap.push_back(0);
  }
  if (!c->fork && cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    c->fork = nullptr;
    return set_err(c, LSR_E_CUDA, "event creation failed");
  }
  for (int l = 0; l < S; ++l) {
    if (c->lane_cap[l] >= bytes) continue;
    TRY_CUDA(c, cudaStreamSynchronize(c->lanes[l]), "workspace sync");
    if (c->lane_ws[l]) cudaFree(c->lane_ws[l]);
    c->lane_ws[l] = nullptr;
    c->lane_cap[l] = 0;
    c->gkey.clear();  // a captured batch points into the old workspace
    size_t want = bytes + bytes / 8;
    if (injected_alloc_failure(c)) return set_err(c, LSR_E_OOM, "batch workspace allocation failed (injected)");
    if (cudaMalloc(&c->lane_ws[l], want) != cudaSuccess) {
      cudaGetLastError();
      c->lane_ws[l] = nullptr;
      return set_err(c, LSR_E_OOM, "batch workspace allocation failed");
    }
    c->lane_cap[l] = want;
  }
  return LSR_OK;
}

// Longest processing time first: descending nP * nQ + nP (ties by index),
// each pair to the stream with the least work so far.
std::vector<std::vector<int>> assign_pairs(const BatchIn &b, int m, int S) {
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  auto cost = [&](int i) { return (double)b.nP[i] * (double)b.nQ[i] + 1e4 * (double)b.nP[i]; };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  std::vector<std::vector<int>> lanes(S);
  std::vector<double> load(S, 0.0);
  for (int i : order) {
    int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[l].push_back(i);
    load[l] += cost(i);
  }
  return lanes;
}

int enqueue_batch(lsr_ctx *c, const BatchIn &b, const std::vector<std::vector<int>> &lanes) {
  const int S = (int)lanes.size();
  TRY_CUDA(c, cudaEventRecord(c->fork, c->stream), "fork");
  for (int l = 0; l < S; ++l) {
    cudaStream_t s = c->lanes[l];
    TRY_CUDA(c, cudaStreamWaitEvent(s, c->fork, 0), "fork");
    for (int i : lanes[l]) {
      Arena a(c->lane_ws[l]);
      PairLayout L;
      plan_pair(a, (int)b.nP[i], (int)b.nQ[i], true, true, c->prm.n_hypotheses, c->prm.refine_levels,
                c->prm.match_precision, L);
      const float *dP, *dQ;
      int rc;
      if ((rc = stage_input(c, b.P[i], b.nP[i], L.P.src, &dP, s))) return rc;
      if ((rc = stage_input(c, b.Q[i], b.nQ[i], L.Q.src, &dQ, s))) return rc;
      Timer t{c};
      t.k = 9;  // no per-stage timing inside batches
      if ((rc = enqueue_pair(c, L, dP, dQ, b.vp ? b.vp + 6 * i : nullptr, b.vp ? b.vp + 6 * i + 3 : nullptr,
                             b.pair0 + i, t, s, false)))
        return rc;
      TRY_CUDA(c, cudaMemcpyAsync(&c->st_host[i], L.st, sizeof(RansacState), cudaMemcpyDeviceToHost, s), "D2H");
      TRY_CUDA(c,
               cudaMemcpyAsync(&c->box_host[2 * kBox * i], L.P.box, sizeof(float) * kBox, cudaMemcpyDeviceToHost, s),
               "D2H");
      TRY_CUDA(c,
               cudaMemcpyAsync(&c->box_host[2 * kBox * i + kBox], L.Q.box, sizeof(float) * kBox,
                               cudaMemcpyDeviceToHost, s),
               "D2H");
    }
    TRY_CUDA(c, cudaEventRecord(c->lane_done[l], s), "join");
    TRY_CUDA(c, cudaStreamWaitEvent(c->stream, c->lane_done[l], 0), "join");
  }
  return LSR_OK;
}

// Signature of everything a captured batch graph bakes in.
std::string batch_key(const lsr_ctx *c, const BatchIn &b, const std::vector<std::vector<int>> &lanes) {
  std::string k;
  auto put = [&](const void *p, size_t n) { k.append(reinterpret_cast<const char *>(p), n); };
  put(&c->prm, sizeof(c->prm));
  put(&b.n, sizeof(b.n));
  put(&b.pair0, sizeof(b.pair0));
  for (int i = 0; i < b.n; ++i) {
    put(&b.P[i], sizeof(void *));
    put(&b.Q[i], sizeof(void *));
    put(&b.nP[i], sizeof(int64_t));
    put(&b.nQ[i], sizeof(int64_t));
    if (b.vp) put(b.vp + 6 * i, 6 * sizeof(float));
    int t = match_tile_for(c, (int)b.nP[i]);
    put(&t, sizeof(t));
  }
  for (size_t l = 0; l < lanes.size(); ++l) {
    put(&c->lane_ws[l], sizeof(void *));
    int m = (int)lanes[l].size();
    put(&m, sizeof(m));
    for (int i : lanes[l]) put(&i, sizeof(i));
  }
  put(&c->st_host, sizeof(void *));
  put(&c->box_host, sizeof(void *));
  put(&c->cons_lanes, sizeof(int));
  return k;
}

// ---------------------------------------------------------------- autotuner
// Synthetic FPFH-like rows for tuning: three 11-bin sub-histograms, each the
// cube of counter-based uniform numbers normalised to sum 1 (peaked, as
// FPFH of planar-dominated scenes).
__global__ void k_fake_desc(uint64_t seed, int n, float *F) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * 3; t += gridDim.x * blockDim.x) {
    const int row = t / 3, sub = t - 3 * row;
    float v[kNB], sum = 0.f;
    for (int b = 0; b < kNB; ++b) {
      uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(row * kD + sub * kNB + b + 1);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      float u = (float)(z >> 40) * 5.9604645e-8f;
      v[b] = u * u * u;
      sum += v[b];
    }
    for (int b = 0; b < kNB; ++b) F[(size_t)row * kDS + sub * kNB + b] = v[b] / fmaxf(sum, 1e-30f);
    if (sub == 2)
      for (int b = kD; b < kDS; ++b) F[(size_t)row * kDS + b] = 0.f;
  }
}

// Tensor-core tile shape per size bucket: both shapes timed (CUDA events) on
// synthetic descriptors of the largest query count of that bucket in the batch.
int tune_tiles(lsr_ctx *c, const BatchIn &b) {
  if (c->prm.match_precision == LSR_MATCH_FP32 || c->prm.match_tile) return LSR_OK;
  const bool split = c->prm.match_precision == LSR_MATCH_BF16;
  int want[32] = {};
  for (int i = 0; i < b.n; ++i) {
    int k = size_bucket((int)b.nP[i]);
    if (!c->tile_choice[k]) want[k] = std::max(want[k], (int)std::max(b.nP[i], b.nQ[i]));
  }
  cudaStream_t s = c->stream;
  for (int k = 0; k < 32; ++k) {
    const int n = want[k];
    if (!n) continue;
    auto plan = [&](Arena &a, float *&FP, float *&FQ, int *&nn, float *&d1, int *&flags, char *&tws) {
      FP = a.take<float>((size_t)kDS * n);
      FQ = a.take<float>((size_t)kDS * n);
      nn = a.take<int>(n);
      d1 = a.take<float>(n);
      flags = a.take<int>(2);
      tws = a.take<char>(tc_workspace_bytes(n, n, split));
    };
    Arena m(nullptr);
    float *x1, *x2, *x4;
    int *x3, *x5;
    char *x6;
    plan(m, x1, x2, x3, x4, x5, x6);
    int rc;
    if ((rc = ensure_ws(c, m.off))) return rc;
    Arena a(c->ws);
    float *FP, *FQ, *d1;
    int *nn, *flags;
    char *tws;
    plan(a, FP, FQ, nn, d1, flags, tws);
    LSR_LAUNCH(k_fake_desc<<<nblk(3 * n), 256, 0, s>>>(0x243F6A8885A308D3ull, n, FP));
    LSR_LAUNCH(k_fake_desc<<<nblk(3 * n), 256, 0, s>>>(0x13198A2E03707344ull, n, FQ));
    float best_ms = 0.f;
    int best = 0;
    for (int qt = 1; qt <= 2; ++qt) {
      TRY_CUDA(c, launch_match_bf16(FP, n, FQ, n, split, qt, tws, nn, d1, flags, flags + 1, nullptr, s), "tune");
      TRY_CUDA(c, cudaEventRecord(c->ev[0], s), "tune");
      for (int r = 0; r < 2; ++r)
        TRY_CUDA(c, launch_match_bf16(FP, n, FQ, n, split, qt, tws, nn, d1, flags, flags + 1, nullptr, s), "tune");
      TRY_CUDA(c, cudaEventRecord(c->ev[1], s), "tune");
      TRY_CUDA(c, cudaEventSynchronize(c->ev[1]), "tune");
      float ms = 0.f;
      TRY_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]), "tune");
      if (!best || ms < best_ms) best = qt, best_ms = ms;
    }
    c->tile_choice[k] = best;
  }
  return LSR_OK;
}

// Number of batch streams: 1, 2, 4 and 8 timed on the first pairs of the
// batch (their results are discarded; the real run follows).
int tune_streams(lsr_ctx *c, const BatchIn &b, size_t bytes) {
  const int m = std::min(b.n, 16);
  float best_ms = 0.f;
  int best = 0;
  for (int S = 1; S <= 8 && S <= m; S *= 2) {
    int rc;
    if ((rc = ensure_lanes(c, S, bytes))) return rc;
    auto lanes = assign_pairs(b, m, S);
    TRY_CUDA(c, cudaEventRecord(c->ev[0], c->stream), "tune");
    if ((rc = enqueue_batch(c, b, lanes))) return rc;
    TRY_CUDA(c, cudaEventRecord(c->ev[1], c->stream), "tune");
    TRY_CUDA(c, cudaEventSynchronize(c->ev[1]), "tune");
    float ms = 0.f;
    TRY_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]), "tune");
    if (!best || ms < best_ms) best = S, best_ms = ms;
  }
  c->streams_choice = best;
  return LSR_OK;
}

}  // namespace

// ======================================================================= ABI
extern "C" {

void lsr_default_params(lsr_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->r_normal = 0.05f;
  p->r_feature = 0.125f;
  p->eps_inlier = 0.0375f;
  p->tau = 0.9f;
  p->cos_normal = 0.86602540378f;  // cos(30 deg)
  p->min_inlier_ratio = 0.05f;
  p->mu_scale = 1.0f;
  p->refine_iters = 50;
  p->refine_levels = 3;
  p->n_hypotheses = 4000000;
  p->seed = 0;
  p->pair_id = 0;
  p->match_precision = LSR_MATCH_FP32;
}

const char *lsr_error_string(int code) {
  switch (code) {
    case LSR_OK: return "ok";
    case LSR_E_ARG: return "invalid argument";
    case LSR_E_CUDA: return "CUDA error";
    case LSR_E_OOM: return "out of memory";
    case LSR_E_TIMEOUT: return "device wait timed out";
    case LSR_E_STATE: return "context unusable";
    case LSR_E_TOO_LARGE: return "input exceeds the fixed scratch of the allocation-free entry point";
    case LSR_E_CHECK: return "a device bounds check failed (checked build)";
    default: return "unknown error";
  }
}

const char *lsr_last_error(const lsr_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int lsr_create(lsr_ctx **out, const lsr_params *params, int device, void *cuda_stream) {
  if (!out) return LSR_E_ARG;
  *out = nullptr;
  lsr_params p;
  if (params)
    p = *params;
  else
    lsr_default_params(&p);
  if (check_params(&p) != LSR_OK) return LSR_E_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return LSR_E_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return LSR_E_CUDA;
  }
  lsr_ctx *c = new (std::nothrow) lsr_ctx();
  if (!c) return LSR_E_OOM;
  c->device = device;
  c->prm = p;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return LSR_E_CUDA;
    }
    c->own_stream = true;
  }
  if (const char *e = getenv("LSR_CONSENSUS_LANES")) {
    int v = atoi(e);
    if (v == 1 || v == 2 || v == 4 || v == 8 || v == 16) c->cons_lanes = v;
  }
  for (auto &e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      lsr_destroy(c);
      return LSR_E_CUDA;
    }
  *out = c;
  return LSR_OK;
}

int lsr_destroy(lsr_ctx *c) {
  if (!c) return LSR_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (size_t l = 0; l < c->lanes.size(); ++l) {
    cudaStreamSynchronize(c->lanes[l]);
    if (c->lane_ws[l]) cudaFree(c->lane_ws[l]);
    cudaStreamDestroy(c->lanes[l]);
    cudaEventDestroy(c->lane_done[l]);
  }
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->ws) cudaFree(c->ws);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->box_host) cudaFreeHost(c->box_host);
  for (auto &e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c->ktimer;
  cudaGetLastError();
  delete c;
  return LSR_OK;
}

int lsr_set_kernel_timing(lsr_ctx *c, const char *filter) {
  if (!c) return LSR_E_STATE;
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, LSR_E_CUDA, "cudaSetDevice failed");
  }
  if (c->stream) cudaStreamSynchronize(c->stream);
  delete c->ktimer;
  c->ktimer = nullptr;
  if (!filter) return LSR_OK;
  if (strlen(filter) > 200) return set_err(c, LSR_E_ARG, "kernel filter too long");
  c->ktimer = new KernelTimer();
  c->ktimer->filter = filter;
  return LSR_OK;
}

int32_t lsr_kernel_timing_count(const lsr_ctx *c) {
  return c && c->ktimer ? (int32_t)c->ktimer->table.size() : 0;
}

int lsr_kernel_timing_entry(const lsr_ctx *c, int32_t i, const char **name, int64_t *launches, double *total_ms) {
  if (!c) return LSR_E_STATE;
  if (!c->ktimer || i < 0 || i >= (int32_t)c->ktimer->table.size()) return LSR_E_ARG;
  const KernelTimer::Entry &e = c->ktimer->table[(size_t)i];
  if (name) *name = e.name.c_str();
  if (launches) *launches = e.launches;
  if (total_ms) *total_ms = e.ms;
  return LSR_OK;
}

int lsr_set_params(lsr_ctx *c, const lsr_params *p) {
  if (!c) return LSR_E_STATE;
  if (!p || check_params(p) != LSR_OK) return set_err(c, LSR_E_ARG, "parameter out of range");
  c->prm = *p;
  return LSR_OK;
}

int lsr_get_params(const lsr_ctx *c, lsr_params *p) {
  if (!c) return LSR_E_STATE;
  if (!p) return LSR_E_ARG;
  *p = c->prm;
  return LSR_OK;
}

int lsr_checked_build(void) {
#ifdef LSR_CHECKED
  return 1;
#else
  return 0;
#endif
}

int lsr_debug_inject(lsr_ctx *c, int32_t kind, int32_t count) {
  if (!c) return LSR_E_STATE;
  if (count < 0 || count > 1000000) return set_err(c, LSR_E_ARG, "bad injection count");
  switch (kind) {
    case LSR_INJECT_NONE: c->inject_alloc = c->inject_stall = 0; return LSR_OK;
    case LSR_INJECT_ALLOC: c->inject_alloc = count; return LSR_OK;
    case LSR_INJECT_MATCH_STALL: c->inject_stall = count; return LSR_OK;
    case LSR_INJECT_CHECK: {
      if (!lsr_checked_build()) return set_err(c, LSR_E_ARG, "LSR_INJECT_CHECK needs the checked build");
      if (count == 0) return LSR_OK;
      if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, LSR_E_CUDA, "cudaSetDevice failed");
      }
      TRY_CUDA(c, check_probe_arm(c->stream), "arm probe");
      return LSR_OK;
    }
    default: return set_err(c, LSR_E_ARG, "bad injection kind");
  }
}

int lsr_set_profiling(lsr_ctx *c, int enable) {
  if (!c) return LSR_E_STATE;
  c->profiling = enable != 0;
  return LSR_OK;
}

int64_t lsr_workspace_bytes(const lsr_ctx *c) {
  if (!c) return 0;
  size_t b = c->ws_cap;
  for (size_t x : c->lane_cap) b += x;
  return (int64_t)b;
}

uint64_t lsr_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int lsr_transfer_bytes(int64_t nP, int64_t nQ, int64_t *h2d, int64_t *d2h) {
  if (nP < 0 || nQ < 0) return LSR_E_ARG;
  if (h2d) *h2d = (int64_t)sizeof(float) * 3 * (nP + nQ);
  if (d2h) *d2h = (int64_t)(sizeof(RansacState) + 2 * sizeof(float) * kBox);
  return LSR_OK;
}

// Installs the context's kernel timer for the calling thread while a call
// enqueues on the context stream; launches bracketed by a call that fails
// before its synchronisation are dropped.
struct KernelTimerScope {
  KernelTimer *t = nullptr;
  bool done = false;
  KernelTimerScope(lsr_ctx *c, bool on) {
    if (on && c->ktimer) {
      t = c->ktimer;
      t->stream = c->stream;
      t->failed = false;
      g_ktimer = t;
    }
  }
  void collect() {
    if (t) t->collect();
    done = true;
  }
  ~KernelTimerScope() {
    if (!t) return;
    g_ktimer = nullptr;
    if (!done) {
      t->open.clear();
      t->used = 0;
    }
  }
};

static int register_many(lsr_ctx *c, int32_t n, const float *const *P, const int64_t *nP, const float *const *Q,
                         const int64_t *nQ, const float *vp, uint64_t pair0, lsr_result *out) {
  int rc = guard(c);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!P || !nP || !Q || !nQ || !out))) return set_err(c, LSR_E_ARG, "null argument");
  if (n == 0) return LSR_OK;
  int64_t maxP = 0, maxQ = 0;
  for (int i = 0; i < n; ++i) {
    if (!P[i] || !Q[i]) return set_err(c, LSR_E_ARG, "null cloud");
    if (nP[i] < 4 || nQ[i] < 4) return set_err(c, LSR_E_ARG, "a cloud has fewer than 4 points");
    if (nP[i] > kMaxPoints || nQ[i] > kMaxPoints) return set_err(c, LSR_E_ARG, "a cloud has too many points");
    maxP = std::max(maxP, nP[i]);
    maxQ = std::max(maxQ, nQ[i]);
  }
  if ((rc = ensure_host_slots(c, n))) return rc;
  const BatchIn b{n, P, nP, Q, nQ, vp, pair0};
  if ((rc = tune_tiles(c, b))) return rc;
  const size_t bytes = pair_bytes(c, maxP, maxQ);
  int S = c->prm.batch_streams;
  if (!S && n >= 8) {
    if (!c->streams_choice && (rc = tune_streams(c, b, bytes))) return rc;
    S = c->streams_choice;
  }
  S = std::max(1, std::min(S, (int)n));
  const bool graph = c->prm.batch_graph == 1 && n > 1;
  Timer tm{c};
  KernelTimerScope kts(c, S == 1 && !graph);
  if (S == 1 && !graph) {
    // pairs back to back on the context stream, one workspace
    if ((rc = ensure_ws(c, bytes))) return rc;
    for (int i = 0; i < n; ++i) {
      Arena a(c->ws);
      PairLayout L;
      plan_pair(a, (int)nP[i], (int)nQ[i], true, true, c->prm.n_hypotheses, c->prm.refine_levels,
                c->prm.match_precision, L);
      const float *dP, *dQ;
      if ((rc = stage_input(c, P[i], nP[i], L.P.src, &dP))) return rc;
      if ((rc = stage_input(c, Q[i], nQ[i], L.Q.src, &dQ))) return rc;
      Timer t1{c};
      Timer &t = (n == 1) ? tm : t1;
      if (n != 1) t.k = 9;  // per-stage timing only for single pairs
      if ((rc = enqueue_pair(c, L, dP, dQ, vp ? vp + 6 * i : nullptr, vp ? vp + 6 * i + 3 : nullptr, pair0 + i, t,
                             c->stream, true)))
        return rc;
      TRY_CUDA(c, cudaMemcpyAsync(&c->st_host[i], L.st, sizeof(RansacState), cudaMemcpyDeviceToHost, c->stream),
               "D2H");
      TRY_CUDA(c,
               cudaMemcpyAsync(&c->box_host[2 * kBox * i], L.P.box, sizeof(float) * kBox, cudaMemcpyDeviceToHost,
                               c->stream),
               "D2H");
      TRY_CUDA(c,
               cudaMemcpyAsync(&c->box_host[2 * kBox * i + kBox], L.Q.box, sizeof(float) * kBox,
                               cudaMemcpyDeviceToHost, c->stream),
               "D2H");
    }
  } else {
    if ((rc = ensure_lanes(c, S, bytes))) return rc;
    auto lanes = assign_pairs(b, n, S);
    // device or page-locked host inputs: the host-to-device copies become
    // memcpy nodes of the graph, each on its pair's lane just before the pair
    auto capturable = [](const float *x) { return is_device_ptr(x) || is_pinned_host_ptr(x); };
    bool graph_inputs = true;
    for (int i = 0; i < n && graph_inputs; ++i) graph_inputs = capturable(P[i]) && capturable(Q[i]);
    if (graph && graph_inputs) {
      std::string key = batch_key(c, b, lanes);
      if (!c->gexec || key != c->gkey) {
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        c->gkey.clear();
        // the launches of a capture are counted when the graph runs
        const unsigned long long g0 = lsr_launch_count();
        TRY_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed), "capture");
        rc = enqueue_batch(c, b, lanes);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        const unsigned long long captured = lsr_launch_count() - g0;
        __atomic_fetch_sub(&g_launches, captured, __ATOMIC_RELAXED);
        if (rc || e != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
          return rc ? rc : cuda_err(c, e, "capture");
        }
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          c->gexec = nullptr;
          return cuda_err(c, e, "graph instantiate");
        }
        c->gkey = key;
        c->glaunches = captured;
      }
      TRY_CUDA(c, cudaGraphLaunch(c->gexec, c->stream), "graph launch");
      __atomic_fetch_add(&g_launches, c->glaunches, __ATOMIC_RELAXED);
    } else {
      if ((rc = enqueue_batch(c, b, lanes))) return rc;
    }
  }
  SYNC_CHECKED(c, c->stream);
  TRY_CUDA(c, cudaGetLastError(), "kernel");
  kts.collect();
  for (int i = 0; i < n; ++i) {
    if (c->box_host[2 * kBox * i + 6] != 0.f || c->box_host[2 * kBox * i + kBox + 6] != 0.f)
      return set_err(c, LSR_E_ARG, "non-finite input coordinates");
    if (c->st_host[i].match_err) return set_err(c, LSR_E_TIMEOUT, "BF16 matcher timed out waiting on the tensor cores");
    fill_result(c->st_host[i], &c->box_host[2 * kBox * i], &c->box_host[2 * kBox * i + kBox], &out[i]);
  }
  if (n == 1 && c->profiling && tm.k == 8) {  // 8 marks bound the 7 stages
    float tot = 0.f;
    for (int k = 0; k < 7; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]);
      out[0].stage_ms[k] = ms;
      tot += ms;
    }
    out[0].stage_ms[7] = tot;
  }
  return LSR_OK;
}

int lsr_register_pair(lsr_ctx *c, const float *P, int64_t nP, const float *Q, int64_t nQ, const float *vpP,
                      const float *vpQ, lsr_result *out) {
  if (!c) return LSR_E_STATE;
  float vp[6] = {0, 0, 0, 0, 0, 0};
  if (vpP) vp[0] = vpP[0], vp[1] = vpP[1], vp[2] = vpP[2];
  if (vpQ) vp[3] = vpQ[0], vp[4] = vpQ[1], vp[5] = vpQ[2];
  return register_many(c, 1, &P, &nP, &Q, &nQ, vp, c->prm.pair_id, out);
}

int lsr_register_batch(lsr_ctx *c, int32_t n, const float *const *P, const int64_t *nP, const float *const *Q,
                       const int64_t *nQ, const float *vp, lsr_result *out) {
  if (!c) return LSR_E_STATE;
  return register_many(c, n, P, nP, Q, nQ, vp, c->prm.pair_id, out);
}

// ------------------------------------------------------------------ stages
int lsr_stage_normals(lsr_ctx *c, const float *P, int64_t n, const float *vp, float r, float *normals, int32_t *count,
                      float *curvature) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || n < 1 || n > kMaxPoints || !(r > 0.f)) return set_err(c, LSR_E_ARG, "bad argument");
  Arena m(nullptr);
  CloudLayout Cm;
  plan_cloud(m, (int)n, true, true, false, Cm);
  ScratchLayout Sm;
  plan_scratch(m, (int)n, Cm.cap_f, Sm);
  int *cnt_m = m.take<int>(n);
  float *o_n = m.take<float>(3 * n);
  int *o_c = m.take<int>(n);
  float *o_v = m.take<float>(n);
  (void)cnt_m, (void)o_n, (void)o_c, (void)o_v;
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  CloudLayout C;
  plan_cloud(a, (int)n, true, true, false, C);
  ScratchLayout S;
  plan_scratch(a, (int)n, C.cap_f, S);
  int *cnt = a.take<int>(n);
  float *dn = a.take<float>(3 * n);
  int *dc = a.take<int>(n);
  float *dv = a.take<float>(n);
  const float *src;
  if ((rc = stage_input(c, P, n, C.src, &src))) return rc;
  cudaStream_t s = c->stream;
  TRY_CUDA(c, build_cloud(src, C, r, r, r, true, false, S, s), "grids");
  float3 v = vp ? make_float3(vp[0], vp[1], vp[2]) : make_float3(0.f, 0.f, 0.f);
  TRY_CUDA(c, launch_normals(C.X, (int)n, C.gn, C.start_n, C.Xn, r, v, C.N, cnt, s), "normals");
  LSR_LAUNCH(k_scatter_normals<<<nblk(n), 256, 0, s>>>(C.N, cnt, C.X, (int)n, dn, dc, dv));
  TRY_CUDA(c, cudaGetLastError(), "scatter");
  if (normals && (rc = copy_out(c, normals, dn, sizeof(float) * 3 * n))) return rc;
  if (count && (rc = copy_out(c, count, dc, sizeof(int) * n))) return rc;
  if (curvature && (rc = copy_out(c, curvature, dv, sizeof(float) * n))) return rc;
  SYNC_CHECKED(c, s);
  return LSR_OK;
}

static int stage_desc_common(lsr_ctx *c, const float *P, const float *normals, const float *spfh_in, int64_t n, float r,
                             float *out, int32_t *k_out) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || !normals || n < 1 || n > kMaxPoints || !(r > 0.f)) return set_err(c, LSR_E_ARG, "bad argument");
  auto plan = [&](Arena &a, CloudLayout &C, ScratchLayout &S, float *&nrm, float *&sp, float *&o, int *&kk,
                  int *&ko) {
    plan_cloud(a, (int)n, true, true, false, C);
    plan_scratch(a, (int)n, C.cap_f, S);
    nrm = a.take<float>(3 * n);
    sp = a.take<float>(kD * n);
    o = a.take<float>(kD * n);
    kk = a.take<int>(n);
    ko = a.take<int>(n);
  };
  Arena m(nullptr);
  CloudLayout Cm;
  ScratchLayout Sm;
  float *a1, *a2, *a3;
  int *a4, *a5;
  plan(m, Cm, Sm, a1, a2, a3, a4, a5);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  CloudLayout C;
  ScratchLayout S;
  float *nrm, *sp, *o;
  int *kk, *ko;
  plan(a, C, S, nrm, sp, o, kk, ko);
  cudaStream_t s = c->stream;
  const float *src;
  if ((rc = stage_input(c, P, n, C.src, &src))) return rc;
  TRY_CUDA(c, cudaMemcpyAsync(nrm, normals, sizeof(float) * 3 * n, cudaMemcpyDefault, s), "copy normals");
  TRY_CUDA(c, build_cloud(src, C, r, r, r, false, false, S, s), "grids");
  LSR_LAUNCH(k_gather_normals<<<nblk(n), 256, 0, s>>>(nrm, C.X, (int)n, C.N));
  if (!spfh_in) {
    TRY_CUDA(c, launch_spfh(C.X, C.N, (int)n, C.gf, C.start_f, r, C.S, kk, C.F, s), "spfh");
    LSR_LAUNCH(k_scatter_rows<<<nblk(n * kD), 256, 0, s>>>(C.S, C.X, (int)n, o));
    if (k_out) LSR_LAUNCH(k_scatter_int<<<nblk(n), 256, 0, s>>>(kk, C.X, (int)n, ko));
  } else {
    TRY_CUDA(c, cudaMemcpyAsync(sp, spfh_in, sizeof(float) * kD * n, cudaMemcpyDefault, s), "copy spfh");
    LSR_LAUNCH(k_gather_rows<<<nblk(n * kDS), 256, 0, s>>>(sp, kD, C.X, (int)n, C.S));
    TRY_CUDA(c, launch_fpfh(C.X, C.N, C.S, (int)n, C.gf, C.start_f, r, C.F, s), "fpfh");
    LSR_LAUNCH(k_scatter_rows<<<nblk(n * kD), 256, 0, s>>>(C.F, C.X, (int)n, o));
  }
  TRY_CUDA(c, cudaGetLastError(), "stage kernels");
  if ((rc = copy_out(c, out, o, sizeof(float) * kD * n))) return rc;
  if (k_out && !spfh_in && (rc = copy_out(c, k_out, ko, sizeof(int) * n))) return rc;
  SYNC_CHECKED(c, s);
  return LSR_OK;
}

int lsr_stage_spfh(lsr_ctx *c, const float *P, const float *normals, int64_t n, float r, float *spfh, int32_t *k) {
  if (!spfh) return c ? set_err(c, LSR_E_ARG, "null output") : LSR_E_STATE;
  return stage_desc_common(c, P, normals, nullptr, n, r, spfh, k);
}

int lsr_stage_fpfh(lsr_ctx *c, const float *P, const float *normals, const float *spfh, int64_t n, float r,
                   float *fpfh) {
  if (!spfh || !fpfh) return c ? set_err(c, LSR_E_ARG, "null argument") : LSR_E_STATE;
  return stage_desc_common(c, P, normals, spfh, n, r, fpfh, nullptr);
}

int lsr_stage_match(lsr_ctx *c, const float *FP, int64_t nP, const float *FQ, int64_t nQ, int32_t precision,
                    int32_t *nn, float *d1, int64_t *fallbacks) {
  int rc = guard(c);
  if (rc) return rc;
  if (!FP || !FQ || !nn || nP < 1 || nQ < 1 || nP > kMaxPoints || nQ > kMaxPoints)
    return set_err(c, LSR_E_ARG, "bad argument");
  if (!valid_precision(precision)) return set_err(c, LSR_E_ARG, "bad precision");
  const bool tc = precision != LSR_MATCH_FP32, split = precision == LSR_MATCH_BF16;
  auto plan = [&](Arena &a, float *&fp, float *&fq, float *&FPi, float *&FQi, int *&dn, float *&dd, int *&flags,
                  char *&tws) {
    fp = a.take<float>(kD * nP);
    fq = a.take<float>(kD * nQ);
    FPi = a.take<float>(kDS * nP);
    FQi = a.take<float>(kDS * nQ);
    dn = a.take<int>(nP);
    dd = a.take<float>(nP);
    flags = a.take<int>(2);
    tws = a.take<char>(tc ? tc_workspace_bytes((int)nP, (int)nQ, split) : fp32_workspace_bytes((int)nP, (int)nQ));
  };
  Arena m(nullptr);
  float *x1, *x2, *x3, *x4, *x6;
  int *x5, *x7;
  char *x8;
  plan(m, x1, x2, x3, x4, x5, x6, x7, x8);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  float *fp, *fq, *FPi, *FQi, *dd;
  int *dn, *flags;
  char *tws;
  plan(a, fp, fq, FPi, FQi, dn, dd, flags, tws);
  cudaStream_t s = c->stream;
  TRY_CUDA(c, cudaMemcpyAsync(fp, FP, sizeof(float) * kD * nP, cudaMemcpyDefault, s), "copy FP");
  TRY_CUDA(c, cudaMemcpyAsync(fq, FQ, sizeof(float) * kD * nQ, cudaMemcpyDefault, s), "copy FQ");
  LSR_LAUNCH(k_gather_rows<<<nblk(nP * kDS), 256, 0, s>>>(fp, kD, nullptr, (int)nP, FPi));
  LSR_LAUNCH(k_gather_rows<<<nblk(nQ * kDS), 256, 0, s>>>(fq, kD, nullptr, (int)nQ, FQi));
  if (tc)
    TRY_CUDA(c, launch_match_bf16(FPi, (int)nP, FQi, (int)nQ, split, match_tile_for(c, (int)nP), tws, dn, dd, flags, flags + 1,
                                  nullptr, s, take_tc_fault(c)),
             "match");
  else
    TRY_CUDA(c, launch_match_fp32(FPi, (int)nP, FQi, (int)nQ, tws, dn, dd, s), "match");
  int hflags[2] = {0, 0};
  if (tc) TRY_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s), "copy flags");
  if ((rc = copy_out(c, nn, dn, sizeof(int) * nP))) return rc;
  if (d1 && (rc = copy_out(c, d1, dd, sizeof(float) * nP))) return rc;
  SYNC_CHECKED(c, s);
  if (hflags[1]) return set_err(c, LSR_E_TIMEOUT, "BF16 matcher timed out waiting on the tensor cores");
  if (fallbacks) *fallbacks = hflags[0];
  return LSR_OK;
}

int lsr_match_scores_bf16(lsr_ctx *c, const float *FP, int64_t nP, const float *FQ, int64_t nQ, int32_t precision,
                          float *scores) {
  int rc = guard(c);
  if (rc) return rc;
  if (!FP || !FQ || !scores || nP < 1 || nQ < 1 || nP > 65536 || nQ > 65536)
    return set_err(c, LSR_E_ARG, "bad argument");
  if (precision != LSR_MATCH_BF16 && precision != LSR_MATCH_BF16_PLAIN)
    return set_err(c, LSR_E_ARG, "bad precision");
  const bool split = precision == LSR_MATCH_BF16;
  const int cols = tc_score_cols((int)nQ);
  auto plan = [&](Arena &a, float *&fp, float *&fq, float *&FPi, float *&FQi, float *&sc, int *&flags,
                  char *&tws) {
    fp = a.take<float>(kD * nP);
    fq = a.take<float>(kD * nQ);
    FPi = a.take<float>(kDS * nP);
    FQi = a.take<float>(kDS * nQ);
    sc = a.take<float>((size_t)nP * cols);
    flags = a.take<int>(2);
    tws = a.take<char>(tc_workspace_bytes((int)nP, (int)nQ, split));
  };
  Arena m(nullptr);
  float *x1, *x2, *x3, *x4, *x5;
  int *x6;
  char *x7;
  plan(m, x1, x2, x3, x4, x5, x6, x7);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  float *fp, *fq, *FPi, *FQi, *sc;
  int *flags;
  char *tws;
  plan(a, fp, fq, FPi, FQi, sc, flags, tws);
  cudaStream_t s = c->stream;
  TRY_CUDA(c, cudaMemcpyAsync(fp, FP, sizeof(float) * kD * nP, cudaMemcpyDefault, s), "copy FP");
  TRY_CUDA(c, cudaMemcpyAsync(fq, FQ, sizeof(float) * kD * nQ, cudaMemcpyDefault, s), "copy FQ");
  LSR_LAUNCH(k_gather_rows<<<nblk(nP * kDS), 256, 0, s>>>(fp, kD, nullptr, (int)nP, FPi));
  LSR_LAUNCH(k_gather_rows<<<nblk(nQ * kDS), 256, 0, s>>>(fq, kD, nullptr, (int)nQ, FQi));
  TRY_CUDA(c, launch_match_bf16(FPi, (int)nP, FQi, (int)nQ, split, match_tile_for(c, (int)nP), tws, nullptr, nullptr,
                                flags, flags + 1, sc, s, take_tc_fault(c)),
           "scores");
  int hflags[2] = {0, 0};
  TRY_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s), "copy flags");
  TRY_CUDA(c,
           cudaMemcpy2DAsync(scores, sizeof(float) * nQ, sc, sizeof(float) * cols, sizeof(float) * nQ, nP,
                             cudaMemcpyDefault, s),
           "copy scores");
  SYNC_CHECKED(c, s);
  if (hflags[1]) return set_err(c, LSR_E_TIMEOUT, "BF16 matcher timed out waiting on the tensor cores");
  return LSR_OK;
}

int lsr_stage_hypotheses(lsr_ctx *c, const float *P, int64_t nP, const float *Q, int64_t nQ, const int32_t *nn,
                         const uint8_t *validP, const uint8_t *validQ, int64_t H, uint64_t seed, uint64_t pair_id,
                         float tau, int32_t *surv, int64_t cap, int64_t *nsurv) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || !Q || !nn || !validP || !validQ || !surv || !nsurv || nP < 4 || nQ < 4 || nP > kMaxPoints ||
      nQ > kMaxPoints || H < 1 || H > 2147483647LL || cap < 0 || !(tau > 0.f && tau <= 1.f))
    return set_err(c, LSR_E_ARG, "bad argument");
  auto plan = [&](Arena &a, float *&p, float *&q, float4 *&XP, float4 *&XQ, float4 *&NP, float4 *&NQ, int *&inv,
                  int *&dnn, uint8_t *&vp, uint8_t *&vq, PairLayout &L) {
    p = a.take<float>(3 * nP);
    q = a.take<float>(3 * nQ);
    XP = a.take<float4>(nP);
    XQ = a.take<float4>(nQ);
    NP = a.take<float4>(nP);
    NQ = a.take<float4>(nQ);
    inv = a.take<int>(nP);
    dnn = a.take<int>(nP);
    vp = a.take<uint8_t>(nP);
    vq = a.take<uint8_t>(nQ);
    L.nb = hyp_blocks(H);
    L.blk_cnt = a.take<int>((size_t)L.nb + 2);
    L.blk_off = a.take<int>((size_t)L.nb + 2);
    L.blk_scan = a.take<int>((size_t)scan_scratch_ints(L.nb));
    L.hyp_local = a.take<int>((size_t)hyp_local_ints(H));
    L.surv_cap = (int)std::min<int64_t>(H, (int64_t)1 << 26);
    L.surv = a.take<int>(L.surv_cap);
    L.st = a.take<RansacState>(1);
  };
  Arena m(nullptr);
  float *y1, *y2;
  float4 *y3, *y4, *y5, *y6;
  int *y7, *y8;
  uint8_t *y9, *y10;
  PairLayout Lm;
  plan(m, y1, y2, y3, y4, y5, y6, y7, y8, y9, y10, Lm);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  float *p, *q;
  float4 *XP, *XQ, *NP, *NQ;
  int *inv, *dnn;
  uint8_t *vp, *vq;
  PairLayout L;
  plan(a, p, q, XP, XQ, NP, NQ, inv, dnn, vp, vq, L);
  cudaStream_t s = c->stream;
  TRY_CUDA(c, cudaMemcpyAsync(p, P, sizeof(float) * 3 * nP, cudaMemcpyDefault, s), "copy P");
  TRY_CUDA(c, cudaMemcpyAsync(q, Q, sizeof(float) * 3 * nQ, cudaMemcpyDefault, s), "copy Q");
  TRY_CUDA(c, cudaMemcpyAsync(dnn, nn, sizeof(int) * nP, cudaMemcpyDefault, s), "copy nn");
  TRY_CUDA(c, cudaMemcpyAsync(vp, validP, nP, cudaMemcpyDefault, s), "copy vP");
  TRY_CUDA(c, cudaMemcpyAsync(vq, validQ, nQ, cudaMemcpyDefault, s), "copy vQ");
  TRY_CUDA(c, cudaMemsetAsync(L.st, 0, sizeof(RansacState), s), "memset");
  LSR_LAUNCH(k_pack<<<nblk(nP), 256, 0, s>>>(p, (int)nP, XP));
  LSR_LAUNCH(k_pack<<<nblk(nQ), 256, 0, s>>>(q, (int)nQ, XQ));
  LSR_LAUNCH(k_iota<<<nblk(nP), 256, 0, s>>>(inv, (int)nP));
  LSR_LAUNCH(k_valid_normals<<<nblk(nP), 256, 0, s>>>(vp, (int)nP, NP));
  LSR_LAUNCH(k_valid_normals<<<nblk(nQ), 256, 0, s>>>(vq, (int)nQ, NQ));
  TRY_CUDA(c,
           launch_hypotheses(XP, inv, NP, (int)nP, XQ, NQ, (int)nQ, dnn, nullptr, nullptr, H, seed, pair_id, tau,
                             L.blk_cnt, L.blk_off, L.blk_scan, L.surv, L.surv_cap, L.st, L.hyp_local, s),
           "hypotheses");
  RansacState st;
  TRY_CUDA(c, cudaMemcpyAsync(&st, L.st, sizeof(st), cudaMemcpyDeviceToHost, s), "D2H");
  SYNC_CHECKED(c, s);
  *nsurv = st.n_surv_total;
  int64_t ncopy = std::min<int64_t>(std::min<int64_t>(st.n_surv, cap), st.n_surv_total);
  if (ncopy > 0) {
    TRY_CUDA(c, cudaMemcpy(surv, L.surv, sizeof(int) * ncopy, cudaMemcpyDefault), "copy surv");
  }
  return LSR_OK;
}

int lsr_stage_rigid4(lsr_ctx *c, const float *ps, const float *qs, int64_t nh, float *Rt) {
  int rc = guard(c);
  if (rc) return rc;
  if (!ps || !qs || !Rt || nh < 1 || nh > ((int64_t)1 << 28)) return set_err(c, LSR_E_ARG, "bad argument");
  Arena m(nullptr);
  m.take<float>(12 * nh);
  m.take<float>(12 * nh);
  m.take<float>(12 * nh);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  float *dp = a.take<float>(12 * nh), *dq = a.take<float>(12 * nh), *dr = a.take<float>(12 * nh);
  cudaStream_t s = c->stream;
  TRY_CUDA(c, cudaMemcpyAsync(dp, ps, sizeof(float) * 12 * nh, cudaMemcpyDefault, s), "copy");
  TRY_CUDA(c, cudaMemcpyAsync(dq, qs, sizeof(float) * 12 * nh, cudaMemcpyDefault, s), "copy");
  TRY_CUDA(c, launch_rigid4(dp, dq, (int)nh, dr, s), "rigid4");
  if ((rc = copy_out(c, Rt, dr, sizeof(float) * 12 * nh))) return rc;
  SYNC_CHECKED(c, s);
  return LSR_OK;
}

int lsr_stage_consensus(lsr_ctx *c, const float *P, int64_t nP, const float *Q, int64_t nQ, const float *Rt, int64_t nh,
                        float eps, int32_t *count, double *sumd2) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || !Q || !Rt || !count || !sumd2 || nP < 1 || nQ < 1 || nP > kMaxPoints || nQ > kMaxPoints || nh < 1 ||
      nh > ((int64_t)1 << 26) || !(eps > 0.f && eps <= 10.f))
    return set_err(c, LSR_E_ARG, "bad argument");
  struct Bufs {
    float *p, *pose;
    float4 *XP;
    CloudLayout Cq;
    ScratchLayout S;
    int *cnt, *cnt2;
    unsigned long long *sum;
    double *sd;
    ClsParams *cls;
    unsigned *in_bits, *near_bits;
  };
  auto plan = [&](Arena &a, Bufs &b) {
    b.p = a.take<float>(3 * nP);
    b.XP = a.take<float4>(nP);
    plan_cloud(a, (int)nQ, true, false, true, b.Cq);
    plan_scratch(a, (int)nQ, b.Cq.cap_f, b.S);
    b.pose = a.take<float>(12 * nh);
    b.cnt = a.take<int>(nh);
    b.cnt2 = a.take<int>(nh);
    b.sum = a.take<unsigned long long>(nh);
    b.sd = a.take<double>(nh);
    b.cls = a.take<ClsParams>(1);
    b.in_bits = a.take<unsigned>(kClsCapWords);
    b.near_bits = a.take<unsigned>(kClsCapWords);
  };
  Arena m(nullptr);
  Bufs bm;
  plan(m, bm);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  Bufs b;
  plan(a, b);
  float *p = b.p, *pose = b.pose;
  float4 *XP = b.XP;
  CloudLayout &Cq = b.Cq;
  int *cnt = b.cnt;
  unsigned long long *sum = b.sum;
  double *sd = b.sd;
  cudaStream_t s = c->stream;
  TRY_CUDA(c, cudaMemcpyAsync(p, P, sizeof(float) * 3 * nP, cudaMemcpyDefault, s), "copy P");
  const float *qsrc;
  if ((rc = stage_input(c, Q, nQ, Cq.src, &qsrc))) return rc;
  TRY_CUDA(c, cudaMemcpyAsync(pose, Rt, sizeof(float) * 12 * nh, cudaMemcpyDefault, s), "copy Rt");
  LSR_LAUNCH(k_pack<<<nblk(nP), 256, 0, s>>>(p, (int)nP, XP));
  TRY_CUDA(c, build_cloud(qsrc, Cq, eps, eps, eps, false, true, b.S, s), "grid Q");
  TRY_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int) * nh, s), "memset");
  TRY_CUDA(c, cudaMemsetAsync(b.cnt2, 0, sizeof(int) * nh, s), "memset");
  TRY_CUDA(c, cudaMemsetAsync(sum, 0, sizeof(unsigned long long) * nh, s), "memset");
  // counts as the registration pipeline takes them (voxel classification),
  // sums from the exact kernel
  TRY_CUDA(c, launch_cls_build(Cq.box, eps, Cq.X, (int)nQ, b.cls, b.in_bits, b.near_bits, s), "classify");
  TRY_CUDA(c,
           launch_consensus_count(XP, (int)nP, b.cls, b.in_bits, b.near_bits, Cq.ge, Cq.start_e, Cq.Xe, pose, nullptr,
                                  nullptr, (int)nh, eps, cnt, s),
           "consensus");
  TRY_CUDA(c,
           launch_consensus(XP, (int)nP, Cq.ge, Cq.start_e, Cq.Xe, pose, nullptr, nullptr, (int)nh, eps, b.cnt2, sum, s,
                            c->cons_lanes),
           "consensus sums");
  LSR_LAUNCH(k_sum_to_double<<<nblk(nh), 256, 0, s>>>(sum, (int)nh, sd));
  if ((rc = copy_out(c, count, cnt, sizeof(int) * nh))) return rc;
  if ((rc = copy_out(c, sumd2, sd, sizeof(double) * nh))) return rc;
  SYNC_CHECKED(c, s);
  return LSR_OK;
}

int lsr_stage_refine(lsr_ctx *c, const float *P, int64_t nP, const float *Q, int64_t nQ, const double *T_in,
                     float eps, float mu_scale, int32_t levels, int32_t iters, double *T_out, int32_t *iters_done) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || !Q || !T_in || !T_out || nP < 1 || nQ < 1 || nP > kMaxPoints || nQ > kMaxPoints || iters < 0 ||
      iters > 10000 || levels < 1 || levels > kMaxLevels || !(eps > 0.f && eps * (float)(1 << (levels - 1)) <= 10.f) ||
      !(mu_scale > 0.f))
    return set_err(c, LSR_E_ARG, "bad argument");
  float *boxP = nullptr;
  double *boxP_part = nullptr;
  int *seeds = nullptr;
  auto plan = [&](Arena &a, float *&p, float4 *&XP, CloudLayout &Cq, LevelLayout &V, ScratchLayout &S, double *&part,
                  double *&Td, RansacState *&st) {
    seeds = a.take<int>(nP);
    p = a.take<float>(3 * nP);
    XP = a.take<float4>(nP);
    boxP = a.take<float>(kBox);
    boxP_part = a.take<double>((size_t)kBoxPart * bbox_blocks((int)nP));
    plan_cloud(a, (int)nQ, true, false, true, Cq);
    plan_levels(a, (int)nP, (int)nQ, levels, V);
    plan_scratch(a, (int)nQ, Cq.cap_f, S);
    part = a.take<double>((size_t)refine_partial_doubles());
    Td = a.take<double>(16);
    st = a.take<RansacState>(1);
  };
  Arena m(nullptr);
  float *w1;
  float4 *w2;
  CloudLayout w3;
  LevelLayout w8;
  ScratchLayout w4;
  double *w5, *w6;
  RansacState *w7;
  plan(m, w1, w2, w3, w8, w4, w5, w6, w7);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  float *p;
  float4 *XP;
  CloudLayout Cq;
  LevelLayout V;
  ScratchLayout S;
  double *part, *Td;
  RansacState *st;
  plan(a, p, XP, Cq, V, S, part, Td, st);
  cudaStream_t s = c->stream;
  TRY_CUDA(c, cudaMemcpyAsync(p, P, sizeof(float) * 3 * nP, cudaMemcpyDefault, s), "copy P");
  const float *qsrc;
  if ((rc = stage_input(c, Q, nQ, Cq.src, &qsrc))) return rc;
  TRY_CUDA(c, cudaMemcpyAsync(Td, T_in, sizeof(double) * 16, cudaMemcpyDefault, s), "copy T");
  TRY_CUDA(c, cudaMemsetAsync(st, 0, sizeof(RansacState), s), "memset");
  LSR_LAUNCH(k_pack<<<nblk(nP), 256, 0, s>>>(p, (int)nP, XP));
  TRY_CUDA(c, launch_bbox_xyz(p, (int)nP, boxP_part, bbox_blocks((int)nP), boxP, s), "bbox P");
  TRY_CUDA(c, build_cloud(qsrc, Cq, eps, eps, eps, false, true, S, s), "grid Q");
  TRY_CUDA(c, launch_refine_init(st, boxP, Td, s), "init");
  TRY_CUDA(c,
           enqueue_refine(XP, p, (int)nP, qsrc, (int)nQ, Cq.box, Cq.ge, Cq.start_e, Cq.Xe, V, eps, mu_scale, iters, st,
                          part, seeds, S, s, true),
           "refine");
  RansacState h;
  TRY_CUDA(c, cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s), "D2H");
  SYNC_CHECKED(c, s);
  memcpy(T_out, h.T, sizeof(double) * 16);
  if (iters_done) *iters_done = h.iters_done;
  return LSR_OK;
}

// ------------------------------------------------------------------ objective
int lsr_information_matrix(lsr_ctx *c, const float *P, int64_t nP, const float *Q, int64_t nQ, const double *T,
                           float eps, double *info, int64_t *n_corr) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || !Q || !T || !info || nP < 1 || nQ < 1 || nP > kMaxPoints || nQ > kMaxPoints || !(eps > 0.f && eps <= 10.f))
    return set_err(c, LSR_E_ARG, "bad argument");
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(T[k])) return set_err(c, LSR_E_ARG, "non-finite pose");
  struct Bufs {
    float *p;
    CloudLayout Cq;
    ScratchLayout S;
    double *part, *out;
  };
  auto plan = [&](Arena &a, Bufs &b) {
    b.p = a.take<float>(3 * nP);
    plan_cloud(a, (int)nQ, true, false, true, b.Cq);
    plan_scratch(a, (int)nQ, b.Cq.cap_f, b.S);
    b.part = a.take<double>((size_t)10 * information_blocks((int)nP));
    b.out = a.take<double>(37);
  };
  Arena m(nullptr);
  Bufs bm;
  plan(m, bm);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  Bufs b;
  plan(a, b);
  cudaStream_t s = c->stream;
  const float *psrc, *qsrc;
  if ((rc = stage_input(c, P, nP, b.p, &psrc))) return rc;
  if ((rc = stage_input(c, Q, nQ, b.Cq.src, &qsrc))) return rc;
  TRY_CUDA(c, build_cloud(qsrc, b.Cq, eps, eps, eps, false, true, b.S, s), "grid Q");
  float R[9], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) R[3 * r + q] = (float)T[4 * r + q];
    t[r] = (float)T[4 * r + 3];
  }
  TRY_CUDA(c, launch_information(psrc, (int)nP, b.Cq.ge, b.Cq.start_e, b.Cq.Xe, b.Cq.box, R, t, eps, b.part, b.out, s),
           "information");
  double host[37];
  TRY_CUDA(c, cudaMemcpyAsync(host, b.out, sizeof(host), cudaMemcpyDeviceToHost, s), "D2H");
  SYNC_CHECKED(c, s);
  for (int k = 0; k < 36; ++k) info[k] = host[k];
  if (n_corr) *n_corr = (int64_t)host[36];
  return LSR_OK;
}

int lsr_stage_consensus_modes(lsr_ctx *c, const float *P, const float *NP, int64_t nP, const float *Q, const float *NQ,
                              int64_t nQ, const float *Rt, int64_t nh, float eps, int32_t nn_mode, int32_t normal_mode,
                              float cos_normal, int32_t *count, double *sumd2) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || !Q || !Rt || !count || !sumd2 || nP < 1 || nQ < 1 || nP > kMaxPoints || nQ > kMaxPoints || nh < 1 ||
      nh > ((int64_t)1 << 26) || !(eps > 0.f && eps <= 10.f))
    return set_err(c, LSR_E_ARG, "bad argument");
  if ((nn_mode != LSR_NN_EXACT && nn_mode != LSR_NN_SINGLE_CELL) ||
      (normal_mode != LSR_NORMALS_SAMPLES && normal_mode != LSR_NORMALS_INLIERS))
    return set_err(c, LSR_E_ARG, "bad mode");
  const bool normals = normal_mode == LSR_NORMALS_INLIERS, single = nn_mode == LSR_NN_SINGLE_CELL;
  if (normals && (!NP || !NQ || !(cos_normal >= -1.f && cos_normal <= 1.f)))
    return set_err(c, LSR_E_ARG, "the per-inlier normal check needs both normal arrays and a cosine in [-1, 1]");
  struct Bufs {
    float *p, *pose, *np, *nq;
    float4 *XP, *XQ, *NP4, *NQ4;
    CloudLayout Cq;
    ScratchLayout S;
    int *cnt;
    unsigned long long *sum;
    double *sd;
    int *nrows;
  };
  auto plan = [&](Arena &a, Bufs &b) {
    b.p = a.take<float>(3 * nP);
    b.XP = a.take<float4>(nP);
    b.np = a.take<float>(normals ? 3 * nP : 1);
    b.nq = a.take<float>(normals ? 3 * nQ : 1);
    b.NP4 = a.take<float4>(normals ? nP : 1);
    b.NQ4 = a.take<float4>(normals ? nQ : 1);
    b.XQ = a.take<float4>(normals ? nQ : 1);
    plan_cloud(a, (int)nQ, true, false, true, b.Cq);
    plan_scratch(a, (int)nQ, b.Cq.cap_e, b.S);
    b.pose = a.take<float>(12 * nh);
    b.cnt = a.take<int>(nh);
    b.sum = a.take<unsigned long long>(nh);
    b.sd = a.take<double>(nh);
    b.nrows = a.take<int>(1);
  };
  Arena m(nullptr);
  Bufs bm;
  plan(m, bm);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  Bufs b;
  plan(a, b);
  CloudLayout &Cq = b.Cq;
  cudaStream_t s = c->stream;
  TRY_CUDA(c, cudaMemcpyAsync(b.p, P, sizeof(float) * 3 * nP, cudaMemcpyDefault, s), "copy P");
  const float *qsrc;
  if ((rc = stage_input(c, Q, nQ, Cq.src, &qsrc))) return rc;
  TRY_CUDA(c, cudaMemcpyAsync(b.pose, Rt, sizeof(float) * 12 * nh, cudaMemcpyDefault, s), "copy Rt");
  LSR_LAUNCH(k_pack<<<nblk(nP), 256, 0, s>>>(b.p, (int)nP, b.XP));  // w = caller index
  if (normals) {
    TRY_CUDA(c, cudaMemcpyAsync(b.np, NP, sizeof(float) * 3 * nP, cudaMemcpyDefault, s), "copy NP");
    TRY_CUDA(c, cudaMemcpyAsync(b.nq, NQ, sizeof(float) * 3 * nQ, cudaMemcpyDefault, s), "copy NQ");
    LSR_LAUNCH(k_gather_normals<<<nblk(nP), 256, 0, s>>>(b.np, b.XP, (int)nP, b.NP4));
    LSR_LAUNCH(k_pack<<<nblk(nQ), 256, 0, s>>>(qsrc, (int)nQ, b.XQ));
    LSR_LAUNCH(k_gather_normals<<<nblk(nQ), 256, 0, s>>>(b.nq, b.XQ, (int)nQ, b.NQ4));
  }
  // Q's grid with caller indices in w (exact: cells of eps; single: the eps lattice through the centroid)
  TRY_CUDA(c, launch_bbox_xyz(qsrc, Cq.n, Cq.box_part, bbox_blocks(Cq.n), Cq.box, s), "bbox");
  if (single)
    TRY_CUDA(c, launch_cell_grid_params(Cq.box, eps, Cq.n, Cq.cap_e, Cq.ge, s), "grid params");
  else
    TRY_CUDA(c, launch_grid_params(Cq.box, eps, Cq.n, Cq.cap_e, Cq.ge, s), "grid params");
  TRY_CUDA(c, build_grid_xyz(qsrc, Cq.n, Cq.ge, Cq.cap_e, Cq.start_e, Cq.Xe, Cq.inv, b.S.g, s), "grid");
  if (!single) TRY_CUDA(c, build_nbmask(Cq.ge, Cq.start_e, Cq.cap_e, Cq.mask_e, s), "mask");
  TRY_CUDA(c, cudaMemsetAsync(b.cnt, 0, sizeof(int) * nh, s), "memset");
  TRY_CUDA(c, cudaMemsetAsync(b.sum, 0, sizeof(unsigned long long) * nh, s), "memset");
  const int nh32 = (int)nh;
  TRY_CUDA(c, cudaMemcpyAsync(b.nrows, &nh32, sizeof(int), cudaMemcpyHostToDevice, s), "H2D");
  TRY_CUDA(c,
           launch_consensus_variant(b.XP, (int)nP, b.NP4, Cq.ge, Cq.start_e, Cq.Xe, b.NQ4, (int)nQ, b.pose, nullptr,
                                    b.nrows, eps, single, normals, cos_normal, b.cnt, b.sum, s),
           "consensus variant");
  LSR_LAUNCH(k_sum_to_double<<<nblk(nh), 256, 0, s>>>(b.sum, (int)nh, b.sd));
  if ((rc = copy_out(c, count, b.cnt, sizeof(int) * nh))) return rc;
  if ((rc = copy_out(c, sumd2, b.sd, sizeof(double) * nh))) return rc;
  SYNC_CHECKED(c, s);
  return LSR_OK;
}

int lsr_stage_nn(lsr_ctx *c, const float *Q, int64_t nQ, const float *X, int64_t nX, float r, int32_t mode,
                 int32_t *nn, float *d2) {
  int rc = guard(c);
  if (rc) return rc;
  if (!Q || !X || !nn || nQ < 1 || nX < 1 || nQ > kMaxPoints || nX > kMaxPoints || !(r > 0.f && r <= 10.f))
    return set_err(c, LSR_E_ARG, "bad argument");
  if (mode != LSR_NN_EXACT && mode != LSR_NN_SINGLE_CELL) return set_err(c, LSR_E_ARG, "bad mode");
  struct Bufs {
    float *x;
    CloudLayout Cq;
    ScratchLayout S;
    int *nn;
    float *d2;
  };
  auto plan = [&](Arena &a, Bufs &b) {
    b.x = a.take<float>(3 * nX);
    plan_cloud(a, (int)nQ, true, false, true, b.Cq);
    plan_scratch(a, (int)nQ, b.Cq.cap_e, b.S);
    b.nn = a.take<int>(nX);
    b.d2 = a.take<float>(nX);
  };
  Arena m(nullptr);
  Bufs bm;
  plan(m, bm);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  Bufs b;
  plan(a, b);
  cudaStream_t s = c->stream;
  const float *xsrc, *qsrc;
  if ((rc = stage_input(c, X, nX, b.x, &xsrc))) return rc;
  if ((rc = stage_input(c, Q, nQ, b.Cq.src, &qsrc))) return rc;
  CloudLayout &Cq = b.Cq;
  const bool single = mode == LSR_NN_SINGLE_CELL;
  TRY_CUDA(c, launch_bbox_xyz(qsrc, Cq.n, Cq.box_part, bbox_blocks(Cq.n), Cq.box, s), "bbox");
  if (single)
    TRY_CUDA(c, launch_cell_grid_params(Cq.box, r, Cq.n, Cq.cap_e, Cq.ge, s), "grid params");
  else
    TRY_CUDA(c, launch_grid_params(Cq.box, r, Cq.n, Cq.cap_e, Cq.ge, s), "grid params");
  TRY_CUDA(c, build_grid_xyz(qsrc, Cq.n, Cq.ge, Cq.cap_e, Cq.start_e, Cq.Xe, Cq.inv, b.S.g, s), "grid");
  if (!single) TRY_CUDA(c, build_nbmask(Cq.ge, Cq.start_e, Cq.cap_e, Cq.mask_e, s), "mask");
  TRY_CUDA(c, launch_nn_stage(xsrc, (int)nX, Cq.ge, Cq.start_e, Cq.Xe, r, single ? 1 : 0, b.nn, b.d2, s), "nn");
  if ((rc = copy_out(c, nn, b.nn, sizeof(int) * nX))) return rc;
  if (d2 && (rc = copy_out(c, d2, b.d2, sizeof(float) * nX))) return rc;
  SYNC_CHECKED(c, s);
  return LSR_OK;
}

int lsr_pose_implicit_grad(lsr_ctx *c, const float *P, int64_t nP, const float *Q, int64_t nQ, const double *T,
                           float eps, float mu, const double *dL_dT, float *dP, float *dQ, double *grad,
                           double *hess, double *lambda, int64_t *n_corr) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || !Q || !T || !dL_dT || !dP || !dQ || nP < 1 || nQ < 1 || nP > kMaxPoints || nQ > kMaxPoints ||
      !(eps > 0.f && eps <= 10.f) || !(mu > 0.f))
    return set_err(c, LSR_E_ARG, "bad argument");
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(T[k]) || !std::isfinite(dL_dT[k])) return set_err(c, LSR_E_ARG, "non-finite pose or gradient");
  // dL/dxi of the left perturbation T(xi) = [Exp(w) | v] T: with M = G_R R^T +
  // G_t t^T (G = dL/dT), dL/dw = (M32 - M23, M13 - M31, M21 - M12), dL/dv = G_t
  double M[3][3], dl[6];
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      double v = dL_dT[4 * r + 3] * T[4 * q + 3];
      for (int k = 0; k < 3; ++k) v += dL_dT[4 * r + k] * T[4 * q + k];
      M[r][q] = v;
    }
  dl[0] = M[2][1] - M[1][2], dl[1] = M[0][2] - M[2][0], dl[2] = M[1][0] - M[0][1];
  for (int r = 0; r < 3; ++r) dl[3 + r] = dL_dT[4 * r + 3];
  struct Bufs {
    float *p, *gp, *gq;
    CloudLayout Cq;
    ScratchLayout S;
    double *part, *out, *dl;
  };
  const bool dev_out = is_device_ptr(dP);
  if (dev_out != is_device_ptr(dQ)) return set_err(c, LSR_E_ARG, "dP and dQ must both be device or both host");
  auto plan = [&](Arena &a, Bufs &b) {
    b.p = a.take<float>(3 * nP);
    b.gp = dev_out ? nullptr : a.take<float>(3 * nP);
    b.gq = dev_out ? nullptr : a.take<float>(3 * nQ);
    plan_cloud(a, (int)nQ, true, false, true, b.Cq);
    plan_scratch(a, (int)nQ, b.Cq.cap_f, b.S);
    b.part = a.take<double>((size_t)implicit_partials((int)nP));
    b.out = a.take<double>(50);
    b.dl = a.take<double>(6);
  };
  Arena m(nullptr);
  Bufs bm;
  plan(m, bm);
  if ((rc = ensure_ws(c, m.off))) return rc;
  Arena a(c->ws);
  Bufs b;
  plan(a, b);
  cudaStream_t s = c->stream;
  const float *psrc, *qsrc;
  if ((rc = stage_input(c, P, nP, b.p, &psrc))) return rc;
  if ((rc = stage_input(c, Q, nQ, b.Cq.src, &qsrc))) return rc;
  // eps grid of Q with caller indices in w (build_grid_xyz carries the caller order), so dQ is in caller order
  CloudLayout &Cq = b.Cq;
  TRY_CUDA(c, launch_bbox_xyz(qsrc, Cq.n, Cq.box_part, bbox_blocks(Cq.n), Cq.box, s), "bbox");
  TRY_CUDA(c, launch_grid_params(Cq.box, eps, Cq.n, Cq.cap_e, Cq.ge, s), "grid params");
  TRY_CUDA(c, build_grid_xyz(qsrc, Cq.n, Cq.ge, Cq.cap_e, Cq.start_e, Cq.Xe, Cq.inv, b.S.g, s), "grid");
  TRY_CUDA(c, build_nbmask(Cq.ge, Cq.start_e, Cq.cap_e, Cq.mask_e, s), "mask");
  TRY_CUDA(c, cudaMemcpyAsync(b.dl, dl, sizeof(dl), cudaMemcpyHostToDevice, s), "H2D");
  float *gp = dev_out ? dP : b.gp, *gq = dev_out ? dQ : b.gq;
  TRY_CUDA(c, cudaMemsetAsync(gq, 0, sizeof(float) * 3 * nQ, s), "memset dQ");
  TRY_CUDA(c,
           launch_implicit(psrc, (int)nP, b.Cq.ge, b.Cq.start_e, b.Cq.Xe, (int)nQ, T, eps, (double)mu, b.dl, b.part,
                           b.out, gp, gq, s),
           "implicit");
  double host[50];
  TRY_CUDA(c, cudaMemcpyAsync(host, b.out, sizeof(host), cudaMemcpyDeviceToHost, s), "D2H");
  if (!dev_out) {
    TRY_CUDA(c, cudaMemcpyAsync(dP, gp, sizeof(float) * 3 * nP, cudaMemcpyDeviceToHost, s), "D2H");
    TRY_CUDA(c, cudaMemcpyAsync(dQ, gq, sizeof(float) * 3 * nQ, cudaMemcpyDeviceToHost, s), "D2H");
  }
  SYNC_CHECKED(c, s);
  if (grad)
    for (int k = 0; k < 6; ++k) grad[k] = host[k];
  if (hess)
    for (int k = 0; k < 36; ++k) hess[k] = host[6 + k];
  if (lambda)
    for (int k = 0; k < 6; ++k) lambda[k] = host[42 + k];
  if (n_corr) *n_corr = (int64_t)host[48];
  if (host[49] != 0.0) return set_err(c, LSR_E_ARG, "the Hessian of the held pairs is singular (too few pairs)");
  return LSR_OK;
}

int lsr_voxel_downsample(lsr_ctx *c, const float *P, int64_t n, float leaf, float *out, int64_t cap,
                         int64_t *n_out) {
  int rc = guard(c);
  if (rc) return rc;
  if (!P || !out || !n_out || n < 1 || n > kMaxPoints || cap < 0 || !(leaf > 0.f && leaf <= 100.f))
    return set_err(c, LSR_E_ARG, "bad argument");
  constexpr int64_t kMaxCells = (int64_t)1 << 26;
  int64_t ncells = 0;
  for (int pass = 0; pass < 2; ++pass) {
    struct Bufs {
      float *p, *o;
      int *kb, *ncd, *cnt, *flag, *pos, *scan;
      unsigned long long *sums;
      int64_t *nout;
    };
    auto plan = [&](Arena &a, Bufs &b) {
      b.p = a.take<float>(3 * (size_t)n);
      b.o = a.take<float>(3 * (size_t)(cap > 0 ? cap : 1));
      b.kb = a.take<int>(6);
      b.ncd = a.take<int>(1);
      b.nout = a.take<int64_t>(1);
      b.cnt = a.take<int>((size_t)ncells);
      b.flag = a.take<int>((size_t)ncells);
      b.pos = a.take<int>((size_t)ncells + 1);
      b.scan = a.take<int>((size_t)scan_scratch_ints(ncells));
      b.sums = a.take<unsigned long long>(3 * (size_t)ncells);
    };
    Arena m(nullptr);
    Bufs bm;
    plan(m, bm);
    if ((rc = ensure_ws(c, m.off))) return rc;
    Arena a(c->ws);
    Bufs b;
    plan(a, b);
    cudaStream_t s = c->stream;
    const float *src;
    if ((rc = stage_input(c, P, n, b.p, &src))) return rc;
    TRY_CUDA(c, launch_vox_bounds(src, n, leaf, b.kb, s), "voxel bounds");
    int kb[6];
    TRY_CUDA(c, cudaMemcpyAsync(kb, b.kb, sizeof(kb), cudaMemcpyDeviceToHost, s), "D2H");
    SYNC_CHECKED(c, s);
    const int64_t need = ((int64_t)kb[3] - kb[0] + 1) * ((int64_t)kb[4] - kb[1] + 1) * ((int64_t)kb[5] - kb[2] + 1);
    if (kb[0] > kb[3] || need > kMaxCells) return set_err(c, LSR_E_TOO_LARGE, "voxel grid of the cloud too large");
    if (pass == 0) {
      ncells = need;  // plan again with the cells (the workspace may move)
      continue;
    }
    const int ncells_i = (int)ncells;
    TRY_CUDA(c, cudaMemcpyAsync(b.ncd, &ncells_i, sizeof(int), cudaMemcpyHostToDevice, s), "H2D");
    const bool dev_out = is_device_ptr(out);
    TRY_CUDA(c,
             launch_vox_cells(src, n, leaf, b.kb, ncells, b.ncd, b.cnt, b.sums, b.flag, b.pos, b.scan,
                              dev_out ? out : b.o, cap, b.nout, s),
             "voxel cells");
    int64_t m_out = 0;
    TRY_CUDA(c, cudaMemcpyAsync(&m_out, b.nout, sizeof(m_out), cudaMemcpyDeviceToHost, s), "D2H");
    SYNC_CHECKED(c, s);
    if (!dev_out && cap > 0 && (rc = copy_out(c, out, b.o, sizeof(float) * 3 * (size_t)std::min(m_out, cap))))
      return rc;
    SYNC_CHECKED(c, s);
    *n_out = m_out;
  }
  return LSR_OK;
}

int lsr_surfel_correct(lsr_ctx *c, int64_t n, const float *pos, const float *nrm, const float *t0, const float *tu,
                       int32_t m, const double *T_old, const double *T_new, const float *t_kf, const float *cam,
                       float *pos_out, float *nrm_out, uint8_t *keep, int64_t *n_keep) {
  int rc = guard(c);
  if (rc) return rc;
  if (!pos || !nrm || !t0 || !tu || !T_old || !T_new || !t_kf || !cam || !pos_out || !nrm_out || !keep || n < 1 ||
      n > ((int64_t)1 << 31) || m < 1 || m > (1 << 20))
    return set_err(c, LSR_E_ARG, "bad argument");
  for (int k = 0; k < 7; ++k)
    if (!(std::isfinite(cam[k]) && cam[k] > 0.f) && !(k >= 2 && k <= 3 && std::isfinite(cam[k])))
      return set_err(c, LSR_E_ARG, "bad camera");
  std::vector<KfPose> kf((size_t)m);
  for (int f = 0; f < m; ++f) {
    if (f > 0 && !(t_kf[f] >= t_kf[f - 1])) return set_err(c, LSR_E_ARG, "keyframe stamps must ascend");
    const double *To = T_old + 16 * (size_t)f, *Tn = T_new + 16 * (size_t)f;
    for (int k = 0; k < 16; ++k)
      if (!std::isfinite(To[k]) || !std::isfinite(Tn[k])) return set_err(c, LSR_E_ARG, "non-finite pose");
    // rigid inverse of the camera-to-world pose: [R^T | -R^T t]
    double A[12], M[12];
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) A[4 * r + q] = To[4 * q + r];
      A[4 * r + 3] = -(To[r] * To[3] + To[4 + r] * To[7] + To[8 + r] * To[11]);
    }
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 4; ++q)
        M[4 * r + q] = Tn[4 * r] * A[q] + Tn[4 * r + 1] * A[4 + q] + Tn[4 * r + 2] * A[8 + q] + (q == 3 ? Tn[4 * r + 3] : 0.0);
    for (int k = 0; k < 12; ++k) kf[f].A[k] = (float)A[k], kf[f].M[k] = (float)M[k];
  }
  const SurfelCam sc{cam[0], cam[1], cam[2], cam[3], cam[4], cam[5], cam[6]};
  struct Bufs {
    float *pos, *nrm, *t0, *tu, *tk, *po, *no;
    KfPose *kf;
    uint8_t *keep;
    unsigned long long *cnt;
  };
  auto plan = [&](Arena &a, Bufs &b) {
    b.pos = a.take<float>(3 * (size_t)n);
    b.nrm = a.take<float>(3 * (size_t)n);
    b.t0 = a.take<float>((size_t)n);
    b.tu = a.take<float>((size_t)n);
    b.po = a.take<float>(3 * (size_t)n);
    b.no = a.take<float>(3 * (size_t)n);
    b.keep = a.take<uint8_t>((size_t)n);
    b.kf = a.take<KfPose>((size_t)m);
    b.tk = a.take<float>((size_t)m);
    b.cnt = a.take<unsigned long long>(1);
  };
  Arena mm(nullptr);
  Bufs bm;
  plan(mm, bm);
  if ((rc = ensure_ws(c, mm.off))) return rc;
  Arena a(c->ws);
  Bufs b;
  plan(a, b);
  cudaStream_t s = c->stream;
  auto in = [&](const float *src, size_t cnt, float *dst, const float **out) -> int {
    if (is_device_ptr(src)) {
      *out = src;
      return LSR_OK;
    }
    TRY_CUDA(c, cudaMemcpyAsync(dst, src, sizeof(float) * cnt, cudaMemcpyHostToDevice, s), "H2D");
    *out = dst;
    return LSR_OK;
  };
  const float *dpos, *dnrm, *dt0, *dtu;
  if ((rc = in(pos, 3 * (size_t)n, b.pos, &dpos)) || (rc = in(nrm, 3 * (size_t)n, b.nrm, &dnrm)) ||
      (rc = in(t0, (size_t)n, b.t0, &dt0)) || (rc = in(tu, (size_t)n, b.tu, &dtu)))
    return rc;
  TRY_CUDA(c, cudaMemcpyAsync(b.kf, kf.data(), sizeof(KfPose) * (size_t)m, cudaMemcpyHostToDevice, s), "H2D");
  TRY_CUDA(c, cudaMemcpyAsync(b.tk, t_kf, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, s), "H2D");
  const bool dev_out = is_device_ptr(pos_out) && is_device_ptr(nrm_out) && is_device_ptr(keep);
  float *po = dev_out ? pos_out : b.po, *no = dev_out ? nrm_out : b.no;
  uint8_t *ko = dev_out ? keep : b.keep;
  TRY_CUDA(c, launch_surfel_correct(n, dpos, dnrm, dt0, dtu, m, b.kf, b.tk, sc, po, no, ko, b.cnt, s), "surfels");
  if (!dev_out) {
    if ((rc = copy_out(c, pos_out, po, sizeof(float) * 3 * (size_t)n))) return rc;
    if ((rc = copy_out(c, nrm_out, no, sizeof(float) * 3 * (size_t)n))) return rc;
    if ((rc = copy_out(c, keep, ko, (size_t)n))) return rc;
  }
  unsigned long long cnt = 0;
  TRY_CUDA(c, cudaMemcpyAsync(&cnt, b.cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s), "D2H");
  SYNC_CHECKED(c, s);
  if (n_keep) *n_keep = (int64_t)cnt;
  return LSR_OK;
}

static void host_exp_so3(const double w[3], double R[9]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], th = sqrt(th2);
  double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double a = th < 1e-6 ? 1.0 - th2 / 6.0 : sin(th) / th;
  double b = th < 1e-6 ? 0.5 - th2 / 24.0 : (1.0 - cos(th)) / th2;
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      double k2 = K[3 * r] * K[q] + K[3 * r + 1] * K[3 + q] + K[3 * r + 2] * K[6 + q];
      R[3 * r + q] = (r == q ? 1.0 : 0.0) + a * K[3 * r + q] + b * k2;
    }
}

// Left Jacobian of SO(3): Exp(w + d) = Exp(J_l(w) d) Exp(w) to first order.
static void host_left_jacobian(const double w[3], double J[9]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], th = sqrt(th2);
  double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double a = th < 1e-5 ? 0.5 - th2 / 24.0 : (1.0 - cos(th)) / th2;
  double b = th < 1e-5 ? 1.0 / 6.0 - th2 / 120.0 : (th - sin(th)) / (th2 * th);
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      double k2 = K[3 * r] * K[q] + K[3 * r + 1] * K[3 + q] + K[3 * r + 2] * K[6 + q];
      J[3 * r + q] = (r == q ? 1.0 : 0.0) + a * K[3 * r + q] + b * k2;
    }
}

static int objective_impl(lsr_ctx *c, int32_t n, const float *const *P, const int64_t *nP, const float *const *Q,
                          const int64_t *nQ, const double *xi, const double *T0, float eps, float mu, const double *dE,
                          double *E, float *const *dP, float *const *dQ, double *dxi) {
  int rc = guard(c);
  if (rc) return rc;
  bool grad = dE != nullptr;
  if (n < 0 || (n > 0 && (!P || !nP || !Q || !nQ || !xi || !T0)) || !(eps > 0.f && eps <= 10.f) || !(mu > 0.f) ||
      (!grad && !E) || (grad && (!dP || !dQ || !dxi)))
    return set_err(c, LSR_E_ARG, "bad argument");
  int64_t maxP = 0, maxQ = 0;
  for (int i = 0; i < n; ++i) {
    if (!P[i] || !Q[i] || nP[i] < 1 || nQ[i] < 1 || nP[i] > kMaxPoints || nQ[i] > kMaxPoints)
      return set_err(c, LSR_E_ARG, "bad cloud");
    if (!is_device_ptr(P[i]) || !is_device_ptr(Q[i])) return set_err(c, LSR_E_ARG, "objective clouds must be on the device");
    if (grad && (!dP[i] || !dQ[i] || !is_device_ptr(dP[i]) || !is_device_ptr(dQ[i])))
      return set_err(c, LSR_E_ARG, "objective gradients must be device arrays");
    maxP = std::max(maxP, nP[i]);
    maxQ = std::max(maxQ, nQ[i]);
  }
  if (n == 0) return LSR_OK;
  // pairs round-robin over S lanes (own stream and workspace each): at these
  // sizes every pair is a chain of short launches, and the lanes overlap them
  const int nl = std::max(1, std::min((int)n, c->prm.batch_streams > 0 ? c->prm.batch_streams : 4));
  auto plan = [&](Arena &a, CloudLayout &Cq, ScratchLayout &Sc, double *&part) {
    plan_cloud(a, (int)maxQ, false, false, true, Cq);
    plan_scratch(a, (int)maxQ, Cq.cap_f, Sc);
    part = a.take<double>((size_t)7 * objective_blocks((int)maxP));
  };
  Arena m(nullptr);
  CloudLayout q1;
  ScratchLayout q2;
  double *q3;
  plan(m, q1, q2, q3);
  if ((rc = ensure_lanes(c, nl, m.off))) return rc;
  if ((rc = ensure_ws(c, sizeof(double) * 7 * (size_t)n))) return rc;
  double *out7 = reinterpret_cast<double *>(c->ws);
  TRY_CUDA(c, cudaEventRecord(c->fork, c->stream), "fork");
  for (int l = 0; l < nl; ++l) TRY_CUDA(c, cudaStreamWaitEvent(c->lanes[l], c->fork, 0), "fork");
  std::vector<double> host7((size_t)7 * n);
  for (int i = 0; i < n; ++i) {
    const int l = i % nl;
    cudaStream_t s = c->lanes[l];
    Arena a(c->lane_ws[l]);
    CloudLayout Cq;
    ScratchLayout Sc;
    double *part;
    plan(a, Cq, Sc, part);
    Cq.n = (int)nQ[i];
    const double *w = xi + 6 * i, *T = T0 + 16 * i;
    double Rw[9], Tm[16];
    host_exp_so3(w, Rw);
    double M[16] = {Rw[0], Rw[1], Rw[2], w[3], Rw[3], Rw[4], Rw[5], w[4], Rw[6], Rw[7], Rw[8], w[5], 0, 0, 0, 1};
    for (int r = 0; r < 4; ++r)
      for (int q = 0; q < 4; ++q) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += M[4 * r + k] * T[4 * k + q];
        Tm[4 * r + q] = acc;
      }
    const double vd[3] = {w[3], w[4], w[5]};
    // eps grid of Q with caller indices (build_grid_xyz carries caller order)
    TRY_CUDA(c, launch_bbox_xyz(Q[i], Cq.n, Cq.box_part, bbox_blocks(Cq.n), Cq.box, s), "bbox");
    TRY_CUDA(c, launch_grid_params(Cq.box, eps, Cq.n, Cq.cap_e, Cq.ge, s), "grid params");
    TRY_CUDA(c, build_grid_xyz(Q[i], Cq.n, Cq.ge, Cq.cap_e, Cq.start_e, Cq.Xe, Cq.inv, Sc.g, s), "grid");
    TRY_CUDA(c, build_nbmask(Cq.ge, Cq.start_e, Cq.cap_e, Cq.mask_e, s), "mask");
    if (grad) TRY_CUDA(c, cudaMemsetAsync(dQ[i], 0, sizeof(float) * 3 * nQ[i], s), "memset dQ");
    TRY_CUDA(c,
             launch_objective(P[i], (int)nP[i], Cq.ge, Cq.start_e, Cq.Xe, Tm, vd, eps, mu,
                              grad ? dE[i] : 1.0, grad ? 1 : 0, part, out7 + 7 * i, grad ? dP[i] : nullptr,
                              grad ? dQ[i] : nullptr, s),
             "objective");
  }
  for (int l = 0; l < nl; ++l) {
    TRY_CUDA(c, cudaEventRecord(c->lane_done[l], c->lanes[l]), "join");
    TRY_CUDA(c, cudaStreamWaitEvent(c->stream, c->lane_done[l], 0), "join");
  }
  TRY_CUDA(c, cudaMemcpyAsync(host7.data(), out7, sizeof(double) * 7 * n, cudaMemcpyDeviceToHost, c->stream), "D2H");
  SYNC_CHECKED(c, c->stream);
  for (int i = 0; i < n; ++i) {
    const double *o = &host7[(size_t)7 * i];
    if (E) E[i] = o[0];
    if (grad) {
      double J[9];
      host_left_jacobian(xi + 6 * i, J);
      for (int q = 0; q < 3; ++q) dxi[6 * i + q] = dE[i] * (J[0 * 3 + q] * o[4] + J[1 * 3 + q] * o[5] + J[2 * 3 + q] * o[6]);
      for (int q = 0; q < 3; ++q) dxi[6 * i + 3 + q] = dE[i] * o[1 + q];
    }
  }
  return LSR_OK;
}

int lsr_objective_fwd(lsr_ctx *c, int32_t n, const float *const *P, const int64_t *nP, const float *const *Q,
                      const int64_t *nQ, const double *xi, const double *T0, float eps, float mu, double *E) {
  return objective_impl(c, n, P, nP, Q, nQ, xi, T0, eps, mu, nullptr, E, nullptr, nullptr, nullptr);
}

int lsr_objective_bwd(lsr_ctx *c, int32_t n, const float *const *P, const int64_t *nP, const float *const *Q,
                      const int64_t *nQ, const double *xi, const double *T0, float eps, float mu, const double *dE,
                      float *const *dP, float *const *dQ, double *dxi) {
  if (!dE) return c ? set_err(c, LSR_E_ARG, "null dE") : LSR_E_STATE;
  return objective_impl(c, n, P, nP, Q, nQ, xi, T0, eps, mu, dE, nullptr, dP, dQ, dxi);
}

}  // extern "C"
