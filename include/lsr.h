/*
 * lsr.h -- C ABI of the GB300 (sm_103a) implementation of the global point
 * cloud registration of LoopSmart (Zhang & Chen, arXiv 1801.01572), Sec. IV,
 * Algorithm 1 ("Global Registration on GPU"), with the robust refinement and
 * alignment objective of eq. (3)-(5).
 *
 * Given two fragments P and Q (float32 xyz, N x 3 row-major), the library
 * estimates T_QP (q ~ T p) with no initial pose: radius-PCA normals, FPFH
 * descriptors (Rusu et al. 2009, the descriptor of Alg. 1), the feature
 * pre-matching cache (Alg. 1, "Parallel FPFH feature pre-matching"), 4-point
 * hypotheses with polygon pre-rejection (Alg. 1, tau of Sec. IV), stream
 * compaction, consensus on a 3D grid (eq. (1)), selection, and a robust
 * Geman-McClure refinement (the line process of eq. (4) eliminated).
 *
 * Conventions shared by every entry point:
 *  - Return value: LSR_OK (0) or a negative LSR_E_* code. On error, outputs
 *    are unspecified and lsr_last_error(ctx) holds a one-line message.
 *    "No alignment found" is NOT an error: it is result.status (Alg. 1 only
 *    returns a pose "if hypothesis found").
 *  - Point / descriptor arrays may be device pointers (cudaMalloc, torch CUDA
 *    tensors) or host pointers (pageable or pinned); host inputs are copied to
 *    the device inside the call and host outputs are copied back before it
 *    returns. Arrays must be contiguous and 4-byte aligned. The caller owns all
 *    input and output buffers; the library owns its device workspace, which
 *    grows on demand and is released by lsr_destroy.
 *  - All device work is ordered on the context's stream. Entry points that
 *    return results in host memory synchronise that stream once before
 *    returning.
 *  - A context is not thread-safe: use one context per host thread.
 *  - Indices are 0-based and refer to the caller's point order.
 */
#ifndef LSR_H
#define LSR_H

#include <stdint.h>

#if defined(__GNUC__)
#define LSR_API __attribute__((visibility("default")))
#else
#define LSR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define LSR_OK 0
#define LSR_E_ARG (-1)     /* invalid argument: NULL pointer, n < 4, size too large, bad parameter */
#define LSR_E_CUDA (-2)    /* a CUDA runtime call or kernel launch failed */
#define LSR_E_OOM (-3)     /* device or host memory allocation failed */
#define LSR_E_TIMEOUT (-4) /* a bounded device-side wait ran out */
#define LSR_E_STATE (-5)   /* context not usable (NULL, destroyed, or a previous sticky CUDA error) */
#define LSR_E_TOO_LARGE (-6) /* input larger than the fixed scratch of lsr_consensus_static allows */
#define LSR_E_CHECK (-7)   /* checked build only: a device bounds check failed (the access was skipped) */

#define LSR_STATUS_ALIGNED 0
#define LSR_STATUS_NO_ALIGNMENT 1

#define LSR_MATCH_FP32 0 /* descriptor matching on FP32 SIMT cores */
#define LSR_MATCH_BF16 1 /* tensor cores: descriptors as hi + lo BF16 pairs (K = 112),
                            top-8 candidates, exact FP32 re-rank, certified */
#define LSR_MATCH_BF16_PLAIN 2 /* tensor cores: descriptors rounded to one BF16 each,
                                  zero-padded to K = 48; same re-rank and certificate */

#define LSR_DESC_DIM 33 /* FPFH: 3 angular features x 11 bins */

typedef struct lsr_ctx lsr_ctx;

/* Parameters. Defaults (lsr_default_params) are the paper's hyper-parameters
 * (Sec. IV: normal radius 0.1 m, FPFH radius 0.25 m, 4,000,000 hypotheses,
 * maximum correspondence distance 0.075 m, tau = 0.9) with the radii scaled to
 * the 5 cm / 12.5 cm neighbourhoods of the synthetic fragments, keeping the
 * paper's ratio eps = 0.75 r_normal. */
typedef struct {
  float r_normal;         /* normal estimation radius (m), default 0.05 */
  float r_feature;        /* FPFH radius (m), default 0.125 */
  float eps_inlier;       /* maximum correspondence distance (m), default 0.0375 */
  float tau;              /* polygon similarity threshold, default 0.9 */
  float cos_normal;       /* normal check: reject a hypothesis if any sampled pair has cos(R n_p, n_q) below this; default cos(30 deg) */
  float min_inlier_ratio; /* accept the best hypothesis if inliers / |P| >= this; default 0.05 */
  float mu_scale;         /* Geman-McClure scale: mu = mu_scale * r^2 at refinement radius r; default 1 */
  int32_t refine_iters;   /* maximum refinement iterations per level, default 50 */
  int64_t n_hypotheses;   /* sampled hypotheses per pair, default 4,000,000 (at most 2^31 - 1) */
  uint64_t seed;          /* hypothesis RNG key word 0 (Philox-4x64-10 key = (seed, pair_id)) */
  uint64_t pair_id;       /* RNG key word 1 for lsr_register_pair; a batch uses pair_id + i */
  int32_t match_precision; /* LSR_MATCH_FP32 (default), LSR_MATCH_BF16 or LSR_MATCH_BF16_PLAIN */
  int32_t refine_levels;  /* graduated refinement levels L (1..8), default 3: radius eps * 2^(L-1-l) at level l */
  int32_t batch_streams;  /* lsr_register_batch: pairs run concurrently on this many streams (1..16), each with
                             its own workspace; 0 (default) = chosen by the autotuner on the first batch */
  int32_t batch_graph;    /* lsr_register_batch with device-resident clouds: 1 = capture the whole batch as one
                             CUDA graph and replay it when the same batch (same pointers, sizes, viewpoints and
                             parameters) is registered again; 0 (default) = launch directly */
  int32_t match_tile;     /* tensor-core matcher work unit: 1 or 2 query tiles of 128 per CTA; 0 (default) =
                             chosen per cloud size by the autotuner */
  int32_t nn_mode;        /* inlier test of the consensus: LSR_NN_EXACT (default: the nearest Q point over every
                             grid cell the eps-ball overlaps) or LSR_NN_SINGLE_CELL (the O(1) lookup of eq. (1):
                             only the query's own cell of edge eps, centred on Q's centroid; approximate, it can
                             only miss inliers) */
  int32_t normal_mode;    /* normal check: LSR_NORMALS_SAMPLES (default: the 4 sampled pairs of a hypothesis) or
                             LSR_NORMALS_INLIERS (every inlier instead: a point counts only if its nearest Q
                             point's normal agrees with its rotated normal, cos >= cos_normal) */
  int32_t reserved_[2];
} lsr_params;

#define LSR_NN_EXACT 0
#define LSR_NN_SINGLE_CELL 1
#define LSR_NORMALS_SAMPLES 0
#define LSR_NORMALS_INLIERS 1

/* Result of one registration. */
typedef struct {
  double T[16];           /* row-major 4x4 T_QP (q ~ T p); identity if status is NO_ALIGNMENT */
  double T_hyp[16];       /* pose of the selected 4-point hypothesis before refinement */
  int64_t inliers;        /* points of P with a Q point closer than eps under T */
  int64_t hyp_inliers;    /* inliers of the selected hypothesis */
  int64_t survivors;      /* hypotheses left after pre-rejection */
  int64_t n_normal_ok;    /* survivors that also pass the normal check */
  int64_t best_h;         /* id of the selected hypothesis, -1 if none */
  int64_t match_fallbacks; /* BF16 matching: queries re-scanned exactly in FP32 */
  int64_t match_terms;    /* FP32 matching with profiling enabled: descriptor terms (a_k - b_k)^2 evaluated, of
                             nP * nQ * 33 for a scan without early exit; else 0 */
  float fitness;          /* mean squared inlier distance under T (m^2) */
  float hyp_fitness;      /* the same for the selected hypothesis */
  int32_t status;         /* LSR_STATUS_ALIGNED or LSR_STATUS_NO_ALIGNMENT */
  int32_t refine_iters_done;
  float stage_ms[8];      /* per-stage device time when profiling is enabled, else 0:
                             [0] pack+grids [1] normals [2] SPFH+FPFH [3] matching
                             [4] hypotheses [5] consensus [6] selection+refinement [7] total */
} lsr_result;

/* Fill p with the defaults described above. */
LSR_API void lsr_default_params(lsr_params *p);

/* Create a context on CUDA device `device`. params may be NULL (defaults).
 * cuda_stream: a cudaStream_t to order all work on, or NULL for a new
 * non-blocking stream owned by the context. */
LSR_API int lsr_create(lsr_ctx **out, const lsr_params *params, int device, void *cuda_stream);

/* Release the context, its stream (if owned) and its workspace. NULL is a no-op. */
LSR_API int lsr_destroy(lsr_ctx *ctx);

/* Replace the context's parameters (validated; LSR_E_ARG if out of range). */
LSR_API int lsr_set_params(lsr_ctx *ctx, const lsr_params *params);
LSR_API int lsr_get_params(const lsr_ctx *ctx, lsr_params *params);

/* Test hooks: make failures happen without faulting or hanging a GPU, so
 * that the error paths can be exercised. (The paper has no counterpart.)
 *  LSR_INJECT_ALLOC: the next `count` device workspace allocations of this
 *    context fail as if the device were out of memory (no cudaMalloc is made);
 *    the call returns LSR_E_OOM and the context stays usable.
 *  LSR_INJECT_MATCH_STALL: the next `count` tensor-core matcher launches of
 *    this context issue no copy and no MMA, so the first bounded wait of their
 *    epilogue runs out (after 20 ms instead of the normal 2 s); the kernel
 *    releases its tensor memory and returns, and the call returns
 *    LSR_E_TIMEOUT. A batch graph captured while a stall is pending keeps it.
 *  LSR_INJECT_CHECK (checked build only, else LSR_E_ARG): with count > 0, the
 *    next hypothesis-count kernel on the context's stream asks the bounds
 *    checks about one out-of-range index (no memory access follows), so that
 *    call returns LSR_E_CHECK through the same path a real violation takes.
 *  LSR_INJECT_NONE: clear the first two.
 * Returns LSR_OK, LSR_E_ARG (unknown kind, count outside [0, 10^6]) or
 * LSR_E_STATE (NULL context). */
#define LSR_INJECT_NONE 0
#define LSR_INJECT_ALLOC 1
#define LSR_INJECT_MATCH_STALL 2
#define LSR_INJECT_CHECK 3
LSR_API int lsr_debug_inject(lsr_ctx *ctx, int32_t kind, int32_t count);

/* 1 if this library is the checked build (compiled with LSR_CHECKED: device
 * bounds checks on the grid walks, the hypothesis samples and the matchers'
 * rows record the first violation and skip the access; every synchronising
 * call then returns LSR_E_CHECK with the site, index and bound in
 * lsr_last_error), else 0. Results of the two builds are identical. */
LSR_API int lsr_checked_build(void);

/* Per-kernel timing (a profiling aid; the paper has no counterpart). With a
 * non-NULL filter, every kernel launch of a later lsr_register_pair (and of a
 * lsr_register_batch that runs on one stream without a graph) whose kernel
 * name starts with `filter` ("" = every kernel) is bracketed by two CUDA
 * events on the context's stream; after the call has synchronised, the
 * elapsed times are added to a per-kernel table. NULL turns timing off. Each
 * call clears the table. The events add a few microseconds per timed launch.
 * lsr_kernel_timing_count returns the table's entries; lsr_kernel_timing_entry
 * gives entry i: the kernel name (valid until the table is cleared), its timed
 * launches and their total milliseconds. Returns LSR_OK, LSR_E_ARG (filter
 * over 200 characters, i out of range, timing off) or LSR_E_STATE. */
LSR_API int lsr_set_kernel_timing(lsr_ctx *ctx, const char *filter);
LSR_API int32_t lsr_kernel_timing_count(const lsr_ctx *ctx);
LSR_API int lsr_kernel_timing_entry(const lsr_ctx *ctx, int32_t i, const char **name, int64_t *launches,
                                    double *total_ms);

/* Enable (1) or disable (0) per-stage CUDA-event timing in lsr_result.stage_ms. */
LSR_API int lsr_set_profiling(lsr_ctx *ctx, int enable);

/* Static message for a return code, and the last error message of a context. */
LSR_API const char *lsr_error_string(int code);
LSR_API const char *lsr_last_error(const lsr_ctx *ctx);

/* Bytes of device workspace currently held by the context. */
LSR_API int64_t lsr_workspace_bytes(const lsr_ctx *ctx);

/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts); the difference across a call counts that call's launches. */
LSR_API uint64_t lsr_launch_count(void);

/* Bytes a registration of host-resident clouds of nP and nQ points copies
 * host to device (*h2d) and device to host (*d2h) inside lsr_register_pair.
 * Either pointer may be NULL. */
LSR_API int lsr_transfer_bytes(int64_t nP, int64_t nQ, int64_t *h2d, int64_t *d2h);

/* Algorithm 1 followed by the robust refinement, for one pair.
 * P: nP x 3 float32, Q: nQ x 3 float32 (device or host). vpP / vpQ: viewpoints
 * (3 floats, host) the normals of each cloud are oriented toward; NULL means
 * the origin. out: host. nP, nQ >= 4. */
LSR_API int lsr_register_pair(lsr_ctx *ctx, const float *P, int64_t nP, const float *Q, int64_t nQ, const float *vpP,
                      const float *vpQ, lsr_result *out);

/* Batched loop-candidate verification: n independent pairs, pair i with RNG
 * key (seed, pair_id + i). P[i], Q[i]: clouds (device or host); vp: n x 6 host
 * floats (vpP, vpQ per pair) or NULL; out: n host results. Equivalent to n
 * calls of lsr_register_pair, scheduled together. */
LSR_API int lsr_register_batch(lsr_ctx *ctx, int32_t n, const float *const *P, const int64_t *nP, const float *const *Q,
                       const int64_t *nQ, const float *vp, lsr_result *out);

/* ------------------------------------------------------------------------
 * Stage entry points. Each runs one stage of the path on caller-supplied
 * inputs (the same kernels the full registration launches), so that every
 * stage can be checked on its own. Arrays are in the caller's point order.
 * ------------------------------------------------------------------------ */

/* Normals (needed by FPFH, Alg. 1; radius of Sec. IV): eigenvector of
 * the smallest eigenvalue of the covariance of the points within r (inclusive,
 * the point itself included), oriented toward vp; fewer than 3 neighbours give
 * a zero normal and curvature -1. normals: n x 3, count: n (neighbours),
 * curvature: n (lambda0 / sum lambda). Any output may be NULL. */
LSR_API int lsr_stage_normals(lsr_ctx *ctx, const float *P, int64_t n, const float *vp, float r, float *normals, int32_t *count,
                      float *curvature);

/* SPFH (Rusu et al. 2009) of every point from given normals (n x 3, zero =
 * invalid): per pair within r, the Darboux-frame angles (alpha, phi, theta)
 * binned 3 x 11, each sub-histogram scaled to sum 1. spfh: n x 33, k: n pairs
 * used (either may be NULL). */
LSR_API int lsr_stage_spfh(lsr_ctx *ctx, const float *P, const float *normals, int64_t n, float r, float *spfh, int32_t *k);

/* FPFH from given SPFH (n x 33): F(p) = SPFH(p) + (1/k) sum SPFH(q) / |q - p|
 * over valid neighbours within r, each sub-histogram rescaled to sum 1. */
LSR_API int lsr_stage_fpfh(lsr_ctx *ctx, const float *P, const float *normals, const float *spfh, int64_t n, float r,
                   float *fpfh);

/* Feature pre-matching (Alg. 1): nn[i] = argmin_j |FP_i - FQ_j|^2 (ties to the
 * smallest j), d1[i] its squared distance. FP: nP x 33, FQ: nQ x 33.
 * precision: LSR_MATCH_FP32, LSR_MATCH_BF16 or LSR_MATCH_BF16_PLAIN; every
 * precision returns the same nn and d1 (the tensor-core modes re-rank their
 * top-8 candidates in FP32 and re-scan, in FP32, every query for which a
 * rounding-error bound cannot prove that the FP32 winner is a candidate).
 * fallbacks (host, may be NULL): queries re-scanned that way. */
LSR_API int lsr_stage_match(lsr_ctx *ctx, const float *FP, int64_t nP, const float *FQ, int64_t nQ, int32_t precision,
                    int32_t *nn, float *d1, int64_t *fallbacks);

/* The tensor-core contraction behind the BF16 modes (Alg. 1 feature
 * pre-matching, |a - b|^2 = |a|^2 + |b|^2 - 2 a.b), for validation. With c a
 * mean descriptor and a~, b~ the BF16 forms of a - c, b - c (precision as in
 * lsr_stage_match; LSR_MATCH_FP32 is rejected), d2[i * nQ + j] = |b~_j|^2 -
 * 2 a~_i . b~_j + |a~_i|^2 as accumulated in FP32 by the tensor cores: an
 * approximation of |FP_i - FQ_j|^2. FP: nP x 33, FQ: nQ x 33, d2: nP x nQ
 * (host or device); nP, nQ <= 65536. LSR_E_TIMEOUT if a bounded wait ran out. */
LSR_API int lsr_match_scores_bf16(lsr_ctx *ctx, const float *FP, int64_t nP, const float *FQ, int64_t nQ,
                                  int32_t precision, float *d2);

/* Hypothesis sampling + polygon pre-rejection + compaction (Alg. 1). Samples
 * hypotheses h = 0..H-1 with Philox-4x64-10(counter (h,0,0,0), key (seed,
 * pair_id)), index k = floor(word_k * nP / 2^64); rejects repeated indices,
 * invalid points (valid* == 0), cyclic edges shorter than 1e-6, and edges with
 * |p_k - p_k+1| < tau |q_k - q_k+1| or the reverse. surv (capacity cap,
 * device or host): surviving ids in ascending order; *nsurv (host): their
 * number (may exceed cap, in which case only cap ids are written). */
LSR_API int lsr_stage_hypotheses(lsr_ctx *ctx, const float *P, int64_t nP, const float *Q, int64_t nQ, const int32_t *nn,
                         const uint8_t *validP, const uint8_t *validQ, int64_t H, uint64_t seed, uint64_t pair_id,
                         float tau, int32_t *surv, int64_t cap, int64_t *nsurv);

/* Rigid transform from 4 point pairs per hypothesis (Alg. 1, "Estimate
 * transformation"): ps, qs: nh x 4 x 3; Rt: nh x 12 (row-major [R | t]). */
LSR_API int lsr_stage_rigid4(lsr_ctx *ctx, const float *ps, const float *qs, int64_t nh, float *Rt);

/* Consensus (Alg. 1, "Consensus for the remaining quadruple pairs"; grid of
 * eq. (1)): for each pose Rt (nh x 12, row-major [R | t]) count the points of
 * P whose nearest Q point is closer than eps, and sum their squared distances.
 * count: nh int32, sumd2: nh double. */
LSR_API int lsr_stage_consensus(lsr_ctx *ctx, const float *P, int64_t nP, const float *Q, int64_t nQ, const float *Rt,
                        int64_t nh, float eps, int32_t *count, double *sumd2);

/* Pose scoring that allocates nothing. (The paper has no counterpart: this is
 * a service for callers that must not allocate device memory when they score
 * poses -- a loop-closure check inside a real-time loop, or a process whose
 * device memory belongs to another framework's pool.)
 * Same result as lsr_stage_consensus: for each pose Rt (nh x 12, row-major
 * [R | t]), count[k] = points of P whose nearest Q point is closer than eps,
 * sumd2[k] = the sum of their squared distances. P: nP x 3, Q: nQ x 3 float32;
 * Rt, count (int32, nh), sumd2 (double, nh) may be device or host arrays.
 * Scratch comes from one fixed 16 MiB array in the library's device image
 * (held by every GPU that loads the library until the process exits), so:
 *  - limits: nP <= 65536, nQ <= 65536, nh <= 4096, else LSR_E_TOO_LARGE;
 *  - no context is needed; work runs on the calling thread's current device,
 *    on cuda_stream (NULL: the legacy default stream), and the call
 *    synchronises that stream before returning;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it; the cached address does not
 *    survive a reset of the device (cudaDeviceReset), after which the call
 *    must not be used;
 *  - every call on a device shares the array, which keeps the previous call's
 *    contents (the call clears what must start at zero): calls that overlap
 *    on the GPU (other streams, other host threads) race and must not be
 *    issued.
 * Returns LSR_OK, LSR_E_ARG, LSR_E_TOO_LARGE or LSR_E_CUDA. */
LSR_API int lsr_consensus_static(const float *P, int64_t nP, const float *Q, int64_t nQ, const float *Rt, int64_t nh,
                                 float eps, int32_t *count, double *sumd2, void *cuda_stream);

/* Consensus with the variant modes of lsr_params (nn_mode, normal_mode), on
 * caller-supplied inputs: for each pose Rt (nh x 12, row-major [R | t]),
 * count[k] = points p of P whose nearest Q point q -- exact (LSR_NN_EXACT) or
 * in p's own cell of the eps lattice through Q's centroid
 * (LSR_NN_SINGLE_CELL, eq. (1)) -- is closer than eps and, with
 * LSR_NORMALS_INLIERS, whose rotated normal R n_p agrees with n_q
 * (cos >= cos_normal, both normals non-zero); sumd2[k] = the sum of their
 * squared distances. NP (nP x 3), NQ (nQ x 3): normals in the caller's order
 * (zero = invalid), needed only with LSR_NORMALS_INLIERS. Every array may be
 * device or host. The registration pipeline runs the same kernels when the
 * context's modes are not the defaults. */
LSR_API int lsr_stage_consensus_modes(lsr_ctx *ctx, const float *P, const float *NP, int64_t nP, const float *Q,
                                      const float *NQ, int64_t nQ, const float *Rt, int64_t nh, float eps,
                                      int32_t nn_mode, int32_t normal_mode, float cos_normal, int32_t *count,
                                      double *sumd2);

/* Nearest neighbours of the consensus (eq. (1) and the inlier test of Alg.
 * 1): for every query x (X: nX x 3 float32), the nearest point of Q (nQ x 3
 * float32), both device or host. mode LSR_NN_EXACT: the nearest Q point
 * within r over every grid cell the r-ball overlaps (ties to the smaller
 * index). mode LSR_NN_SINGLE_CELL: the O(1) lookup of eq. (1): Q binned into
 * cells of edge r on a lattice through Q's centroid c (cell index
 * floor((x - c) / r) per axis, evaluated in FP32), and the nearest point of
 * the query's own cell, at any distance. nn (nX int32, device or host): the Q
 * index or -1 (none within r / empty cell); d2 (nX float32, may be NULL): its
 * squared distance or +inf. */
LSR_API int lsr_stage_nn(lsr_ctx *ctx, const float *Q, int64_t nQ, const float *X, int64_t nX, float r, int32_t mode,
                         int32_t *nn, float *d2);

/* Graduated robust refinement from T_in (host, 4x4 row-major double). Level
 * l = 0..levels-1 iterates Geman-McClure IRLS (at most iters steps) with exact
 * NN within r_l = eps * 2^(levels-1-l), mu_l = mu_scale * r_l^2, on the points
 * of P and Q whose caller index is a multiple of s_l = max(1, min(4^(levels-1-l),
 * N / 4096)) (per cloud). T_out (host, double[16]); iters_done (host, may be
 * NULL): total steps taken. */
LSR_API int lsr_stage_refine(lsr_ctx *ctx, const float *P, int64_t nP, const float *Q, int64_t nQ, const double *T_in,
                             float eps, float mu_scale, int32_t levels, int32_t iters, double *T_out,
                             int32_t *iters_done);

/* ------------------------------------------------------------------------
 * Robust alignment objective (the refinement's cost, eq. (3)-(4) with the
 * line process eliminated) and its adjoint, for n pairs.
 * Pair i: E_i = sum_j rho~(|T_i p_j - q_nn(j)|^2) over the points whose nearest
 * Q point is within eps, with T_i = [Exp(xi_i[0:3]) | xi_i[3:6]] * T0_i
 * (xi = (alpha, beta, gamma, x, y, z) as in eq. (5)), rho(s) = mu s / (mu + s)
 * and rho~(s) = rho(s) - rho(eps^2). Nearest neighbours are recomputed by the
 * backward call, never stored.
 * P[i], Q[i]: device float32 clouds; xi: n x 6 double; T0: n x 16 double;
 * E: n double (all host or all device, as the point arrays). dE: n double
 * upstream gradients. dP[i], dQ[i]: device float32 gradients (written, not
 * accumulated), dxi: n x 6 double.
 * ------------------------------------------------------------------------ */
LSR_API int lsr_objective_fwd(lsr_ctx *ctx, int32_t n, const float *const *P, const int64_t *nP, const float *const *Q,
                      const int64_t *nQ, const double *xi, const double *T0, float eps, float mu, double *E);
LSR_API int lsr_objective_bwd(lsr_ctx *ctx, int32_t n, const float *const *P, const int64_t *nP, const float *const *Q,
                      const int64_t *nQ, const double *xi, const double *T0, float eps, float mu, const double *dE,
                      float *const *dP, float *const *dQ, double *dxi);

/* Information matrix of a verified pair (loop verification, eq. (5)-(6)):
 * info = sum over the correspondences K of G_p^T G_p, G_p = [-[p]_x | I],
 * where K holds the points p = T p' (p' in P, moved into Q's frame by the
 * row-major 4x4 pose T) whose nearest Q point is closer than eps (the paper
 * takes eps = 0.05 m). xi^T info xi is then the first-order alignment error of
 * the pair under a small motion xi = (alpha, beta, gamma, x, y, z).
 * P: nP x 3, Q: nQ x 3 float32, device or host. T: 16 double, host.
 * info: 36 double, host, row-major (symmetric); n_corr (host, may be NULL):
 * |K|. Sums in FP32 per thread about the centre of Q's box, FP64 across
 * blocks in a fixed order (deterministic). Errors: LSR_E_ARG for null
 * pointers, sizes outside [1, 2^26], eps outside (0, 10] or a non-finite T. */
LSR_API int lsr_information_matrix(lsr_ctx *ctx, const float *P, int64_t nP, const float *Q, int64_t nQ,
                                   const double *T, float eps, double *info, int64_t *n_corr);

/* Gradient of the refined pose with respect to the points (implicit
 * differentiation of the robust alignment of eq. (3)-(4) at its optimum; the
 * pose perturbation of eq. (5)). At the refined pose T (the pose
 * lsr_stage_refine or lsr_register_pair returns), the held pairs are the
 * points p of P whose nearest Q point q lies within eps under T (the finest
 * refinement level's correspondences, recomputed here), rho(s) = mu s /
 * (mu + s). The optimality condition g(T) = 0 of E = sum rho(|T p - q|^2)
 * makes T a function of the points; for a loss L with gradient dL_dT
 * (host, 16 doubles, row-major d L / d T; the last row is ignored), it gives
 *   lambda = H^-1 dL/dxi,  dL/dp = -R^T d(lambda . g_p)/dz,  dL/dq = -d(lambda . g_p)/dq,
 * with xi = (w, v) the left perturbation T(xi) = [Exp(w) | v] T, g_p the pair's
 * term of the gradient of E in xi and H its exact Hessian (rho'' and the
 * second-order term of Exp included).
 * P: nP x 3, Q: nQ x 3 float32 (device or host). T: 16 doubles (host).
 * dP (nP x 3) and dQ (nQ x 3) float32: both device or both host, written
 * (points without a pair get 0; a Q point sums the terms of every pair it
 * closes). grad (6), hess (36, row-major), lambda (6): host doubles, each may
 * be NULL: g, H and lambda at T. n_corr (host, may be NULL): held pairs. The
 * terms are evaluated and summed in FP64 (fixed order over blocks), the
 * neighbours found in FP32, dQ scattered with FP32 atomics. Errors: LSR_E_ARG
 * for null pointers, sizes outside [1, 2^26], eps outside (0, 10], mu <= 0, a
 * non-finite T or dL_dT, or a singular H (too few pairs). */
LSR_API int lsr_pose_implicit_grad(lsr_ctx *ctx, const float *P, int64_t nP, const float *Q, int64_t nQ,
                                   const double *T, float eps, float mu, const double *dL_dT, float *dP, float *dQ,
                                   double *grad, double *hess, double *lambda, int64_t *n_corr);

/* Voxel downsampling (Algorithm 1, first line): one point per occupied voxel
 * of edge leaf, the mean of the points in it. Voxels are aligned to the
 * coordinate origin (key = floor(x / leaf) per axis, evaluated in FP64) and
 * the output is ordered by voxel, z slowest, then y, then x. The means come
 * from 64-bit integer sums of the offsets from the voxel corner (units of
 * leaf / 2^36), so they do not depend on the order of the points.
 * P: n x 3 float32 (device or host). out: cap x 3 float32 (device or host);
 * at most cap points are written and *n_out (host) receives the number of
 * occupied voxels (cap = n always suffices). Errors: LSR_E_ARG for null
 * pointers, n outside [1, 2^26], leaf outside (0, 100]; LSR_E_TOO_LARGE when
 * the keys' bounding box holds more than 2^26 voxels. */
LSR_API int lsr_voxel_downsample(lsr_ctx *ctx, const float *P, int64_t n, float leaf, float *out, int64_t cap,
                                 int64_t *n_out);

/* Dense model correction after a loop closure (eq. (7)): every surfel moves
 * with the keyframes that observe it,
 *   p' = (1/k) sum_{f in F} T_f_new T_f_old^-1 p,
 *   n' = normalize(sum_{f in F} R_f_new R_f_old^-1 n),
 * F = the keyframes with t0 < t_f < tu (the surfel's initialisation and
 * last-update stamps) whose camera before the correction sees the surfel:
 * z > 0 and z <= max depth in the camera frame, and the pinhole projection
 * u = fx x / z + cx, v = fy y / z + cy inside [0, width) x [0, height).
 * A surfel with k = |F| = 0 is removed: keep = 0, p and n copied unchanged.
 * pos, nrm: n x 3 float32; t0, tu: n float32 (device or host). T_old, T_new:
 * m x 16 double row-major rigid camera-to-world poses; t_kf: m float32 in
 * ascending order; cam: 7 float32 (fx, fy, cx, cy, width, height, max depth)
 * (all host). pos_out, nrm_out (n x 3 float32) and keep (n bytes): all device
 * or all host; n_keep (host, may be NULL): surfels kept. FP32 on the device,
 * the keyframe transforms composed in FP64 on the host. Errors: LSR_E_ARG for
 * null pointers, n outside [1, 2^31], m outside [1, 2^20], non-ascending
 * stamps, a non-finite pose or a non-positive camera parameter. */
LSR_API int lsr_surfel_correct(lsr_ctx *ctx, int64_t n, const float *pos, const float *nrm, const float *t0,
                               const float *tu, int32_t m, const double *T_old, const double *T_new,
                               const float *t_kf, const float *cam, float *pos_out, float *nrm_out, uint8_t *keep,
                               int64_t *n_keep);

#ifdef __cplusplus
}
#endif

#endif /* LSR_H */
