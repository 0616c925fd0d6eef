/*
 * lsr_oracle.c -- plain, slow, FP64 CPU oracle for the global point-cloud
 * registration of LoopSmart (Zhang & Chen, arXiv 1801.01572), Sec. IV,
 * Algorithm 1, eq. (1), and the robust pose objective of eq. (3)-(5).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py are the only callers. The product
 * path (the CUDA library) never links, loads or calls this file, and the two
 * share no code, headers, tables or constants.
 *
 * Conventions. Points are row-major N x 3 doubles. Descriptors are N x 33
 * doubles (alpha bins 0..10, phi bins 11..21, theta bins 22..32). A normal of
 * (0,0,0) marks a point whose neighbourhood was too small (fewer than 3
 * points); such a point has a zero descriptor and is never sampled.
 *
 * Where the paper is silent the reading taken is stated at each function.
 * Parity is pinned for every function here by the CPU tests (brute force on
 * tiny inputs, closed forms, invariances, an independent library Philox).
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_D 33
#define ORC_NB 11

/* ------------------------------------------------------------------------ */
/* Parallel for: worker threads pull fixed-size chunks from an atomic        */
/* counter. Results never depend on the thread count: every reduction below */
/* is done per fixed chunk and summed in chunk order.                       */
/* ------------------------------------------------------------------------ */
static int g_threads = 0;

void orc_set_threads(int n) { g_threads = n; }

int orc_get_threads(void) {
  if (g_threads > 0) return g_threads;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

typedef void (*orc_body)(void *ctx, int64_t lo, int64_t hi);
typedef struct {
  orc_body fn;
  void *ctx;
  int64_t n, chunk;
  atomic_llong next;
} orc_pf;

static void *orc_pf_worker(void *arg) {
  orc_pf *pf = (orc_pf *)arg;
  for (;;) {
    int64_t lo = atomic_fetch_add(&pf->next, pf->chunk);
    if (lo >= pf->n) break;
    int64_t hi = lo + pf->chunk < pf->n ? lo + pf->chunk : pf->n;
    pf->fn(pf->ctx, lo, hi);
  }
  return NULL;
}

static void orc_parallel_for(int64_t n, int64_t chunk, orc_body fn, void *ctx) {
  if (n <= 0) return;
  if (chunk < 1) chunk = 1;
  orc_pf pf;
  pf.fn = fn;
  pf.ctx = ctx;
  pf.n = n;
  pf.chunk = chunk;
  atomic_init(&pf.next, 0);
  int nt = orc_get_threads();
  int64_t nchunks = (n + chunk - 1) / chunk;
  if (nt > nchunks) nt = (int)nchunks;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)(nt > 1 ? nt - 1 : 1));
  int started = 0;
  for (int i = 0; i < nt - 1; ++i)
    if (pthread_create(&th[i], NULL, orc_pf_worker, &pf) == 0) ++started;
  orc_pf_worker(&pf);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free(th);
}

/* ------------------------------------------------------------------------ */
/* Small vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double dist2(const double *a, const double *b) {
  double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return dx * dx + dy * dy + dz * dz;
}
static inline int is_zero3(const double *a) { return a[0] == 0.0 && a[1] == 0.0 && a[2] == 0.0; }

/* y = R x + t with R row-major 3x3 */
static inline void xform(const double *R, const double *t, const double *x, double *y) {
  y[0] = R[0] * x[0] + R[1] * x[1] + R[2] * x[2] + t[0];
  y[1] = R[3] * x[0] + R[4] * x[1] + R[5] * x[2] + t[1];
  y[2] = R[6] * x[0] + R[7] * x[1] + R[8] * x[2] + t[2];
}

/* ------------------------------------------------------------------------ */
/* Exact radius search on a uniform grid (eq. (1) cell indexing, read with  */
/* a floor). The cell edge is the search radius times 1.001, so the 27      */
/* cells around a query contain every point within the radius (and within  */
/* 0.1 % beyond it, which the margin diagnostics need). Exactness does not  */
/* depend on the grid: it only prunes points that are provably too far.    */
/* The CPU tests pin it against brute force.                                */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t k[3];
  int64_t idx;
} orc_cell_entry;

typedef struct {
  double cell, o[3];
  int64_t n, g[3];
  orc_cell_entry *e; /* sorted by (k2, k1, k0, idx) */
} orc_grid;

static int cmp_entry(const void *a, const void *b) {
  const orc_cell_entry *x = (const orc_cell_entry *)a, *y = (const orc_cell_entry *)b;
  for (int d = 2; d >= 0; --d) {
    if (x->k[d] != y->k[d]) return x->k[d] < y->k[d] ? -1 : 1;
  }
  return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

static void grid_build(orc_grid *g, const double *P, int64_t n, double radius) {
  g->cell = radius * 1.001;
  g->n = n;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      if (P[3 * i + d] < lo[d]) lo[d] = P[3 * i + d];
      if (P[3 * i + d] > hi[d]) hi[d] = P[3 * i + d];
    }
  for (int d = 0; d < 3; ++d) {
    g->o[d] = n > 0 ? lo[d] : 0.0;
    g->g[d] = n > 0 ? (int64_t)floor((hi[d] - lo[d]) / g->cell) + 1 : 1;
  }
  g->e = (orc_cell_entry *)malloc(sizeof(orc_cell_entry) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    for (int d = 0; d < 3; ++d) g->e[i].k[d] = (int64_t)floor((P[3 * i + d] - g->o[d]) / g->cell);
    g->e[i].idx = i;
  }
  qsort(g->e, (size_t)n, sizeof(orc_cell_entry), cmp_entry);
}

static void grid_free(orc_grid *g) {
  free(g->e);
  g->e = NULL;
}

/* first entry with key >= k (idx ignored) */
static int64_t grid_lower(const orc_grid *g, const int64_t *k) {
  int64_t lo = 0, hi = g->n;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    const int64_t *m = g->e[mid].k;
    int less = 0;
    for (int d = 2; d >= 0; --d) {
      if (m[d] != k[d]) {
        less = m[d] < k[d];
        goto done;
      }
    }
  done:
    if (less)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

/* Visit every point in the 27 cells around x. The visitor gets the index and
 * the squared distance. Queries far outside the grid visit nothing. */
typedef void (*orc_visit)(void *ctx, int64_t j, double d2);

static void grid_visit(const orc_grid *g, const double *P, const double *x, orc_visit fn, void *ctx) {
  double c[3];
  for (int d = 0; d < 3; ++d) {
    c[d] = floor((x[d] - g->o[d]) / g->cell);
    if (!(c[d] >= -2.0 && c[d] <= (double)g->g[d] + 1.0)) return; /* also rejects NaN */
  }
  int64_t base[3] = {(int64_t)c[0], (int64_t)c[1], (int64_t)c[2]};
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t k[3] = {base[0] + dx, base[1] + dy, base[2] + dz};
        for (int64_t s = grid_lower(g, k); s < g->n; ++s) {
          const orc_cell_entry *e = &g->e[s];
          if (e->k[0] != k[0] || e->k[1] != k[1] || e->k[2] != k[2]) break;
          fn(ctx, e->idx, dist2(P + 3 * e->idx, x));
        }
      }
}

/* Growable index list used by the visitors */
typedef struct {
  int64_t *idx;
  double *d2;
  int64_t n, cap;
  double r2, margin_band2_lo, margin_band2_hi;
  int64_t n_near_edge; /* points whose squared distance is within the band of r^2 */
} orc_list;

static void list_push(orc_list *L, int64_t j, double d2) {
  if (L->n == L->cap) {
    L->cap = L->cap ? 2 * L->cap : 256;
    L->idx = (int64_t *)realloc(L->idx, sizeof(int64_t) * (size_t)L->cap);
    L->d2 = (double *)realloc(L->d2, sizeof(double) * (size_t)L->cap);
  }
  L->idx[L->n] = j;
  L->d2[L->n] = d2;
  L->n++;
}

static void visit_radius(void *ctx, int64_t j, double d2) {
  orc_list *L = (orc_list *)ctx;
  if (d2 >= L->margin_band2_lo && d2 <= L->margin_band2_hi) L->n_near_edge++;
  if (d2 <= L->r2) list_push(L, j, d2);
}

static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Neighbours of x with ||p - x||^2 <= r^2, returned in ascending index order.
 * band: relative band on r^2 counted as "near the radius" (for margins). */
static void radius_query(const orc_grid *g, const double *P, const double *x, double r, double band, orc_list *L) {
  L->n = 0;
  L->n_near_edge = 0;
  L->r2 = r * r;
  L->margin_band2_lo = r * r * (1.0 - band);
  L->margin_band2_hi = r * r * (1.0 + band);
  grid_visit(g, P, x, visit_radius, L);
  /* sort ascending by index (d2 recomputed by callers where needed) */
  if (L->n > 1) {
    qsort(L->idx, (size_t)L->n, sizeof(int64_t), cmp_i64);
    for (int64_t s = 0; s < L->n; ++s) L->d2[s] = dist2(P + 3 * L->idx[s], x);
  }
}

static void list_free(orc_list *L) {
  free(L->idx);
  free(L->d2);
  L->idx = NULL;
  L->d2 = NULL;
  L->n = L->cap = 0;
}

/* Public: brute-force and grid radius counts, used by the tests to pin the
 * grid against the definition. */
void orc_radius_count_brute(const double *P, int64_t n, const double *X, int64_t m, double r, int64_t *count) {
  for (int64_t i = 0; i < m; ++i) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j)
      if (dist2(P + 3 * j, X + 3 * i) <= r * r) ++c;
    count[i] = c;
  }
}

void orc_radius_count_grid(const double *P, int64_t n, const double *X, int64_t m, double r, int64_t *count) {
  orc_grid g;
  grid_build(&g, P, n, r);
  orc_list L = {0};
  for (int64_t i = 0; i < m; ++i) {
    radius_query(&g, P, X + 3 * i, r, 0.0, &L);
    count[i] = L.n;
  }
  list_free(&L);
  grid_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations, run until  */
/* the off-diagonal part is below 1e-30 of the squared Frobenius norm.      */
/* Eigenvalues ascending in w[], eigenvectors in the columns of V.          */
/* ------------------------------------------------------------------------ */
static void jacobi3(const double A_in[9], double w[3], double V[9]) {
  double A[9];
  memcpy(A, A_in, sizeof(A));
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < 9; ++i) fro += A[i] * A[i];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    if (off <= 1e-30 * fro || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        double apq = A[3 * p + q];
        if (apq == 0.0) continue;
        double app = A[3 * p + p], aqq = A[3 * q + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* A <- J^T A J with the rotation in the (p,q) plane */
        for (int k = 0; k < 3; ++k) {
          double akp = A[3 * k + p], akq = A[3 * k + q];
          A[3 * k + p] = c * akp - s * akq;
          A[3 * k + q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          double apk = A[3 * p + k], aqk = A[3 * q + k];
          A[3 * p + k] = c * apk - s * aqk;
          A[3 * q + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = V[3 * k + p], vkq = V[3 * k + q];
          V[3 * k + p] = c * vkp - s * vkq;
          V[3 * k + q] = s * vkp + c * vkq;
        }
      }
  }
  double d[3] = {A[0], A[4], A[8]};
  int ord[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (d[ord[j]] < d[ord[i]]) {
        int tmp = ord[i];
        ord[i] = ord[j];
        ord[j] = tmp;
      }
  double Vs[9];
  for (int c = 0; c < 3; ++c) {
    w[c] = d[ord[c]];
    for (int r = 0; r < 3; ++r) Vs[3 * r + c] = V[3 * r + ord[c]];
  }
  memcpy(V, Vs, sizeof(Vs));
}

void orc_eig3(const double A[9], double w[3], double V[9]) { jacobi3(A, w, V); }

/* ------------------------------------------------------------------------ */
/* Normals (needed by the FPFH step of Alg. 1; radius r_n of Sec. IV).      */
/* Reading: the paper does not state the method. The normal is the          */
/* eigenvector of the smallest eigenvalue of the covariance of all points  */
/* with ||q - p||^2 <= r^2 (p itself included), oriented so that            */
/* n . (vp - p) >= 0. With fewer than 3 neighbours the normal is invalid   */
/* (zero) and the curvature is -1.                                          */
/* diag per query: [ (l1 - l0) / max(l2, tiny), |n . (vp - p)| / |vp - p|,  */
/*                   number of points within 1e-5 relative of r^2 ]         */
/* ------------------------------------------------------------------------ */
typedef struct {
  const double *P, *vp;
  int64_t n;
  double r;
  const int64_t *qidx;
  double *nrm, *curv, *diag;
  int64_t *cnt;
  const orc_grid *g;
} normals_ctx;

static void normals_body(void *vctx, int64_t lo, int64_t hi) {
  normals_ctx *c = (normals_ctx *)vctx;
  orc_list L = {0};
  for (int64_t s = lo; s < hi; ++s) {
    int64_t i = c->qidx ? c->qidx[s] : s;
    const double *p = c->P + 3 * i;
    radius_query(c->g, c->P, p, c->r, 1e-5, &L);
    int64_t k = L.n;
    c->cnt[s] = k;
    c->diag[3 * s + 2] = (double)L.n_near_edge;
    double *n = c->nrm + 3 * s;
    if (k < 3) {
      n[0] = n[1] = n[2] = 0.0;
      c->curv[s] = -1.0;
      c->diag[3 * s + 0] = 0.0;
      c->diag[3 * s + 1] = 0.0;
      continue;
    }
    double mu[3] = {0, 0, 0};
    for (int64_t a = 0; a < k; ++a)
      for (int d = 0; d < 3; ++d) mu[d] += c->P[3 * L.idx[a] + d];
    for (int d = 0; d < 3; ++d) mu[d] /= (double)k;
    double C[9] = {0};
    for (int64_t a = 0; a < k; ++a) {
      double v[3];
      for (int d = 0; d < 3; ++d) v[d] = c->P[3 * L.idx[a] + d] - mu[d];
      for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) C[3 * r + q] += v[r] * v[q];
    }
    for (int q = 0; q < 9; ++q) C[q] /= (double)k;
    double w[3], V[9];
    jacobi3(C, w, V);
    n[0] = V[0];
    n[1] = V[3];
    n[2] = V[6];
    double tv[3] = {c->vp[0] - p[0], c->vp[1] - p[1], c->vp[2] - p[2]};
    double o = dot3(n, tv);
    if (o < 0.0) {
      n[0] = -n[0];
      n[1] = -n[1];
      n[2] = -n[2];
    }
    double sum = w[0] + w[1] + w[2];
    c->curv[s] = sum > 0.0 ? w[0] / sum : 0.0;
    c->diag[3 * s + 0] = (w[1] - w[0]) / (w[2] > 1e-300 ? w[2] : 1e-300);
    double tn = sqrt(dot3(tv, tv));
    c->diag[3 * s + 1] = tn > 0 ? fabs(o) / tn : 0.0;
  }
  list_free(&L);
}

void orc_normals(const double *P, int64_t n, const double vp[3], double r, const int64_t *qidx, int64_t nq,
                 double *nrm, double *curv, int64_t *cnt, double *diag) {
  orc_grid g;
  grid_build(&g, P, n, r);
  normals_ctx c = {P, vp, n, r, qidx, nrm, curv, diag, cnt, &g};
  orc_parallel_for(qidx ? nq : n, 64, normals_body, &c);
  grid_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Point-pair features of FPFH (Rusu, Blodow, Beetz, ICRA 2009, cited by    */
/* the paper as the descriptor of Alg. 1's FPFH step).                      */
/* Source is the point whose normal makes the smaller angle with the line  */
/* joining the two points (|n . e| larger; ties keep p as source).          */
/* Darboux frame u = n_s, v = (u x e)/|u x e|, w = u x v, e = (p_t-p_s)/d.  */
/* alpha = v . n_t, phi = u . e, theta = atan2(w . n_t, u . n_t).           */
/* A pair with |u x e|^2 < 1e-12 has no frame and is skipped.              */
/* ------------------------------------------------------------------------ */
#define ORC_FRAME_EPS2 1e-12

static int pair_features_oriented(const double *ps, const double *ns, const double *pt, const double *nt, double f[3],
                                  double *vn2_out) {
  double e[3] = {pt[0] - ps[0], pt[1] - ps[1], pt[2] - ps[2]};
  double d = sqrt(dot3(e, e));
  for (int k = 0; k < 3; ++k) e[k] /= d;
  double v[3];
  cross3(ns, e, v);
  double vn2 = dot3(v, v);
  if (vn2_out) *vn2_out = vn2;
  if (vn2 < ORC_FRAME_EPS2) return 0;
  double vn = sqrt(vn2);
  for (int k = 0; k < 3; ++k) v[k] /= vn;
  double w[3];
  cross3(ns, v, w);
  f[0] = dot3(v, nt);
  f[1] = dot3(ns, e);
  f[2] = atan2(dot3(w, nt), dot3(ns, nt));
  return 1;
}

/* feature -> continuous bin coordinate x in [0, 11); bin = clamp(floor(x)) */
static inline double feat_x(int which, double f) {
  if (which < 2) return (f + 1.0) * 0.5 * (double)ORC_NB;
  return (f + M_PI) / (2.0 * M_PI) * (double)ORC_NB;
}
static inline int x_bin(double x) {
  int b = (int)floor(x);
  if (b < 0) b = 0;
  if (b > ORC_NB - 1) b = ORC_NB - 1;
  return b;
}
/* distance from x to the nearest interior bin edge (1..10) */
static inline double x_edge_margin(double x) {
  double m = INFINITY;
  for (int e = 1; e < ORC_NB; ++e) {
    double dd = fabs(x - (double)e);
    if (dd < m) m = dd;
  }
  return m;
}

/* Public for tests: features of one ordered/unordered pair.
 * returns 1 if the pair contributes; f = (alpha, phi, theta). */
int orc_pair_features(const double ps[3], const double ns[3], const double pt[3], const double nt[3], double f[3]) {
  double e[3] = {pt[0] - ps[0], pt[1] - ps[1], pt[2] - ps[2]};
  double d = sqrt(dot3(e, e));
  if (d == 0.0) return 0;
  double cs = fabs(dot3(ns, e)) / d, ct = fabs(dot3(nt, e)) / d;
  if (cs < ct) return pair_features_oriented(pt, nt, ps, ns, f, NULL);
  return pair_features_oriented(ps, ns, pt, nt, f, NULL);
}

/* SPFH of the query points. delta: bin-coordinate band counted as "close to
 * a bin edge". nclose counts contributing-or-borderline pairs whose bins could
 * differ under small perturbations: a feature within delta of a bin edge, a
 * source/target choice within 1e-6 whose alternative gives other bins, a
 * frame norm near the skip threshold, or a distance near the radius. */
typedef struct {
  const double *P, *N;
  int64_t n;
  double r, delta;
  const int64_t *qidx;
  double *spfh;
  int64_t *k, *nclose;
  const orc_grid *g;
} spfh_ctx;

static void spfh_body(void *vctx, int64_t lo, int64_t hi) {
  spfh_ctx *c = (spfh_ctx *)vctx;
  orc_list L = {0};
  for (int64_t s = lo; s < hi; ++s) {
    int64_t i = c->qidx ? c->qidx[s] : s;
    double *h = c->spfh + (size_t)ORC_D * s;
    for (int b = 0; b < ORC_D; ++b) h[b] = 0.0;
    c->k[s] = 0;
    c->nclose[s] = 0;
    const double *pi = c->P + 3 * i, *ni = c->N + 3 * i;
    if (is_zero3(ni)) continue;
    radius_query(c->g, c->P, pi, c->r, 1e-5, &L);
    int64_t kk = 0, close = L.n_near_edge;
    for (int64_t a = 0; a < L.n; ++a) {
      int64_t j = L.idx[a];
      if (j == i || L.d2[a] == 0.0) continue;
      const double *pj = c->P + 3 * j, *nj = c->N + 3 * j;
      if (is_zero3(nj)) continue;
      double e[3] = {pj[0] - pi[0], pj[1] - pi[1], pj[2] - pi[2]};
      double d = sqrt(L.d2[a]);
      double cs = fabs(dot3(ni, e)) / d, ct = fabs(dot3(nj, e)) / d;
      int swap = cs < ct;
      double f[3], vn2;
      int ok = swap ? pair_features_oriented(pj, nj, pi, ni, f, &vn2) : pair_features_oriented(pi, ni, pj, nj, f, &vn2);
      int is_close = (vn2 > 0.25 * ORC_FRAME_EPS2 && vn2 < 4.0 * ORC_FRAME_EPS2);
      if (fabs(cs - ct) < 1e-6) {
        double f2[3], vn2b;
        int ok2 = swap ? pair_features_oriented(pi, ni, pj, nj, f2, &vn2b) : pair_features_oriented(pj, nj, pi, ni, f2, &vn2b);
        if (ok2 != ok)
          is_close = 1;
        else if (ok)
          for (int q = 0; q < 3; ++q)
            if (x_bin(feat_x(q, f[q])) != x_bin(feat_x(q, f2[q]))) is_close = 1;
      }
      if (!ok) {
        close += is_close;
        continue;
      }
      for (int q = 0; q < 3; ++q) {
        double x = feat_x(q, f[q]);
        if (x_edge_margin(x) < c->delta) is_close = 1;
        h[q * ORC_NB + x_bin(x)] += 1.0;
      }
      close += is_close;
      ++kk;
    }
    if (kk > 0)
      for (int b = 0; b < ORC_D; ++b) h[b] /= (double)kk;
    c->k[s] = kk;
    c->nclose[s] = close;
  }
  list_free(&L);
}

void orc_spfh(const double *P, const double *N, int64_t n, double r, const int64_t *qidx, int64_t nq, double delta,
              double *spfh, int64_t *k, int64_t *nclose) {
  orc_grid g;
  grid_build(&g, P, n, r);
  spfh_ctx c = {P, N, n, r, delta, qidx, spfh, k, nclose, &g};
  orc_parallel_for(qidx ? nq : n, 32, spfh_body, &c);
  grid_free(&g);
}

/* ------------------------------------------------------------------------ */
/* FPFH (Rusu 2009): F(p) = SPFH(p) + (1/k) sum_{q in N(p)} SPFH(q) / |q-p| */
/* over the valid-normal neighbours q != p with 0 < |q-p| <= r. Reading:    */
/* each 11-bin sub-histogram of F is then rescaled to sum 1.                */
/* spfh holds the SPFH of ALL n points.                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  const double *P, *N, *spfh;
  int64_t n;
  double r;
  const int64_t *qidx;
  double *fpfh;
  const orc_grid *g;
} fpfh_ctx;

static void fpfh_body(void *vctx, int64_t lo, int64_t hi) {
  fpfh_ctx *c = (fpfh_ctx *)vctx;
  orc_list L = {0};
  for (int64_t s = lo; s < hi; ++s) {
    int64_t i = c->qidx ? c->qidx[s] : s;
    double *F = c->fpfh + (size_t)ORC_D * s;
    for (int b = 0; b < ORC_D; ++b) F[b] = 0.0;
    if (is_zero3(c->N + 3 * i)) continue;
    radius_query(c->g, c->P, c->P + 3 * i, c->r, 0.0, &L);
    double acc[ORC_D] = {0};
    int64_t kk = 0;
    for (int64_t a = 0; a < L.n; ++a) {
      int64_t j = L.idx[a];
      if (j == i || L.d2[a] == 0.0 || is_zero3(c->N + 3 * j)) continue;
      double w = 1.0 / sqrt(L.d2[a]);
      for (int b = 0; b < ORC_D; ++b) acc[b] += w * c->spfh[(size_t)ORC_D * j + b];
      ++kk;
    }
    for (int b = 0; b < ORC_D; ++b) F[b] = c->spfh[(size_t)ORC_D * i + b] + (kk > 0 ? acc[b] / (double)kk : 0.0);
    for (int q = 0; q < 3; ++q) {
      double sum = 0.0;
      for (int b = 0; b < ORC_NB; ++b) sum += F[q * ORC_NB + b];
      if (sum > 0.0)
        for (int b = 0; b < ORC_NB; ++b) F[q * ORC_NB + b] /= sum;
    }
  }
  list_free(&L);
}

void orc_fpfh(const double *P, const double *N, const double *spfh, int64_t n, double r, const int64_t *qidx, int64_t nq,
              double *fpfh) {
  orc_grid g;
  grid_build(&g, P, n, r);
  fpfh_ctx c = {P, N, spfh, n, r, qidx, fpfh, &g};
  orc_parallel_for(qidx ? nq : n, 32, fpfh_body, &c);
  grid_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Feature pre-matching cache (Alg. 1, "Parallel FPFH feature pre-matching"):*/
/* nn[i] = argmin_j ||F(p_i) - F(q_j)||^2 by brute force, ties to the       */
/* smallest j. d1, d2 = smallest and second smallest squared distance.     */
/* ------------------------------------------------------------------------ */
typedef struct {
  const double *A, *B;
  int64_t nb, dim;
  const int64_t *qidx;
  int64_t *nn;
  double *d1, *d2;
} match_ctx;

static void match_body(void *vctx, int64_t lo, int64_t hi) {
  match_ctx *c = (match_ctx *)vctx;
  for (int64_t s = lo; s < hi; ++s) {
    int64_t i = c->qidx ? c->qidx[s] : s;
    const double *a = c->A + (size_t)c->dim * i;
    double b1 = INFINITY, b2 = INFINITY;
    int64_t j1 = -1;
    for (int64_t j = 0; j < c->nb; ++j) {
      const double *b = c->B + (size_t)c->dim * j;
      double d = 0.0;
      for (int64_t k = 0; k < c->dim; ++k) {
        double t = a[k] - b[k];
        d += t * t;
      }
      if (d < b1) {
        b2 = b1;
        b1 = d;
        j1 = j;
      } else if (d < b2) {
        b2 = d;
      }
    }
    c->nn[s] = j1;
    c->d1[s] = b1;
    c->d2[s] = b2;
  }
}

void orc_match(const double *A, int64_t na, const double *B, int64_t nb, int64_t dim, const int64_t *qidx, int64_t nq,
               int64_t *nn, double *d1, double *d2) {
  match_ctx c = {A, B, nb, dim, qidx, nn, d1, d2};
  (void)na;
  orc_parallel_for(qidx ? nq : na, 16, match_body, &c);
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers for "randomly picked (p0,p1,p2,p3)" of      */
/* Alg. 1: Philox-4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11),  */
/* written from its published definition: each round multiplies words 0    */
/* and 2 by the two round multipliers, and the key is bumped by the two    */
/* Weyl constants between rounds.                                           */
/* Hypothesis h of a registration with (seed, pair) uses key = (seed, pair)*/
/* and counter = (h, 0, 0, 0); word k becomes the index floor(x_k * N/2^64).*/
/* ------------------------------------------------------------------------ */
static inline void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, &hi0, &lo0);
    mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

static inline void sample4(uint64_t seed, uint64_t pair, int64_t h, int64_t n, int64_t idx[4]) {
  uint64_t ctr[4] = {(uint64_t)h, 0, 0, 0}, key[2] = {seed, pair}, out[4];
  orc_philox4x64_10(ctr, key, out);
  for (int k = 0; k < 4; ++k) {
    uint64_t hi, lo;
    mulhilo64(out[k], (uint64_t)n, &hi, &lo);
    idx[k] = (int64_t)hi;
  }
}

void orc_sample_indices(uint64_t seed, uint64_t pair, int64_t h0, int64_t nh, int64_t n, int64_t *out) {
  for (int64_t h = 0; h < nh; ++h) sample4(seed, pair, h0 + h, n, out + 4 * h);
}

/* ------------------------------------------------------------------------ */
/* Hypothesis sampling and polygon pre-rejection (Alg. 1, "Randomly sample  */
/* hypotheses" and "Hypotheses pre-rejection", tau of Sec. IV).             */
/* Readings: the edges (k, k+1) are cyclic over the four points; lengths   */
/* are compared squared against tau^2; a hypothesis with a repeated index, */
/* a point without a valid normal, or an edge shorter than 1e-6 is rejected*/
/* (never resampled).                                                       */
/* flag per hypothesis: 0 rejected, 1 survives, 2 ambiguous (some deciding  */
/* comparison within 1e-5 relative, so FP32 may decide it either way).      */
/* ------------------------------------------------------------------------ */
typedef struct {
  const double *P, *Q;
  int64_t nP, nQ;
  const int64_t *nn;
  const uint8_t *vP, *vQ;
  uint64_t seed, pair;
  double tau2;
  uint8_t *flag;
} hyp_ctx;

static void hyp_body(void *vctx, int64_t lo, int64_t hi) {
  hyp_ctx *c = (hyp_ctx *)vctx;
  const double rel = 1e-5, min_e2 = 1e-12;
  for (int64_t h = lo; h < hi; ++h) {
    int64_t idx[4];
    sample4(c->seed, c->pair, h, c->nP, idx);
    uint8_t fate = 1;
    for (int a = 0; a < 4 && fate; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (idx[a] == idx[b]) fate = 0;
    int64_t j[4];
    for (int a = 0; a < 4 && fate; ++a) {
      if (!c->vP[idx[a]]) fate = 0;
      j[a] = c->nn[idx[a]];
      if (fate && (j[a] < 0 || j[a] >= c->nQ || !c->vQ[j[a]])) fate = 0;
    }
    if (!fate) {
      c->flag[h] = 0;
      continue;
    }
    int sure_reject = 0, amb = 0;
    for (int a = 0; a < 4; ++a) {
      int b = (a + 1) & 3;
      double ep = dist2(c->P + 3 * idx[a], c->P + 3 * idx[b]);
      double eq = dist2(c->Q + 3 * j[a], c->Q + 3 * j[b]);
      /* degenerate edge */
      if (ep < min_e2 || eq < min_e2) {
        if (ep < min_e2 * (1 - rel) || eq < min_e2 * (1 - rel))
          sure_reject = 1;
        else
          amb = 1;
      } else if (ep < min_e2 * (1 + rel) || eq < min_e2 * (1 + rel)) {
        amb = 1;
      }
      /* ||p_k - p_k+1|| < tau ||q_k - q_k+1|| or the reverse */
      double l1 = ep, r1 = c->tau2 * eq, l2 = eq, r2 = c->tau2 * ep;
      if (l1 < r1) {
        if (r1 - l1 > rel * (l1 + r1))
          sure_reject = 1;
        else
          amb = 1;
      } else if (l1 - r1 <= rel * (l1 + r1)) {
        amb = 1;
      }
      if (l2 < r2) {
        if (r2 - l2 > rel * (l2 + r2))
          sure_reject = 1;
        else
          amb = 1;
      } else if (l2 - r2 <= rel * (l2 + r2)) {
        amb = 1;
      }
    }
    c->flag[h] = sure_reject ? 0 : (amb ? 2 : 1);
  }
}

/* Writes the flag of every hypothesis 0..H-1 (H bytes). */
void orc_hypotheses(const double *P, int64_t nP, const double *Q, int64_t nQ, const int64_t *nn, const uint8_t *validP,
                    const uint8_t *validQ, int64_t H, uint64_t seed, uint64_t pair, double tau, uint8_t *flag) {
  hyp_ctx c = {P, Q, nP, nQ, nn, validP, validQ, seed, pair, tau * tau, flag};
  orc_parallel_for(H, 8192, hyp_body, &c);
}

/* ------------------------------------------------------------------------ */
/* Least-squares rigid transform from point pairs (Alg. 1, "Estimate        */
/* transformation T_QP from S_P[i] to S_Q[i]"): minimise sum |R p + t - q|^2*/
/* through the SVD H = U S V^T of the cross-covariance H = sum (p-pm)(q-qm)^T*/
/* with R = V diag(1, 1, det(V U^T)) U^T and t = qm - R pm. The SVD is the  */
/* one-sided (Hestenes) Jacobi method: rotate column pairs of H until they */
/* are orthogonal; the rotations accumulate into V and the normalised       */
/* columns are U. Rank-deficient cases complete U by cross products.       */
/* ------------------------------------------------------------------------ */
static void svd3_hestenes(const double H[9], double U[9], double sig[3], double V[9]) {
  double A[9];
  memcpy(A, H, sizeof(A));
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    for (int i = 0; i < 2; ++i)
      for (int j = i + 1; j < 3; ++j) {
        double a = 0, b = 0, g = 0;
        for (int k = 0; k < 3; ++k) {
          a += A[3 * k + i] * A[3 * k + i];
          b += A[3 * k + j] * A[3 * k + j];
          g += A[3 * k + i] * A[3 * k + j];
        }
        if (g == 0.0 || fabs(g) <= 1e-17 * sqrt(a * b)) continue;
        rotated = 1;
        double zeta = (b - a) / (2.0 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int k = 0; k < 3; ++k) {
          double x = A[3 * k + i], y = A[3 * k + j];
          A[3 * k + i] = c * x - s * y;
          A[3 * k + j] = s * x + c * y;
          double vx = V[3 * k + i], vy = V[3 * k + j];
          V[3 * k + i] = c * vx - s * vy;
          V[3 * k + j] = s * vx + c * vy;
        }
      }
    if (!rotated) break;
  }
  double nrm[3];
  for (int c = 0; c < 3; ++c) nrm[c] = sqrt(A[c] * A[c] + A[3 + c] * A[3 + c] + A[6 + c] * A[6 + c]);
  int ord[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (nrm[ord[j]] > nrm[ord[i]]) {
        int tmp = ord[i];
        ord[i] = ord[j];
        ord[j] = tmp;
      }
  double Vs[9];
  for (int c = 0; c < 3; ++c) {
    sig[c] = nrm[ord[c]];
    for (int r = 0; r < 3; ++r) {
      Vs[3 * r + c] = V[3 * r + ord[c]];
      U[3 * r + c] = A[3 * r + ord[c]];
    }
  }
  memcpy(V, Vs, sizeof(Vs));
  /* normalise U's columns; complete rank-deficient ones */
  for (int c = 0; c < 3; ++c) {
    int ok = sig[0] > 0 && sig[c] > 1e-13 * sig[0];
    if (ok) {
      for (int r = 0; r < 3; ++r) U[3 * r + c] /= sig[c];
    } else if (c == 2) {
      double u0[3] = {U[0], U[3], U[6]}, u1[3] = {U[1], U[4], U[7]}, u2[3];
      cross3(u0, u1, u2);
      for (int r = 0; r < 3; ++r) U[3 * r + 2] = u2[r];
    } else if (c == 1) {
      double u0[3] = {U[0], U[3], U[6]}, a[3] = {1, 0, 0}, u1[3];
      if (fabs(u0[0]) > 0.9) {
        a[0] = 0;
        a[1] = 1;
      }
      cross3(u0, a, u1);
      double n1 = sqrt(dot3(u1, u1));
      for (int r = 0; r < 3; ++r) U[3 * r + 1] = u1[r] / n1;
    }
  }
}

void orc_svd3(const double H[9], double U[9], double sig[3], double V[9]) { svd3_hestenes(H, U, sig, V); }

void orc_kabsch(const double *p, const double *q, int64_t m, double R[9], double t[3]) {
  double pm[3] = {0, 0, 0}, qm[3] = {0, 0, 0};
  for (int64_t i = 0; i < m; ++i)
    for (int d = 0; d < 3; ++d) {
      pm[d] += p[3 * i + d];
      qm[d] += q[3 * i + d];
    }
  for (int d = 0; d < 3; ++d) {
    pm[d] /= (double)m;
    qm[d] /= (double)m;
  }
  double H[9] = {0};
  for (int64_t i = 0; i < m; ++i) {
    double a[3], b[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = p[3 * i + d] - pm[d];
      b[d] = q[3 * i + d] - qm[d];
    }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) H[3 * r + c] += a[r] * b[c];
  }
  double U[9], sig[3], V[9];
  svd3_hestenes(H, U, sig, V);
  if (!(sig[0] > 0)) {
    /* all points coincide: no rotation is determined, take the identity */
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int d = 0; d < 3; ++d) t[d] = qm[d] - pm[d];
    return;
  }
  /* R = V diag(1,1,d) U^T, d = det(V U^T) */
  double VUt[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) VUt[3 * r + c] = V[3 * r + 0] * U[3 * c + 0] + V[3 * r + 1] * U[3 * c + 1] + V[3 * r + 2] * U[3 * c + 2];
  double det = VUt[0] * (VUt[4] * VUt[8] - VUt[5] * VUt[7]) - VUt[1] * (VUt[3] * VUt[8] - VUt[5] * VUt[6]) +
               VUt[2] * (VUt[3] * VUt[7] - VUt[4] * VUt[6]);
  double dsign = det < 0 ? -1.0 : 1.0;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = V[3 * r + 0] * U[3 * c + 0] + V[3 * r + 1] * U[3 * c + 1] + dsign * V[3 * r + 2] * U[3 * c + 2];
  double Rp[3];
  Rp[0] = R[0] * pm[0] + R[1] * pm[1] + R[2] * pm[2];
  Rp[1] = R[3] * pm[0] + R[4] * pm[1] + R[5] * pm[2];
  Rp[2] = R[6] * pm[0] + R[7] * pm[1] + R[8] * pm[2];
  for (int d = 0; d < 3; ++d) t[d] = qm[d] - Rp[d];
}

/* ------------------------------------------------------------------------ */
/* Nearest neighbour within a radius (the grid search of eq. (1) and its   */
/* surrounding text, read as an exact search over all cells that overlap  */
/* the ball): smallest squared distance < r^2, ties to the smallest index. */
/* ------------------------------------------------------------------------ */
typedef struct {
  double best;
  int64_t arg;
  double r2;
} nn_state;

static void visit_nn(void *ctx, int64_t j, double d2) {
  nn_state *s = (nn_state *)ctx;
  if (d2 < s->r2 && (d2 < s->best || (d2 == s->best && j < s->arg))) {
    s->best = d2;
    s->arg = j;
  }
}

static inline int64_t nn_within(const orc_grid *g, const double *Q, const double *x, double r, double *d2) {
  nn_state s = {INFINITY, -1, r * r};
  grid_visit(g, Q, x, visit_nn, &s);
  *d2 = s.best;
  return s.arg;
}

/* Public for tests: exact NN within r by the grid and by brute force. */
void orc_nn_within_grid(const double *Q, int64_t nQ, const double *X, int64_t m, double r, int64_t *nn, double *d2) {
  orc_grid g;
  grid_build(&g, Q, nQ, r);
  for (int64_t i = 0; i < m; ++i) nn[i] = nn_within(&g, Q, X + 3 * i, r, d2 + i);
  grid_free(&g);
}

void orc_nn_within_brute(const double *Q, int64_t nQ, const double *X, int64_t m, double r, int64_t *nn, double *d2) {
  for (int64_t i = 0; i < m; ++i) {
    double best = INFINITY;
    int64_t arg = -1;
    for (int64_t j = 0; j < nQ; ++j) {
      double d = dist2(Q + 3 * j, X + 3 * i);
      if (d < r * r && d < best) {
        best = d;
        arg = j;
      }
    }
    nn[i] = arg;
    d2[i] = best;
  }
}

/* ------------------------------------------------------------------------ */
/* Hypothesis testing (Alg. 1, "Consensus for the remaining quadruple      */
/* pairs"): for a pose (R, t), every p in P with min_q |R p + t - q| < eps  */
/* is an inlier. count = number of inliers, sumd2 = sum of their squared   */
/* NN distances (fitness = sumd2 / count, the mean squared inlier distance */
/* of the PCL-derived pipeline the paper starts from). namb counts points  */
/* whose NN distance lies within band of eps (FP32 may decide them either  */
/* way).                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
  const double *P, *Q, *Rs, *ts;
  int64_t nP;
  double eps, band;
  int64_t *count, *namb;
  double *sumd2;
  const orc_grid *g;
} cons_ctx;

static void cons_body(void *vctx, int64_t lo, int64_t hi) {
  cons_ctx *c = (cons_ctx *)vctx;
  for (int64_t h = lo; h < hi; ++h) {
    const double *R = c->Rs + 9 * h, *t = c->ts + 3 * h;
    int64_t cnt = 0, amb = 0;
    double sum = 0.0;
    double eps_hi = c->eps + c->band, eps_lo = c->eps - c->band;
    for (int64_t i = 0; i < c->nP; ++i) {
      double x[3], d2;
      xform(R, t, c->P + 3 * i, x);
      /* search slightly beyond eps so the margin can be seen */
      int64_t j = nn_within(c->g, c->Q, x, eps_hi, &d2);
      if (j < 0) continue;
      if (d2 > eps_lo * eps_lo) ++amb;
      if (d2 < c->eps * c->eps) {
        ++cnt;
        sum += d2;
      }
    }
    c->count[h] = cnt;
    c->sumd2[h] = sum;
    c->namb[h] = amb;
  }
}

void orc_consensus(const double *P, int64_t nP, const double *Q, int64_t nQ, const double *Rs, const double *ts, int64_t nh,
                   double eps, double band, int64_t *count, double *sumd2, int64_t *namb) {
  orc_grid g;
  grid_build(&g, Q, nQ, eps + band);
  cons_ctx c = {P, Q, Rs, ts, nP, eps, band, count, namb, sumd2, &g};
  orc_parallel_for(nh, 1, cons_body, &c);
  grid_free(&g);
}

/* ------------------------------------------------------------------------ */
/* SO(3) exponential (Rodrigues) and the left-multiplied pose update used  */
/* for the 6-vector xi = (alpha, beta, gamma, x, y, z) of eq. (5):         */
/* T(xi) = [Exp(alpha, beta, gamma) | (x, y, z)] * T0, so that to first    */
/* order x' = x - [x]_x w + v, i.e. the Jacobian G_p = [-[p]_x | I].       */
/* ------------------------------------------------------------------------ */
void orc_exp_so3(const double w[3], double R[9]) {
  double th2 = dot3(w, w), th = sqrt(th2);
  double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double K2[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) K2[3 * r + c] = K[3 * r + 0] * K[0 + c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
  double a, b;
  if (th < 1e-6) {
    a = 1.0 - th2 / 6.0;
    b = 0.5 - th2 / 24.0;
  } else {
    a = sin(th) / th;
    b = (1.0 - cos(th)) / th2;
  }
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + a * K[i] + b * K2[i];
}

/* T_out = [Exp(xi[0:3]) | xi[3:6]] * T_in (4x4 row-major) */
void orc_apply_xi(const double xi[6], const double T_in[16], double T_out[16]) {
  double R[9];
  orc_exp_so3(xi, R);
  double M[16] = {R[0], R[1], R[2], xi[3], R[3], R[4], R[5], xi[4], R[6], R[7], R[8], xi[5], 0, 0, 0, 1};
  double out[16];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += M[4 * r + k] * T_in[4 * k + c];
      out[4 * r + c] = s;
    }
  memcpy(T_out, out, sizeof(out));
}

/* Left Jacobian of SO(3): Exp(w + d) = Exp(J_l(w) d) Exp(w) to first order. */
static void left_jacobian_so3(const double w[3], double J[9]) {
  double th2 = dot3(w, w), th = sqrt(th2);
  double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double K2[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) K2[3 * r + c] = K[3 * r + 0] * K[0 + c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
  double a, b;
  if (th < 1e-5) {
    a = 0.5 - th2 / 24.0;
    b = 1.0 / 6.0 - th2 / 120.0;
  } else {
    a = (1.0 - cos(th)) / th2;
    b = (th - sin(th)) / (th2 * th);
  }
  for (int i = 0; i < 9; ++i) J[i] = (i % 4 == 0 ? 1.0 : 0.0) + a * K[i] + b * K2[i];
}

/* 6x6 SPD solve A x = b by Cholesky; returns 0 if A is not positive definite */
static int chol6_solve(const double A_in[36], const double b[6], double x[6]) {
  double L[36] = {0};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A_in[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      if (i == j) {
        if (!(s > 0.0)) return 0;
        L[6 * i + i] = sqrt(s);
      } else {
        L[6 * i + j] = s / L[6 * j + j];
      }
    }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
    y[i] = s / L[6 * i + i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
    x[i] = s / L[6 * i + i];
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Robust refinement (the line-process objective of eq. (3)-(4) with the   */
/* Jacobian G_p = [-[p]_x | I] of eq. (5)). Eliminating the line process l */
/* from l*r^2 + mu*(sqrt(l) - 1)^2 gives l* = (mu / (mu + r^2))^2 and the   */
/* Geman-McClure cost rho(r^2) = mu r^2 / (mu + r^2). Each iteration takes */
/* the exact NN within eps_r of every transformed point, weights w = l*,    */
/* builds A = sum w J^T J and b = sum w J^T r, solves A d = -b (Cholesky), */
/* and sets T <- [Exp(d_w) | d_v] T. Stops after iters or when |d| < tol.   */
/* The sums are taken per fixed chunk of 1024 points and added in order.   */
/* ------------------------------------------------------------------------ */
#define ORC_CHUNK 1024
typedef struct {
  const double *P, *Q;
  int64_t nP;
  double R[9], t[3], eps_r, mu;
  double *part; /* nchunks x 27 (21 upper-tri of A + 6 of b) */
  const orc_grid *g;
} refine_ctx;

static void refine_body(void *vctx, int64_t lo, int64_t hi) {
  refine_ctx *c = (refine_ctx *)vctx;
  for (int64_t ch = lo; ch < hi; ++ch) {
    double A[36] = {0}, b[6] = {0};
    int64_t i0 = ch * ORC_CHUNK, i1 = i0 + ORC_CHUNK < c->nP ? i0 + ORC_CHUNK : c->nP;
    for (int64_t i = i0; i < i1; ++i) {
      double x[3], d2;
      xform(c->R, c->t, c->P + 3 * i, x);
      int64_t j = nn_within(c->g, c->Q, x, c->eps_r, &d2);
      if (j < 0) continue;
      const double *q = c->Q + 3 * j;
      double r[3] = {x[0] - q[0], x[1] - q[1], x[2] - q[2]};
      double s = dot3(r, r);
      double l = c->mu / (c->mu + s);
      double w = l * l;
      /* J = [-[x]_x | I], 3 x 6 */
      double J[18] = {0, x[2], -x[1], 1, 0, 0, -x[2], 0, x[0], 0, 1, 0, x[1], -x[0], 0, 0, 0, 1};
      for (int a = 0; a < 6; ++a) {
        for (int bb = 0; bb < 6; ++bb) A[6 * a + bb] += w * (J[a] * J[bb] + J[6 + a] * J[6 + bb] + J[12 + a] * J[12 + bb]);
        b[a] += w * (J[a] * r[0] + J[6 + a] * r[1] + J[12 + a] * r[2]);
      }
    }
    double *o = c->part + 27 * ch;
    int k = 0;
    for (int a = 0; a < 6; ++a)
      for (int bb = a; bb < 6; ++bb) o[k++] = A[6 * a + bb];
    for (int a = 0; a < 6; ++a) o[21 + a] = b[a];
  }
}

int orc_refine(const double *P, int64_t nP, const double *Q, int64_t nQ, const double T_in[16], double eps_r, double mu,
               int iters, double tol, double T_out[16]) {
  orc_grid g;
  grid_build(&g, Q, nQ, eps_r);
  double T[16];
  memcpy(T, T_in, sizeof(T));
  int64_t nch = (nP + ORC_CHUNK - 1) / ORC_CHUNK;
  double *part = (double *)malloc(sizeof(double) * 27 * (size_t)(nch > 0 ? nch : 1));
  int it;
  for (it = 0; it < iters; ++it) {
    refine_ctx c;
    c.P = P;
    c.Q = Q;
    c.nP = nP;
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) c.R[3 * r + q] = T[4 * r + q];
      c.t[r] = T[4 * r + 3];
    }
    c.eps_r = eps_r;
    c.mu = mu;
    c.part = part;
    c.g = &g;
    orc_parallel_for(nch, 1, refine_body, &c);
    double A[36] = {0}, b[6] = {0};
    for (int64_t ch = 0; ch < nch; ++ch) {
      const double *o = part + 27 * ch;
      int k = 0;
      for (int a = 0; a < 6; ++a)
        for (int bb = a; bb < 6; ++bb) {
          A[6 * a + bb] += o[k];
          if (bb != a) A[6 * bb + a] += o[k];
          ++k;
        }
      for (int a = 0; a < 6; ++a) b[a] += o[21 + a];
    }
    double nb[6], d[6];
    for (int a = 0; a < 6; ++a) nb[a] = -b[a];
    if (!chol6_solve(A, nb, d)) break;
    orc_apply_xi(d, T, T);
    double nd = 0;
    for (int a = 0; a < 6; ++a) nd += d[a] * d[a];
    if (sqrt(nd) < tol) {
      ++it;
      break;
    }
  }
  memcpy(T_out, T, sizeof(T));
  free(part);
  grid_free(&g);
  return it;
}

/* ------------------------------------------------------------------------ */
/* Graduated refinement (reading: the paper gives no refinement schedule;    */
/* this follows the graduated non-convexity of Fast Global Registration,    */
/* Zhou et al. 2016, which the paper compares against). Level l = 0..L-1     */
/* runs the refinement above with radius eps_l = eps * 2^(L-1-l) and          */
/* mu_l = mu_scale * eps_l^2 on the subsets P_l = {p_i : i mod sP_l = 0} and */
/* Q_l = {q_j : j mod sQ_l = 0}, s_l = max(1, min(4^(L-1-l), N / 4096)), so  */
/* the coarse levels see a smooth cost and the result does not depend on    */
/* which nearby hypothesis started it.                                        */
/* ------------------------------------------------------------------------ */
int64_t orc_gnc_stride(int64_t n, int level, int levels) {
  int64_t f = 1;
  for (int k = 0; k < levels - 1 - level; ++k) f *= 4;
  int64_t cap = n / 4096;
  if (f > cap) f = cap;
  return f < 1 ? 1 : f;
}

int orc_refine_gnc(const double *P, int64_t nP, const double *Q, int64_t nQ, const double T_in[16], double eps,
                   double mu_scale, int levels, int iters, double tol, double T_out[16]) {
  double T[16];
  memcpy(T, T_in, sizeof(T));
  int total = 0;
  for (int l = 0; l < levels; ++l) {
    double e = eps * (double)(1LL << (levels - 1 - l));
    int64_t sp = orc_gnc_stride(nP, l, levels), sq = orc_gnc_stride(nQ, l, levels);
    int64_t mp = (nP + sp - 1) / sp, mq = (nQ + sq - 1) / sq;
    double *Ps = (double *)malloc(sizeof(double) * 3 * (size_t)mp), *Qs = (double *)malloc(sizeof(double) * 3 * (size_t)mq);
    for (int64_t i = 0; i < mp; ++i) memcpy(Ps + 3 * i, P + 3 * i * sp, sizeof(double) * 3);
    for (int64_t j = 0; j < mq; ++j) memcpy(Qs + 3 * j, Q + 3 * j * sq, sizeof(double) * 3);
    total += orc_refine(Ps, mp, Qs, mq, T, e, mu_scale * e * e, iters, tol, T);
    free(Ps);
    free(Qs);
  }
  memcpy(T_out, T, sizeof(T));
  return total;
}

/* ------------------------------------------------------------------------ */
/* Information matrix of a verified pair (loop verification, eq. (5)-(6)):  */
/* the quadratic form that approximates the alignment error of the pair is  */
/* xi^T (sum over (p, q) in K of G_p^T G_p) xi with G_p = [-[p]_x | I] and K */
/* the nearest-neighbour pairs between the moved cloud T P and Q closer     */
/* than eps (the paper uses eps = 0.05 m). Reading: both clouds are in Q's  */
/* frame, so p in G_p is the moved point T p. info is row-major 6 x 6, n the */
/* size of K. namb counts the points of P whose NN distance lies within     */
/* band of eps (FP32 may decide those either way) and amb_max is the largest */
/* |T p|^2 among them.                                                      */
/* ------------------------------------------------------------------------ */
void orc_information(const double *P, int64_t nP, const double *Q, int64_t nQ, const double T[16], double eps,
                     double band, double info[36], int64_t *n, int64_t *namb, double *amb_max) {
  const double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]}, t[3] = {T[3], T[7], T[11]};
  orc_grid g;
  grid_build(&g, Q, nQ, eps + band);
  for (int k = 0; k < 36; ++k) info[k] = 0.0;
  *n = 0;
  *namb = 0;
  *amb_max = 0.0;
  for (int64_t i = 0; i < nP; ++i) {
    double x[3], d2;
    xform(R, t, P + 3 * i, x);
    if (nn_within(&g, Q, x, eps + band, &d2) < 0) continue;
    if (fabs(sqrt(d2) - eps) <= band) {
      ++*namb;
      if (dot3(x, x) > *amb_max) *amb_max = dot3(x, x);
    }
    if (!(d2 < eps * eps)) continue;
    /* G = [-[x]_x | I], three rows of six */
    const double G[3][6] = {{0.0, x[2], -x[1], 1.0, 0.0, 0.0},
                            {-x[2], 0.0, x[0], 0.0, 1.0, 0.0},
                            {x[1], -x[0], 0.0, 0.0, 0.0, 1.0}};
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) info[6 * a + b] += G[0][a] * G[0][b] + G[1][a] * G[1][b] + G[2][a] * G[2][b];
    ++*n;
  }
  grid_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Robust alignment objective and its analytic gradient (the objective of   */
/* the refinement above, with NN correspondences recomputed at the given   */
/* pose): E = sum_i rho~(s_i), s_i = |T(xi) p_i - q_n(i)|^2 over the points */
/* whose NN lies within eps, rho~(s) = rho(s) - rho(eps^2) so that E is     */
/* continuous as a pair leaves the eps-ball, rho'(s) = mu^2 / (mu + s)^2.    */
/* dE/dp_i = 2 rho' R^T r_i; dE/dq_j = -sum_{n(i)=j} 2 rho' r_i;            */
/* dE/dv = sum 2 rho' r_i; dE/dw = J_l(w)^T sum 2 rho' (z_i x r_i),         */
/* z_i = Exp(w) T0 p_i. dP, dQ or dxi may be NULL.                          */
/* ------------------------------------------------------------------------ */
double orc_objective(const double *P, int64_t nP, const double *Q, int64_t nQ, const double xi[6], const double T0[16],
                     double eps, double mu, double *dP, double *dQ, double dxi[6], int64_t *nn_out) {
  orc_grid g;
  grid_build(&g, Q, nQ, eps);
  double T[16];
  orc_apply_xi(xi, T0, T);
  double R[9], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) R[3 * r + q] = T[4 * r + q];
    t[r] = T[4 * r + 3];
  }
  double rho_eps = mu * eps * eps / (mu + eps * eps);
  if (dQ) memset(dQ, 0, sizeof(double) * 3 * (size_t)nQ);
  double gw[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
  double E = 0.0;
  for (int64_t i = 0; i < nP; ++i) {
    double x[3], d2;
    xform(R, t, P + 3 * i, x);
    int64_t j = nn_within(&g, Q, x, eps, &d2);
    if (nn_out) nn_out[i] = j;
    if (dP) dP[3 * i] = dP[3 * i + 1] = dP[3 * i + 2] = 0.0;
    if (j < 0) continue;
    double r[3] = {x[0] - Q[3 * j], x[1] - Q[3 * j + 1], x[2] - Q[3 * j + 2]};
    double s = dot3(r, r);
    E += mu * s / (mu + s) - rho_eps;
    double dr = mu * mu / ((mu + s) * (mu + s));
    double gr[3] = {2 * dr * r[0], 2 * dr * r[1], 2 * dr * r[2]};
    if (dP)
      for (int a = 0; a < 3; ++a) dP[3 * i + a] = R[0 * 3 + a] * gr[0] + R[1 * 3 + a] * gr[1] + R[2 * 3 + a] * gr[2];
    if (dQ)
      for (int a = 0; a < 3; ++a) dQ[3 * j + a] -= gr[a];
    double z[3] = {x[0] - xi[3], x[1] - xi[4], x[2] - xi[5]}, zr[3];
    cross3(z, gr, zr);
    for (int a = 0; a < 3; ++a) {
      gw[a] += zr[a];
      gv[a] += gr[a];
    }
  }
  if (dxi) {
    double J[9];
    left_jacobian_so3(xi, J);
    for (int a = 0; a < 3; ++a) dxi[a] = J[0 * 3 + a] * gw[0] + J[1 * 3 + a] * gw[1] + J[2 * 3 + a] * gw[2];
    for (int a = 0; a < 3; ++a) dxi[3 + a] = gv[a];
  }
  grid_free(&g);
  return E;
}

/* ------------------------------------------------------------------------ */
/* The whole of Algorithm 1 for one pair, in the paper's order, followed by*/
/* the robust refinement. Parameters (Sec. IV, scaled as stated in the     */
/* design notes): normal radius, feature radius, eps (maximum correspondence*/
/* distance), tau, the normal check threshold (cos), the minimum inlier    */
/* ratio, mu = mu_scale * eps^2, hypotheses, refinement iterations, seed.  */
/* ------------------------------------------------------------------------ */
typedef struct {
  double r_normal, r_feature, eps_inlier, tau, cos_normal, min_inlier_ratio, mu_scale;
  int64_t n_hypotheses;
  int32_t refine_iters;  /* per level */
  int32_t refine_levels;
  uint64_t seed;
  uint64_t pair_id;
} orc_params;

typedef struct {
  double T[16];
  double T_hyp[16];
  int64_t inliers, survivors, best_h, hyp_inliers, n_normal_ok;
  double fitness, hyp_fitness;
  int32_t status; /* 0 aligned, 1 no alignment */
  int32_t refine_iters_done;
} orc_result;

/* What an FP32 implementation of the same steps may legitimately decide the */
/* other way, reported beside a registration (reporting only: nothing here  */
/* changes the result). Bands: 1e-5 on the descriptor NN gap (d2 - d1),    */
/* the relative band of the pre-rejection comparisons, and 1e-5 m about eps */
/* for the inlier test.                                                    */
#define ORC_DIAG_TOP 16
typedef struct {
  int64_t nn_amb;     /* points of P whose second-nearest descriptor is within 1e-5 of the nearest */
  int64_t hyp_amb;    /* hypotheses whose pre-rejection is decided within its band */
  int64_t surv_touch; /* survivors with at least one sampled point counted in nn_amb */
  int64_t n_top;      /* entries of top[] filled */
  int64_t top_h[ORC_DIAG_TOP];     /* the best normal-checked hypotheses, in selection order */
  int64_t top_count[ORC_DIAG_TOP]; /* their inlier counts */
  int64_t top_amb[ORC_DIAG_TOP];   /* their points whose NN distance lies within 1e-5 of eps */
  int64_t top_touch[ORC_DIAG_TOP]; /* 1 if one of their sampled points is counted in nn_amb */
  double top_fitness[ORC_DIAG_TOP];
  int64_t final_amb;  /* the same band count at the refined pose */
} orc_diag;

/* Selection (Alg. 1, "Find the hypothesis that has max inlier ratio and     */
/* fitness score passing minimum threshold"): reading: the largest inlier   */
/* count wins, then the smaller fitness, then the smaller hypothesis id; it */
/* is accepted if count / |P| >= min_inlier_ratio.                          */
static int better(int64_t c, double f, int64_t h, int64_t bc, double bf, int64_t bh) {
  if (c != bc) return c > bc;
  if (f != bf) return f < bf;
  return h < bh;
}

int orc_register(const double *P, int64_t nP, const double *Q, int64_t nQ, const double vpP[3], const double vpQ[3],
                 const orc_params *prm, orc_result *res, double *dbg_fP, double *dbg_fQ, int64_t *dbg_nn,
                 orc_diag *diag) {
  memset(res, 0, sizeof(*res));
  if (diag) memset(diag, 0, sizeof(*diag));
  for (int i = 0; i < 16; ++i) res->T[i] = res->T_hyp[i] = (i % 5 == 0) ? 1.0 : 0.0;
  res->status = 1;
  res->best_h = -1;
  if (nP < 4 || nQ < 4) return -1;
  /* Alg. 1, FPFH step: normals and FPFH of both clouds */
  double *NP = malloc(sizeof(double) * 3 * nP), *NQ = malloc(sizeof(double) * 3 * nQ);
  double *cv = malloc(sizeof(double) * (nP > nQ ? nP : nQ)), *dg = malloc(sizeof(double) * 3 * (nP > nQ ? nP : nQ));
  int64_t *ct = malloc(sizeof(int64_t) * (nP > nQ ? nP : nQ));
  orc_normals(P, nP, vpP, prm->r_normal, NULL, 0, NP, cv, ct, dg);
  orc_normals(Q, nQ, vpQ, prm->r_normal, NULL, 0, NQ, cv, ct, dg);
  double *SP = malloc(sizeof(double) * ORC_D * nP), *SQ = malloc(sizeof(double) * ORC_D * nQ);
  double *FP = dbg_fP ? dbg_fP : malloc(sizeof(double) * ORC_D * nP);
  double *FQ = dbg_fQ ? dbg_fQ : malloc(sizeof(double) * ORC_D * nQ);
  int64_t *kk = malloc(sizeof(int64_t) * (nP > nQ ? nP : nQ)), *nc = malloc(sizeof(int64_t) * (nP > nQ ? nP : nQ));
  orc_spfh(P, NP, nP, prm->r_feature, NULL, 0, 1e-4, SP, kk, nc);
  orc_spfh(Q, NQ, nQ, prm->r_feature, NULL, 0, 1e-4, SQ, kk, nc);
  orc_fpfh(P, NP, SP, nP, prm->r_feature, NULL, 0, FP);
  orc_fpfh(Q, NQ, SQ, nQ, prm->r_feature, NULL, 0, FQ);
  /* pre-matching cache */
  int64_t *nn = dbg_nn ? dbg_nn : malloc(sizeof(int64_t) * nP);
  double *d1 = malloc(sizeof(double) * nP), *d2 = malloc(sizeof(double) * nP);
  orc_match(FP, nP, FQ, nQ, ORC_D, NULL, 0, nn, d1, d2);
  /* validity: a valid normal (and hence a non-zero descriptor) */
  uint8_t *vP = malloc(nP), *vQ = malloc(nQ);
  for (int64_t i = 0; i < nP; ++i) vP[i] = !is_zero3(NP + 3 * i);
  for (int64_t i = 0; i < nQ; ++i) vQ[i] = !is_zero3(NQ + 3 * i);
  /* hypotheses + pre-rejection + compaction (ascending id) */
  int64_t H = prm->n_hypotheses;
  uint8_t *flag = malloc((size_t)(H > 0 ? H : 1));
  orc_hypotheses(P, nP, Q, nQ, nn, vP, vQ, H, prm->seed, prm->pair_id, prm->tau, flag);
  int64_t S = 0;
  for (int64_t h = 0; h < H; ++h) S += flag[h] != 0;
  if (diag) {
    for (int64_t i = 0; i < nP; ++i) diag->nn_amb += (d2[i] - d1[i]) <= 1e-5;
    for (int64_t h = 0; h < H; ++h) diag->hyp_amb += flag[h] == 2;
  }
  int64_t *surv = malloc(sizeof(int64_t) * (S > 0 ? S : 1));
  S = 0;
  for (int64_t h = 0; h < H; ++h)
    if (flag[h]) surv[S++] = h;
  res->survivors = S;
  /* per survivor: transform from the 4 pairs, normal check */
  double *Rs = malloc(sizeof(double) * 9 * (S > 0 ? S : 1)), *ts = malloc(sizeof(double) * 3 * (S > 0 ? S : 1));
  uint8_t *nok = malloc((size_t)(S > 0 ? S : 1));
  int64_t nvalid = 0;
  for (int64_t s = 0; s < S; ++s) {
    int64_t idx[4];
    sample4(prm->seed, prm->pair_id, surv[s], nP, idx);
    double ps[12], qs[12];
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) {
        ps[3 * a + d] = P[3 * idx[a] + d];
        qs[3 * a + d] = Q[3 * nn[idx[a]] + d];
      }
    orc_kabsch(ps, qs, 4, Rs + 9 * s, ts + 3 * s);
    if (diag) {
      int touch = 0;
      for (int a = 0; a < 4; ++a) touch |= (d2[idx[a]] - d1[idx[a]]) <= 1e-5;
      diag->surv_touch += touch;
    }
    /* Reading: the normal check compares R n_p with n_q for the 4 samples */
    uint8_t ok = 1;
    for (int a = 0; a < 4; ++a) {
      const double *np = NP + 3 * idx[a], *nq = NQ + 3 * nn[idx[a]];
      const double *R = Rs + 9 * s;
      double rn[3] = {R[0] * np[0] + R[1] * np[1] + R[2] * np[2], R[3] * np[0] + R[4] * np[1] + R[5] * np[2],
                      R[6] * np[0] + R[7] * np[1] + R[8] * np[2]};
      if (dot3(rn, nq) < prm->cos_normal) ok = 0;
    }
    nok[s] = ok;
    nvalid += ok;
  }
  res->n_normal_ok = nvalid;
  /* consensus for the hypotheses that pass the normal check */
  double *Rv = malloc(sizeof(double) * 9 * (nvalid > 0 ? nvalid : 1)), *tv = malloc(sizeof(double) * 3 * (nvalid > 0 ? nvalid : 1));
  int64_t *hv = malloc(sizeof(int64_t) * (nvalid > 0 ? nvalid : 1));
  int64_t m = 0;
  for (int64_t s = 0; s < S; ++s)
    if (nok[s]) {
      memcpy(Rv + 9 * m, Rs + 9 * s, sizeof(double) * 9);
      memcpy(tv + 3 * m, ts + 3 * s, sizeof(double) * 3);
      hv[m++] = surv[s];
    }
  int64_t *cnt = malloc(sizeof(int64_t) * (m > 0 ? m : 1)), *amb = malloc(sizeof(int64_t) * (m > 0 ? m : 1));
  double *sd = malloc(sizeof(double) * (m > 0 ? m : 1));
  double eps = prm->eps_inlier;
  /* the band only widens the search to see points just past eps: the counts are exact either way */
  const double band = diag ? 1e-5 : 0.0;
  orc_consensus(P, nP, Q, nQ, Rv, tv, m, eps, band, cnt, sd, amb);
  if (diag) {
    /* the ORC_DIAG_TOP best hypotheses in selection order (repeated selection of the best not yet taken) */
    uint8_t *taken = calloc((size_t)(m > 0 ? m : 1), 1);
    for (int k = 0; k < ORC_DIAG_TOP; ++k) {
      int64_t b = -1;
      for (int64_t s = 0; s < m; ++s) {
        if (taken[s]) continue;
        double f = cnt[s] > 0 ? sd[s] / (double)cnt[s] : INFINITY;
        double fb = b >= 0 && cnt[b] > 0 ? sd[b] / (double)cnt[b] : INFINITY;
        if (b < 0 || better(cnt[s], f, hv[s], cnt[b], fb, hv[b])) b = s;
      }
      if (b < 0) break;
      taken[b] = 1;
      diag->top_h[k] = hv[b];
      diag->top_count[k] = cnt[b];
      diag->top_amb[k] = amb[b];
      diag->top_fitness[k] = cnt[b] > 0 ? sd[b] / (double)cnt[b] : 0.0;
      int64_t idx[4];
      sample4(prm->seed, prm->pair_id, hv[b], nP, idx);
      for (int a = 0; a < 4; ++a) diag->top_touch[k] |= (d2[idx[a]] - d1[idx[a]]) <= 1e-5;
      diag->n_top = k + 1;
    }
    free(taken);
  }
  int64_t best = -1, bc = -1;
  double bf = INFINITY;
  int64_t bh = INT64_MAX;
  for (int64_t s = 0; s < m; ++s) {
    double f = cnt[s] > 0 ? sd[s] / (double)cnt[s] : INFINITY;
    if (best < 0 || better(cnt[s], f, hv[s], bc, bf, bh)) {
      best = s;
      bc = cnt[s];
      bf = f;
      bh = hv[s];
    }
  }
  if (best >= 0 && (double)bc >= prm->min_inlier_ratio * (double)nP) {
    double T0[16] = {Rv[9 * best + 0], Rv[9 * best + 1], Rv[9 * best + 2], tv[3 * best + 0], Rv[9 * best + 3], Rv[9 * best + 4],
                     Rv[9 * best + 5], tv[3 * best + 1], Rv[9 * best + 6], Rv[9 * best + 7], Rv[9 * best + 8], tv[3 * best + 2],
                     0, 0, 0, 1};
    memcpy(res->T_hyp, T0, sizeof(T0));
    res->best_h = bh;
    res->hyp_inliers = bc;
    res->hyp_fitness = bf;
    res->refine_iters_done =
        orc_refine_gnc(P, nP, Q, nQ, T0, eps, prm->mu_scale, prm->refine_levels, prm->refine_iters, 1e-10, res->T);
    double R[9], t[3];
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) R[3 * r + q] = res->T[4 * r + q];
      t[r] = res->T[4 * r + 3];
    }
    int64_t c1, a1;
    double s1;
    orc_consensus(P, nP, Q, nQ, R, t, 1, eps, band, &c1, &s1, &a1);
    if (diag) diag->final_amb = a1;
    res->inliers = c1;
    res->fitness = c1 > 0 ? s1 / (double)c1 : 0.0;
    res->status = 0;
  }
  free(NP);
  free(NQ);
  free(cv);
  free(dg);
  free(ct);
  free(SP);
  free(SQ);
  if (!dbg_fP) free(FP);
  if (!dbg_fQ) free(FQ);
  free(kk);
  free(nc);
  if (!dbg_nn) free(nn);
  free(d1);
  free(d2);
  free(vP);
  free(vQ);
  free(flag);
  free(surv);
  free(Rs);
  free(ts);
  free(nok);
  free(Rv);
  free(tv);
  free(hv);
  free(cnt);
  free(amb);
  free(sd);
  return 0;
}
