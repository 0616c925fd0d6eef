// lsr_implicit.cu -- gradient of the refined pose with respect to the points
// (implicit differentiation of the robust alignment at its optimum).
//
// The refinement ends at T* minimising E(xi) = sum_i rho(|T(xi) p_i - q_i|^2)
// over the pairs it holds at convergence (eq. (3)-(4) with the line process
// eliminated, rho(s) = mu s / (mu + s); T(xi) = [Exp(w) | v] T*, the left
// perturbation whose Jacobian is G_p = [-[p]_x | I] of eq. (5)). The
// first-order condition g(xi = 0) = 0 defines T* as a function of the points,
// so for a loss L with gradient dL/dxi in that perturbation,
//   lambda = H^-1 dL/dxi,   dL/dp_i = -R^T dphi_i/dz_i,   dL/dq_i = -dphi_i/dq_i,
// with phi_i = lambda . g_i = 2 rho'(s_i) a_i . r_i, a_i = w_l x z_i + v_l,
// z_i = R p_i + t, r_i = z_i - q_i, and H the exact Hessian of E in xi:
//   H = sum 4 rho''(s) (J^T r)(J^T r)^T + 2 rho'(s) (J^T J + S),
// J^T r = (z x r, r), J^T J = [[|z|^2 I - z z^T, [z]_x], [-[z]_x, I]], and S
// (rotation block only) = (r z^T + z r^T) / 2 - (r . z) I, the second
// derivative of r . Exp(w) z at w = 0, which does not vanish for a robust
// kernel away from a zero residual.
//
// Three launches: (1) every point finds its nearest Q point within eps
// (FP32 grid walk, as the refinement's finest level) and adds its terms of g
// and H, evaluated in FP64, to FP64 per-block partials; (2) one thread sums
// the partials in block order (deterministic) and solves H lambda = dL/dxi by
// Gaussian elimination with partial pivoting in FP64; (3) every point
// recomputes its neighbour (nothing is stored between launches) and writes
// dL/dp_i, and scatters dL/dq_j into its neighbour's row.
#include "lsr_internal.cuh"

namespace lsr {

namespace {

constexpr int kImpThreads = 256;
constexpr int kImpG = 4;        // lanes per nearest-neighbour query
constexpr int kImpSums = 28;    // g (6), H upper triangle (21), count

struct ImpArgs {
  float Rf[9], tf[3];   // the pose in FP32 for the neighbour search
  double R[9], t[3];    // and in FP64 for the terms
  float eps2;
  double mu;
};

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Nearest Q point within eps of R p + t for the point of this lane group;
// every lane of the group returns the same (bt, z in FP32).
__device__ __forceinline__ int imp_nn(const GridParams &g, const int *__restrict__ start,
                                      const float4 *__restrict__ Xe, const ImpArgs &a, float px, float py, float pz) {
  const float x = fmaf(a.Rf[0], px, fmaf(a.Rf[1], py, fmaf(a.Rf[2], pz, a.tf[0])));
  const float y = fmaf(a.Rf[3], px, fmaf(a.Rf[4], py, fmaf(a.Rf[5], pz, a.tf[1])));
  const float z = fmaf(a.Rf[6], px, fmaf(a.Rf[7], py, fmaf(a.Rf[8], pz, a.tf[2])));
  float best;
  int bt, bidx;
  group_nn<kImpG>(g, start, Xe, x, y, z, a.eps2, best, bt, bidx);
  return bt;
}

__device__ __forceinline__ void imp_point(const ImpArgs &a, float px, float py, float pz, float4 q, double z[3],
                                          double r[3], double &s, double &d1, double &d2) {
  const double p[3] = {px, py, pz};
  for (int k = 0; k < 3; ++k) z[k] = a.R[3 * k] * p[0] + a.R[3 * k + 1] * p[1] + a.R[3 * k + 2] * p[2] + a.t[k];
  r[0] = z[0] - (double)q.x, r[1] = z[1] - (double)q.y, r[2] = z[2] - (double)q.z;
  s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  const double den = a.mu + s;
  d1 = a.mu * a.mu / (den * den);            // rho'(s)
  d2 = -2.0 * a.mu * a.mu / (den * den * den);  // rho''(s)
}

__global__ void __launch_bounds__(kImpThreads) k_implicit_sums(const float *__restrict__ P, int nP,
                                                               const GridParams *gep, const int *__restrict__ start,
                                                               const float4 *__restrict__ Xe, ImpArgs a,
                                                               double *__restrict__ partials) {
  constexpr int G = kImpG, GPB = kImpThreads / G;
  const GridParams g = *gep;
  const int grp = threadIdx.x / G, sub = threadIdx.x & (G - 1);
  double acc[kImpSums];
#pragma unroll
  for (int k = 0; k < kImpSums; ++k) acc[k] = 0.0;
  // block-uniform trip count: every lane reaches the group shuffles
  for (int r0 = blockIdx.x * GPB; r0 < nP; r0 += gridDim.x * GPB) {
    const int i = r0 + grp;
    const bool valid = i < nP;
    const float px = valid ? P[3 * i] : __int_as_float(0x7fc00000), py = valid ? P[3 * i + 1] : 0.f,
                pz = valid ? P[3 * i + 2] : 0.f;  // NaN: the query visits no cell
    const int bt = imp_nn(g, start, Xe, a, px, py, pz);
    if (!valid || bt < 0 || sub != 0) continue;
    double z[3], r[3], s, d1, d2;
    imp_point(a, px, py, pz, Xe[bt], z, r, s, d1, d2);
    const double jr[6] = {z[1] * r[2] - z[2] * r[1], z[2] * r[0] - z[0] * r[2], z[0] * r[1] - z[1] * r[0],
                          r[0], r[1], r[2]};
    const double zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2], rz = r[0] * z[0] + r[1] * z[1] + r[2] * z[2];
    // J^T J + S, upper triangle, row-major over (w, v)
    double M[6][6];
    for (int u = 0; u < 3; ++u)
      for (int v = 0; v < 3; ++v) {
        M[u][v] = (u == v ? zz - rz : 0.0) - z[u] * z[v] + 0.5 * (r[u] * z[v] + z[u] * r[v]);
        M[3 + u][3 + v] = u == v ? 1.0 : 0.0;
      }
    // [z]_x in the (w, v) block
    M[0][3] = 0.0, M[0][4] = -z[2], M[0][5] = z[1];
    M[1][3] = z[2], M[1][4] = 0.0, M[1][5] = -z[0];
    M[2][3] = -z[1], M[2][4] = z[0], M[2][5] = 0.0;
    for (int u = 0; u < 6; ++u) acc[u] += 2.0 * d1 * jr[u];
    int k = 6;
    for (int u = 0; u < 6; ++u)
      for (int v = u; v < 6; ++v, ++k) acc[k] += 4.0 * d2 * jr[u] * jr[v] + 2.0 * d1 * M[u][v];
    acc[27] += 1.0;
  }
  __shared__ double sm[kImpThreads / 32][kImpSums];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kImpSums; ++k) {
    const double v = warp_sum_d(acc[k]);
    if (lane == 0) sm[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kImpSums) {
    double s = 0.0;
    for (int q = 0; q < kImpThreads / 32; ++q) s += sm[q][threadIdx.x];
    partials[(size_t)blockIdx.x * kImpSums + threadIdx.x] = s;
  }
}

// out: g (6), H (36, row-major), lambda (6), count, singular flag.
__global__ void k_implicit_solve(const double *__restrict__ partials, int nb, const double *__restrict__ dl,
                                 double *__restrict__ out) {
  __shared__ double seg[256], tot[kImpSums];
  block_sum_partials(partials, nb, kImpSums, kImpSums, seg, tot);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double S[kImpSums];
  for (int k = 0; k < kImpSums; ++k) S[k] = tot[k];
  double H[6][6], A[6][7];
  int k = 6;
  for (int u = 0; u < 6; ++u)
    for (int v = u; v < 6; ++v, ++k) H[u][v] = H[v][u] = S[k];
  for (int u = 0; u < 6; ++u) {
    out[u] = S[u];
    for (int v = 0; v < 6; ++v) out[6 + 6 * u + v] = H[u][v], A[u][v] = H[u][v];
    A[u][6] = dl[u];
  }
  // Gaussian elimination with partial pivoting
  double scale = 0.0;
  for (int u = 0; u < 6; ++u) scale = fmax(scale, fabs(H[u][u]));
  int singular = !(scale > 0.0);
  for (int c = 0; c < 6 && !singular; ++c) {
    int piv = c;
    for (int r = c + 1; r < 6; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (!(fabs(A[piv][c]) > 1e-14 * scale)) {
      singular = 1;
      break;
    }
    if (piv != c)
      for (int q = 0; q < 7; ++q) {
        const double tmp = A[c][q];
        A[c][q] = A[piv][q];
        A[piv][q] = tmp;
      }
    for (int r = c + 1; r < 6; ++r) {
      const double f = A[r][c] / A[c][c];
      for (int q = c; q < 7; ++q) A[r][q] -= f * A[c][q];
    }
  }
  double lam[6] = {0, 0, 0, 0, 0, 0};
  if (!singular)
    for (int c = 5; c >= 0; --c) {
      double v = A[c][6];
      for (int q = c + 1; q < 6; ++q) v -= A[c][q] * lam[q];
      lam[c] = v / A[c][c];
    }
  for (int u = 0; u < 6; ++u) out[42 + u] = lam[u];
  out[48] = S[27];
  out[49] = singular;
}

__global__ void __launch_bounds__(kImpThreads) k_implicit_grad(const float *__restrict__ P, int nP,
                                                               const GridParams *gep, const int *__restrict__ start,
                                                               const float4 *__restrict__ Xe, ImpArgs a,
                                                               const double *__restrict__ solved, int nQ,
                                                               float *__restrict__ dP, float *__restrict__ dQ) {
  constexpr int G = kImpG, GPB = kImpThreads / G;
  const GridParams g = *gep;
  const int grp = threadIdx.x / G, sub = threadIdx.x & (G - 1);
  const double wl[3] = {solved[42], solved[43], solved[44]}, vl[3] = {solved[45], solved[46], solved[47]};
  for (int r0 = blockIdx.x * GPB; r0 < nP; r0 += gridDim.x * GPB) {
    const int i = r0 + grp;
    const bool valid = i < nP;
    const float px = valid ? P[3 * i] : __int_as_float(0x7fc00000), py = valid ? P[3 * i + 1] : 0.f,
                pz = valid ? P[3 * i + 2] : 0.f;
    const int bt = imp_nn(g, start, Xe, a, px, py, pz);
    if (!valid || sub != 0) continue;
    if (bt < 0) {
      dP[3 * i] = dP[3 * i + 1] = dP[3 * i + 2] = 0.f;
      continue;
    }
    const float4 q = Xe[bt];
    double z[3], r[3], s, d1, d2;
    imp_point(a, px, py, pz, q, z, r, s, d1, d2);
    // a_i = w_l x z + v_l
    const double A[3] = {wl[1] * z[2] - wl[2] * z[1] + vl[0], wl[2] * z[0] - wl[0] * z[2] + vl[1],
                         wl[0] * z[1] - wl[1] * z[0] + vl[2]};
    const double ar = A[0] * r[0] + A[1] * r[1] + A[2] * r[2];
    // r x w_l
    const double rw[3] = {r[1] * wl[2] - r[2] * wl[1], r[2] * wl[0] - r[0] * wl[2], r[0] * wl[1] - r[1] * wl[0]};
    double dz[3], gq[3];
    for (int k = 0; k < 3; ++k) {
      dz[k] = 4.0 * d2 * ar * r[k] + 2.0 * d1 * (A[k] + rw[k]);
      gq[k] = 4.0 * d2 * ar * r[k] + 2.0 * d1 * A[k];  // -dphi/dq
    }
    // dL/dp = -R^T dphi/dz
    for (int c = 0; c < 3; ++c)
      dP[3 * i + c] = (float)(-(a.R[c] * dz[0] + a.R[3 + c] * dz[1] + a.R[6 + c] * dz[2]));
    const int j = __float_as_int(q.w);
    if (LSR_IN_BOUNDS(j, nQ, kSiteGridPoint))
      for (int c = 0; c < 3; ++c) atomicAdd(&dQ[3 * j + c], (float)gq[c]);
  }
}

}  // namespace

int implicit_blocks(int nP) {
  int64_t b = lsr_div_up((int64_t)(nP > 0 ? nP : 1) * kImpG, kImpThreads);
  return (int)(b < 1 ? 1 : (b > kSms * 4 ? kSms * 4 : b));
}
int implicit_partials(int nP) { return implicit_blocks(nP) * kImpSums; }

cudaError_t launch_implicit(const float *P, int nP, const GridParams *ge, const int *start_e, const float4 *Xe,
                            int nQ, const double T[16], float eps, double mu, const double *dl_dev,
                            double *partials, double *out, float *dP, float *dQ, cudaStream_t s) {
  ImpArgs a;
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) a.R[3 * r + q] = T[4 * r + q], a.Rf[3 * r + q] = (float)T[4 * r + q];
    a.t[r] = T[4 * r + 3], a.tf[r] = (float)T[4 * r + 3];
  }
  a.eps2 = eps * eps;
  a.mu = mu;
  const int nb = implicit_blocks(nP);
  LSR_LAUNCH(k_implicit_sums<<<nb, kImpThreads, 0, s>>>(P, nP, ge, start_e, Xe, a, partials));
  LSR_LAUNCH(k_implicit_solve<<<1, 256, 0, s>>>(partials, nb, dl_dev, out));
  LSR_LAUNCH(k_implicit_grad<<<nb, kImpThreads, 0, s>>>(P, nP, ge, start_e, Xe, a, out, nQ, dP, dQ));
  return cudaGetLastError();
}

LSR_CHECK_READER(implicit)

}  // namespace lsr
