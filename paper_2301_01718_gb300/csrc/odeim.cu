// ODEIM_{n_p}(Phi) (Eq. odeim of the paper): the DEIM points, then greedy
// oversampling points, each maximising lambda_min(A^T A + phi_i phi_i^T)
// (A = P^T Phi over the points so far, phi_i a candidate row).
//
// Each greedy step is an exact arg-max over all N rows (ties within
// relative tie_tol go to the lowest row), but the exact FP64 score is only
// evaluated on rows that can still win:
//   * rows are bucketed once per basis by an upper bound of their squared
//     norm nrm_i = |Phi[i, :]|^2 (buckets of a factor 2^(1/4), in
//     decreasing order; each bucket records its largest bound);
//   * DEIM step l: |r_i| <= sqrt(nrm_i) sqrt(1 + |c|^2) for the interpolation
//     residual r = phi_l - Phi_{:, <l} c, so rows with
//     nrm_i < s*^2 (1 - 2 tie_tol)^2 / (1 + |c|^2) cannot reach the best score
//     s* found on a probe of the largest-norm rows;
//   * ODEIM step: lambda_min(M + phi phi^T) <= lambda_1(M) + |phi|^2 and
//     <= min(lambda_2, lambda_1 + (w_1 . phi)^2) (Rayleigh quotient on the
//     eigenvector w_1, and interlacing), so rows below either bound are
//     skipped; survivors get the smallest root of the secular equation
//     1 + sum_j z_j^2 / (lambda_j - mu) = 0, z = W^T phi, by bisection.
// Every decision is taken in FP64 on the same quantity an FP64 reference
// computes, so the chosen points do not depend on the pruning.
#include <math.h>

#include <utility>

#include "common.cuh"
#include "internal.h"

namespace hy {

constexpr int kNB = 256;       // norm buckets
constexpr int kProbe = 2048;   // rows scored before the bound is applied

struct OdCtl {
  unsigned long long smax;  // bits of the best score so far (>= 0)
  int argmin;               // winning row (lowest index within the tie window)
  int n_c;                  // ordered rows to score
  double cn2;               // 1 + |c|^2            (DEIM)
  double lam1, lam2, lmax;  // eigenvalues of M (ODEIM)
  unsigned long long lbest;  // packed (heuristic score bits, position) (ODEIM)
  unsigned long long ubest;  // packed (upper bound bits, position) (ODEIM)
  // counters over one ODEIM call: DEIM rows scored, ODEIM rows screened,
  // ODEIM exact scores, greedy steps
  unsigned long long stat[4];
};

size_t odeim_ctl_bytes() { return 256; }

// counters of the last ODEIM call (the control block heads the workspace)
void odeim_stats(const void* ws, unsigned long long* out4, cudaStream_t s) {
  const OdCtl* c = (const OdCtl*)ws;
  cudaMemcpyAsync(out4, c->stat, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
}

// ---- row norms and buckets --------------------------------------------------

HY_DEV int nrm_bucket(float v) {
  if (!(v > 0.0f)) return kNB - 1;
  int b = (int)floorf(24.0f - 4.0f * log2f(v));
  return b < 0 ? 0 : (b > kNB - 2 ? kNB - 2 : b);
}

template <typename T>
__global__ void k_rownorm(const T* __restrict__ phi, int64_t N, int m, float* __restrict__ nrm,
                          unsigned char* __restrict__ bkt, int* __restrict__ bcnt,
                          unsigned int* __restrict__ bmax) {
  __shared__ int sc[kNB];
  __shared__ unsigned int sm[kNB];
  for (int i = threadIdx.x; i < kNB; i += blockDim.x) {
    sc[i] = 0;
    sm[i] = 0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    T acc = (T)0;
    for (int j = 0; j < m; ++j) {
      const T x = phi[(int64_t)j * N + i];
      acc = fma(x, x, acc);
    }
    // an upper bound of the exact squared norm (m terms of relative error
    // <= 2^-24 each for FP32 data; 1e-5 covers m <= 128)
    const float up = __double2float_ru((double)acc * (1.0 + 1e-5));
    nrm[i] = up;
    const int b = nrm_bucket(up);
    bkt[i] = (unsigned char)b;
    atomicAdd(&sc[b], 1);
    atomicMax(&sm[b], __float_as_uint(up));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNB; i += blockDim.x) {
    if (sc[i]) {
      atomicAdd(&bcnt[i], sc[i]);
      atomicMax(&bmax[i], sm[i]);
    }
  }
}

__global__ void k_bucket_scan(const int* __restrict__ bcnt, int* __restrict__ bstart,
                              int* __restrict__ bcur) {
  if (threadIdx.x == 0) {
    int a = 0;
    for (int b = 0; b < kNB; ++b) {
      bstart[b] = a;
      bcur[b] = a;
      a += bcnt[b];
    }
    bstart[kNB] = a;
  }
}

// warp-aggregated: lanes with the same bucket share one atomic
__global__ void k_bucket_scatter(int64_t N, const unsigned char* __restrict__ bkt, int* bcur,
                                 int* __restrict__ ord) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; base < N;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + lane;
    const bool valid = i < N;
    const int b = valid ? bkt[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int pos = 0;
    if (valid && lane == leader) pos = atomicAdd(&bcur[b], __popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (valid) ord[pos + rank] = (int)i;
  }
}

// ---- DEIM -------------------------------------------------------------------

// DEIM interpolation coefficients c = A_l^{-1} Phi[P, l] with A_l = P^T Phi[:, :l]
// (rows in pick order).  A_l = L U is kept as a bordered factorisation: the
// DEIM picks are the partial-pivoting order of A_l, so no pivoting is needed
// (|L| <= 1 up to the tie tolerance).  Each step costs two triangular solves
// (one warp, O(l^2)); k_deim_extend then borders L and U with the new point.
// Lf, Uf: 64 x 64 row-major; y = L^{-1} Phi[P, l] is kept for the border.
template <typename T>
__global__ void k_deim_solve(const T* __restrict__ phi, int64_t N, int l,
                             const int* __restrict__ pts, const double* __restrict__ Lf,
                             const double* __restrict__ Uf, double* __restrict__ yv,
                             double* __restrict__ cvec, OdCtl* ctl) {
  __shared__ double y[64], c[64];
  const int lane = threadIdx.x;
  for (int i = 0; i < l; ++i) {  // forward: L y = b
    double acc = 0.0;
    for (int j = lane; j < i; j += 32) acc = fma(Lf[i * 64 + j], y[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[i] = (double)phi[(int64_t)l * N + pts[i]] - acc;
    __syncwarp();
  }
  for (int i = l - 1; i >= 0; --i) {  // backward: U c = y
    double acc = 0.0;
    for (int j = i + 1 + lane; j < l; j += 32) acc = fma(Uf[i * 64 + j], c[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) c[i] = (y[i] - acc) / Uf[i * 64 + i];
    __syncwarp();
  }
  double cn = 0.0;
  for (int j = lane; j < l; j += 32) {
    cvec[j] = c[j];
    yv[j] = y[j];
    cn = fma(c[j], c[j], cn);
  }
  cn = warp_sum(cn);
  if (lane == 0) {
    ctl->cn2 = 1.0 + cn;
    ctl->smax = 0ull;
    ctl->argmin = 0x7fffffff;
    ctl->n_c = 0;
  }
}

// Border the factors with point p_l (ctl->argmin, already committed):
// U[:l, l] = y, U[l, :l] L-row ell with U^T ell = Phi[p_l, :l], U[l][l] = beta.
template <typename T>
__global__ void k_deim_extend(const T* __restrict__ phi, int64_t N, int l, const OdCtl* ctl,
                              double* __restrict__ Lf, double* __restrict__ Uf,
                              const double* __restrict__ yv) {
  __shared__ double ell[64];
  const int lane = threadIdx.x;
  const int p = ctl->argmin;
  for (int j = 0; j < l; ++j) {  // forward with U^T: ell_j U_jj = a_j - sum_{i<j} U_ij ell_i
    double acc = 0.0;
    for (int i = lane; i < j; i += 32) acc = fma(Uf[i * 64 + j], ell[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) ell[j] = ((double)phi[(int64_t)j * N + p] - acc) / Uf[j * 64 + j];
    __syncwarp();
  }
  double dot = 0.0;
  for (int j = lane; j < l; j += 32) {
    Lf[l * 64 + j] = ell[j];
    Uf[j * 64 + l] = yv[j];
    dot = fma(ell[j], yv[j], dot);
  }
  dot = warp_sum(dot);
  if (lane == 0) {
    Lf[l * 64 + l] = 1.0;
    Uf[l * 64 + l] = (double)phi[(int64_t)l * N + p] - dot;
  }
}

// exact |r_i| for the ordered rows [p0, p1) (p1 < 0: up to ctl->n_c)
template <typename T>
__global__ void k_deim_score(const T* __restrict__ phi, int64_t N, int l,
                             const double* __restrict__ cvec, const int* __restrict__ ord,
                             const unsigned char* __restrict__ picked, int p0, int p1,
                             OdCtl* ctl, double* __restrict__ scores) {
  __shared__ double cs[64];
  for (int j = threadIdx.x; j < l; j += blockDim.x) cs[j] = cvec[j];
  __syncthreads();
  const int end = p1 >= 0 ? p1 : ctl->n_c;
  double best = 0.0;
  for (int pos = p0 + blockIdx.x * blockDim.x + threadIdx.x; pos < end;
       pos += gridDim.x * blockDim.x) {
    const int i = ord[pos];
    double sc = -1.0;
    if (!picked[i]) {
      double s = 0.0;
      for (int j = 0; j < l; ++j) s = fma((double)phi[(int64_t)j * N + i], cs[j], s);
      sc = fabs((double)phi[(int64_t)l * N + i] - s);
      best = sc > best ? sc : best;
    }
    scores[pos] = sc;
  }
  best = block_max(best);
  if (threadIdx.x == 0) atomicMax(&ctl->smax, dbits(best));
}

__global__ void k_deim_plan(OdCtl* ctl,
                            const unsigned int* __restrict__ bmax, const int* __restrict__ bstart,
                            int probe_end, double tie_tol) {
  const double s = bitsd(ctl->smax);
  const double lim = s * (1.0 - 2.0 * tie_tol);
  const double tau = lim * lim / (ctl->cn2 * (1.0 + 1e-5));
  int blast = -1;
  for (int b = 0; b < kNB; ++b)
    if (bstart[b + 1] > bstart[b] && (double)__uint_as_float(bmax[b]) >= tau) blast = b;
  int n = blast >= 0 ? bstart[blast + 1] : 0;
  ctl->n_c = n > probe_end ? n : probe_end;
  ctl->stat[0] += (unsigned long long)(ctl->n_c - probe_end);
}

// lowest row among the scored rows within the tie window of the best
__global__ void k_argmin_tie(const double* __restrict__ scores, const int* __restrict__ ord,
                             OdCtl* ctl, double tie_tol) {
  const double lim = bitsd(ctl->smax) * (1.0 - tie_tol);
  const int end = ctl->n_c;
  int best = 0x7fffffff;
  for (int pos = blockIdx.x * blockDim.x + threadIdx.x; pos < end;
       pos += gridDim.x * blockDim.x) {
    const double sc = scores[pos];
    if (sc >= 0.0 && sc >= lim) {
      const int i = ord[pos];
      best = i < best ? i : best;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const int u = __shfl_xor_sync(0xffffffffu, best, o);
    best = u < best ? u : best;
  }
  if ((threadIdx.x & 31) == 0 && best != 0x7fffffff) atomicMin(&ctl->argmin, best);
}

__global__ void k_commit(OdCtl* ctl, int l, int* __restrict__ pts, unsigned char* picked) {
  const int p = ctl->argmin;
  pts[l] = p;
  picked[p] = 1;
}

// ---- ODEIM oversampling -----------------------------------------------------

// M = A^T A over the first l points (m x m, FP64)
template <typename T>
__global__ void k_odeim_gram(const T* __restrict__ phi, int64_t N, int m, const int* __restrict__ pts,
                             int l, double* __restrict__ M) {
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int a = idx / m, b = idx % m;
    double acc = 0.0;
    for (int r = 0; r < l; ++r)
      acc = fma((double)phi[(int64_t)a * N + pts[r]], (double)phi[(int64_t)b * N + pts[r]], acc);
    M[idx] = acc;
  }
}

// M += phi_p phi_p^T for the point just chosen
template <typename T>
__global__ void k_odeim_rank1(const T* __restrict__ phi, int64_t N, int m, const OdCtl* ctl,
                              double* __restrict__ M) {
  const int p = ctl->argmin;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int a = idx / m, b = idx % m;
    M[idx] = fma((double)phi[(int64_t)a * N + p], (double)phi[(int64_t)b * N + p], M[idx]);
  }
}

// sort the Jacobi eigenpairs ascending: lam_s, W_s (m x m column-major);
// reset the step's control block
__global__ void k_odeim_sort(const double* __restrict__ lam, const double* __restrict__ V, int n,
                             int m, double* __restrict__ lam_s, double* __restrict__ W_s,
                             OdCtl* ctl) {
  __shared__ int perm[128];
  __shared__ unsigned long long key[128];
  for (int i = threadIdx.x; i < m; i += blockDim.x) key[i] = dkey(lam[i]);
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {  // ascending rank
    int r = 0;
    for (int i = 0; i < m; ++i) r += (key[i] < key[j]) || (key[i] == key[j] && i < j);
    perm[r] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) lam_s[i] = lam[perm[i]];
    ctl->lam1 = lam[perm[0]];
    ctl->lam2 = m > 1 ? lam[perm[1]] : INFINITY;
    ctl->lmax = lam[perm[m - 1]];
    ctl->smax = 0ull;
    ctl->lbest = 0ull;
    ctl->ubest = 0ull;
    ctl->argmin = 0x7fffffff;
    ctl->n_c = 0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int j = idx / m, a = idx % m;
    W_s[idx] = V[(int64_t)perm[j] * n + a];
  }
}

// Smallest root of 1 + sum_j z_j^2 / (lam_j - mu) (lam ascending): with
// mu = l1 + tau and d_j = lam_j - l1 it is the root in (0, min(d_2, |z|^2)] of
//   h(tau) = tau (1 + sum_{j>=2} z_j^2 / (d_j - tau)) - z_1^2,
// which is increasing and has no pole at tau = 0 (the secular equation
// multiplied by tau).  Start: the root of the quadratic model with the sum
// expanded to first order in tau; then Newton steps on h kept inside a
// shrinking bracket (bisection when a step leaves it), until the step is
// below 2 ulp of tau.  One warp; lane j holds z_j and z_{j+32}.
__device__ double secular_min_warp(const double* __restrict__ W, const double* __restrict__ lam,
                                   int m, const double* rb, double l1, double l2) {
  const int lane = threadIdx.x & 31;
  double z0 = 0.0, z1 = 0.0;
  const int j0 = lane, j1 = lane + 32;
  if (j0 < m)
    for (int a = 0; a < m; ++a) z0 = fma(W[j0 * m + a], rb[a], z0);
  if (j1 < m)
    for (int a = 0; a < m; ++a) z1 = fma(W[j1 * m + a], rb[a], z1);
  const double q0 = z0 * z0, q1 = z1 * z1;
  const double zz = warp_sum(q0 + q1);
  const double zf = __shfl_sync(0xffffffffu, q0, 0);  // z_1^2
  if (m == 1) return l1 + zf;
  // shifted poles of the other terms (lane 0's first slot is the pole itself)
  const double d0 = lam[j0 < m ? j0 : 0] - l1, d1 = j1 < m ? lam[j1] - l1 : 0.0;
  const double w0 = (j0 >= 1 && j0 < m) ? q0 : 0.0, w1 = j1 < m ? q1 : 0.0;
  double hi = fmin(l2 - l1, zz), lo = 0.0;
  if (!(hi > 0.0) || zf == 0.0) return l1;  // z_1 = 0 or a double eigenvalue
  // quadratic model: S0 = sum w/d, S1 = sum w/d^2
  double s0 = 0.0, s1 = 0.0;
  if (w0 > 0.0) {
    const double r = 1.0 / d0;
    s0 = w0 * r;
    s1 = w0 * r * r;
  }
  if (w1 > 0.0) {
    const double r = 1.0 / d1;
    s0 = s0 + w1 * r;
    s1 = s1 + w1 * r * r;
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  const double bq = 1.0 + s0;
  double tau = 2.0 * zf / (bq + sqrt(bq * bq + 4.0 * s1 * zf));
  if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
  const double eps = 2.220446049250313e-16;
  for (int itr = 0; itr < 200; ++itr) {
    double g = 0.0, dg = 0.0;
    if (w0 > 0.0) {
      const double r = 1.0 / (d0 - tau);
      g = w0 * r;
      dg = w0 * r * r;
    }
    if (w1 > 0.0) {
      const double r = 1.0 / (d1 - tau);
      g = g + w1 * r;
      dg = dg + w1 * r * r;
    }
    g = warp_sum(g);
    dg = warp_sum(dg);
    const double h = tau * (1.0 + g) - zf;
    if (h == 0.0) break;
    if (h < 0.0)
      lo = tau;
    else
      hi = tau;
    if (hi - lo <= 2.0 * eps * hi) {
      tau = hi;
      break;
    }
    double nt = tau - h / ((1.0 + g) + tau * dg);
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    const bool done = fabs(nt - tau) <= 2.0 * eps * tau;
    tau = nt;
    if (done) break;
  }
  return l1 + tau;
}

// One warp per ordered row in [p0, p1) (p1 < 0: up to ctl->n_c).  With
// `prune`, rows whose Rayleigh bound cannot reach lim = smax (1 - 2 tie)
// are skipped (smax read at kernel start).  Lane j holds z_j and z_{j+32}.
template <typename T>
__global__ void k_odeim_score(const T* __restrict__ phi, int64_t N, int m,
                              const double* __restrict__ lam_s, const double* __restrict__ W_s,
                              const int* __restrict__ ord, const unsigned char* __restrict__ picked,
                              int p0, int p1, int prune, double tie_tol, OdCtl* ctl,
                              double* __restrict__ scores) {
  extern __shared__ double sh[];
  double* W = sh;             // m x m column-major (column j = eigenvector j)
  double* lam = W + m * m;    // m
  double* rowbuf = lam + 64;  // per warp: 64
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) W[i] = W_s[i];
  for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = lam_s[i];
  __syncthreads();
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  const double lim = bitsd(ctl->smax) * (1.0 - 2.0 * tie_tol);
  const int end = p1 >= 0 ? p1 : ctl->n_c;
  double* rb = rowbuf + 64 * wid;
  double best = 0.0;
  for (int pos = p0 + blockIdx.x * nw + wid; pos < end; pos += gridDim.x * nw) {
    const int i = ord[pos];
    double sc = -1.0;
    if (!picked[i]) {
      for (int a = lane; a < m; a += 32) rb[a] = (double)phi[(int64_t)a * N + i];
      __syncwarp();
      bool skip = false;
      if (prune) {
        // z_1 = w_1 . phi: Rayleigh-quotient and interlacing upper bound
        double d = 0.0;
        for (int a = lane; a < m; a += 32) d = fma(W[a], rb[a], d);
        d = warp_sum(d);
        const double ub = fmin(l2, l1 + d * d);
        skip = ub * (1.0 + 1e-12) < lim;
      }
      if (!skip) {
        sc = secular_min_warp(W, lam, m, rb, l1, l2);
        best = sc > best ? sc : best;
      }
      __syncwarp();
    }
    if (lane == 0) scores[pos] = sc;
  }
  best = block_max(best);
  if (threadIdx.x == 0) atomicMax(&ctl->smax, dbits(best));
}

// FP32 screen of the ordered rows [p0, ctl->n_c): a rigorous upper bound U
// of lambda_min(M + phi phi^T) into scores[pos] (-1 for picked rows), and
// the rows with the largest upper bound and the largest heuristic lower bound
// (the 2x2 bound of the cited ODEIM construction) packed into ctl->ubest /
// ctl->lbest for the exact probe.  With z = W^T phi and mu the root,
//   z1^2/(mu - l1) = 1 + sum_{j>=2} z_j^2/(l_j - mu)
//                 >= 1 + sum_{2<=j<=KS} z_j^2/(l_j - l1) + rest/(lmax - l1) =: c
// (l1 <= mu <= l_j), so mu <= l1 + z1^2 / c; also mu <= l2.  The KS leading
// z_j are FP32 dot products with |error| <= d = 8e-6 |phi| (m <= 64): z1 is
// rounded up, the others and |phi|^2 down, so the bound stays an upper bound.
constexpr int KS = 8;
template <typename T>
__global__ void k_odeim_screen(const T* __restrict__ phi, int64_t N, int m,
                               const double* __restrict__ W_s, const double* __restrict__ lam_s,
                               const float* __restrict__ nrm, const int* __restrict__ ord,
                               const unsigned char* __restrict__ picked, int p0, OdCtl* ctl,
                               double* __restrict__ scores) {
  __shared__ float wk[KS][64];
  __shared__ double inv[KS];
  const int ks = m < KS ? m : KS;
  const double l1 = ctl->lam1, l2 = ctl->lam2, lm = ctl->lmax;
  for (int i = threadIdx.x; i < KS * 64; i += blockDim.x) {
    const int j = i / 64, a = i % 64;
    wk[j][a] = (j < ks && a < m) ? (float)W_s[j * m + a] : 0.f;
  }
  for (int j = threadIdx.x; j < KS; j += blockDim.x)
    inv[j] = (j >= 1 && j < ks && lam_s[j] > l1) ? 1.0 / (lam_s[j] - l1) : 0.0;
  __syncthreads();
  const double invm = lm > l1 ? 1.0 / (lm - l1) : 0.0;
  const int end = ctl->n_c;
  unsigned long long bestL = 0ull, bestU = 0ull, cnt = 0;
  for (int pos = p0 + blockIdx.x * blockDim.x + threadIdx.x; pos < end;
       pos += gridDim.x * blockDim.x) {
    const int i = ord[pos];
    if (picked[i]) {
      scores[pos] = -1.0;
      continue;
    }
    float zf[KS];
#pragma unroll
    for (int j = 0; j < KS; ++j) zf[j] = 0.f;
    for (int a = 0; a < m; ++a) {
      const float x = (float)phi[(int64_t)a * N + i];
#pragma unroll
      for (int j = 0; j < KS; ++j) zf[j] = fmaf(wk[j][a], x, zf[j]);
    }
    const double nr = (double)nrm[i];
    const double dlt = 8e-6 * sqrt(nr);
    const double z1u = fabs((double)zf[0]) + dlt;
    double c = 1.0, used = z1u * z1u;
#pragma unroll
    for (int j = 1; j < KS; ++j) {
      if (j < ks) {
        const double zl = fmax(fabs((double)zf[j]) - dlt, 0.0);
        c += zl * zl * inv[j];
        used += (fabs((double)zf[j]) + dlt) * (fabs((double)zf[j]) + dlt);
      }
    }
    const double rest = nr * (1.0 - 3e-5) - used;
    if (rest > 0.0) c += rest * invm;
    double U = l1 + z1u * z1u / c;
    if (m > 1) U = fmin(U, l2);
    U = U * (1.0 + 1e-12);
    scores[pos] = U;
    ++cnt;
    const double g = m > 1 ? l2 - l1 : 0.0;
    const double z1 = (double)zf[0];
    const double sg = g + nr;
    const double L = l1 + 0.5 * (sg - sqrt(fmax(sg * sg - 4.0 * g * z1 * z1, 0.0)));
    const unsigned long long kL =
        ((unsigned long long)(__double_as_longlong(L) >> 20) << 32) | (unsigned)pos;
    const unsigned long long kU =
        ((unsigned long long)(__double_as_longlong(U) >> 20) << 32) | (unsigned)pos;
    bestL = kL > bestL ? kL : bestL;
    bestU = kU > bestU ? kU : bestU;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long u = __shfl_xor_sync(0xffffffffu, bestL, o);
    bestL = u > bestL ? u : bestL;
    u = __shfl_xor_sync(0xffffffffu, bestU, o);
    bestU = u > bestU ? u : bestU;
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (bestL) atomicMax(&ctl->lbest, bestL);
    if (bestU) atomicMax(&ctl->ubest, bestU);
    atomicAdd(&ctl->stat[1], cnt);
  }
}

// exact score of the heuristic best row -> raise smax to it
template <typename T>
__global__ void k_odeim_probe_best(const T* __restrict__ phi, int64_t N, int m,
                                   const double* __restrict__ lam_s, const double* __restrict__ W_s,
                                   const int* __restrict__ ord, OdCtl* ctl,
                                   double* __restrict__ scores) {
  __shared__ double W[64 * 64], lam[64], rb[2][64];
  const unsigned long long key[2] = {ctl->lbest, ctl->ubest};
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) W[i] = W_s[i];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    lam[i] = lam_s[i];
    for (int t = 0; t < 2; ++t)
      if (key[t]) rb[t][i] = (double)phi[(int64_t)i * N + ord[(int)(key[t] & 0xffffffffull)]];
  }
  __syncthreads();
  const int t = threadIdx.x >> 5;
  if (t < 2 && key[t]) {
    const double mu = secular_min_warp(W, lam, m, rb[t], ctl->lam1, ctl->lam2);
    if ((threadIdx.x & 31) == 0) atomicMax(&ctl->smax, dbits(mu));
  }
}

// exact scores of the screened rows whose bound reaches smax (1 - 2 tie);
// the others get -1.  One warp per row.
template <typename T>
__global__ void k_odeim_exact(const T* __restrict__ phi, int64_t N, int m,
                              const double* __restrict__ lam_s, const double* __restrict__ W_s,
                              const int* __restrict__ ord, int p0, double tie_tol, OdCtl* ctl,
                              double* __restrict__ scores) {
  extern __shared__ double sh[];
  double* W = sh;
  double* lam = W + m * m;
  double* rowbuf = lam + 64;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) W[i] = W_s[i];
  for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = lam_s[i];
  __syncthreads();
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  const double lim = bitsd(ctl->smax) * (1.0 - 2.0 * tie_tol);
  const int end = ctl->n_c;
  double* rb = rowbuf + 64 * wid;
  double best = 0.0;
  unsigned long long cnt = 0;
  for (int pos = p0 + blockIdx.x * nw + wid; pos < end; pos += gridDim.x * nw) {
    const double U = scores[pos];
    if (U < lim) {
      if (lane == 0 && U >= 0.0) scores[pos] = -1.0;
      continue;
    }
    const int i = ord[pos];
    for (int a = lane; a < m; a += 32) rb[a] = (double)phi[(int64_t)a * N + i];
    __syncwarp();
    const double mu = secular_min_warp(W, lam, m, rb, l1, l2);
    __syncwarp();
    if (lane == 0) scores[pos] = mu;
    best = mu > best ? mu : best;
    ++cnt;
  }
  best = block_max(best);
  if (threadIdx.x == 0) atomicMax(&ctl->smax, dbits(best));
  if (lane == 0 && cnt) atomicAdd(&ctl->stat[2], cnt);
}

__global__ void k_odeim_plan(OdCtl* ctl, const unsigned int* __restrict__ bmax,
                             const int* __restrict__ bstart, int probe_end, double tie_tol) {
  ctl->stat[3] += 1;
  const double lim = bitsd(ctl->smax) * (1.0 - 2.0 * tie_tol);
  const double tau = (lim - ctl->lam1) / (1.0 + 1e-5);
  int blast = -1;
  for (int b = 0; b < kNB; ++b)
    if (bstart[b + 1] > bstart[b] && (double)__uint_as_float(bmax[b]) >= tau) blast = b;
  int n = blast >= 0 ? bstart[blast + 1] : 0;
  ctl->n_c = n > probe_end ? n : probe_end;
}

// ---- rank-one update of the eigensystem of M (one per oversampling step) ----
//
// M' = M + phi phi^T with M = W diag(d) W^T (d ascending).  In the basis W,
// M' = diag(d) + z z^T, z = W^T phi; its eigenvalues are the roots of the
// secular equation 1 + sum_i z_i^2 / (d_i - lambda) = 0 (Golub 1973), one in
// each (d_j, d_{j+1}) and the last in (d_n, d_n + |z|^2).  Components with a
// negligible z_i, and pairs of nearly equal d, are deflated first (a Givens
// rotation folds one z component into its neighbour), as in the
// divide-and-conquer eigensolver (Bunch, Nielsen & Sorensen 1978).  Each
// root is found by bisection in coordinates shifted to its nearer pole, so
// that d_i - lambda_j is known to full relative accuracy; z is then
// recomputed from the roots by Loewner's formula (Gu & Eisenstat 1994), which
// makes the eigenvectors (d_i - lambda_j)^{-1} z_i numerically orthogonal.

struct R1Work {
  int nK;          // non-deflated count
  int nD;          // deflated count
  int K[64];       // original indices (ascending d) of the non-deflated
  int D[64];       // deflated indices
  double dK[64];   // their (possibly rotated) d
  double zK[64];   // their z
  double dD[64];   // deflated eigenvalues
  int org[64];     // root j: origin index into K
  double tau[64];  // root j = dK[org[j]] + tau[j]
};

template <typename T>
__global__ void k_r1_prepare(const T* __restrict__ phi, int64_t N, int m, const OdCtl* ctl,
                             const double* __restrict__ d, const double* __restrict__ W,
                             double* __restrict__ Wrot, R1Work* wk) {
  __shared__ double Ws[64 * 64];
  __shared__ double ph[64], z[64], ds[64];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int p = ctl->argmin;
  for (int a = tid; a < m; a += blockDim.x) {
    ph[a] = (double)phi[(int64_t)a * N + p];
    ds[a] = d[a];
  }
  for (int i = tid; i < m * m; i += blockDim.x) Ws[i] = W[i];
  __syncthreads();
  for (int j = wid; j < m; j += nw) {
    double acc = 0.0;
    for (int a = lane; a < m; a += 32) acc = fma(Ws[j * m + a], ph[a], acc);
    acc = warp_sum(acc);
    if (lane == 0) z[j] = acc;
  }
  __syncthreads();
  __shared__ int nonsmall[64], nns, anyclose;
  __shared__ double tol_s, nz_s;
  {
    double r = 0.0, dm = 0.0;
    for (int j = tid; j < m; j += blockDim.x) {
      r = fma(z[j], z[j], r);
      dm = fmax(dm, fabs(ds[j]));
    }
    r = block_sum(r);
    dm = block_max(dm);
    if (tid == 0) {
      nz_s = sqrt(r);
      tol_s = 8.0 * 2.220446049250313e-16 * fmax(dm, r);
      anyclose = 0;
    }
  }
  __syncthreads();
  const double tol = tol_s, nz = nz_s;
  if (tid == 0) {  // integer work only: ordered list of non-negligible z
    int c = 0;
    for (int i = 0; i < m; ++i)
      if (!(fabs(z[i]) * nz <= tol)) nonsmall[c++] = i;
    nns = c;
  }
  __syncthreads();
  for (int k = 1 + tid; k < nns; k += blockDim.x) {  // adjacent pairs, in parallel
    const int ip = nonsmall[k - 1], i = nonsmall[k];
    const double t = hypot(z[ip], z[i]);
    const double c = z[i] / t, sn = z[ip] / t;
    if (fabs(c * sn * (ds[i] - ds[ip])) <= tol) anyclose = 1;
  }
  __syncthreads();
  if (!anyclose) {
    // fast path: no rotation; K = the non-negligible entries, D = the rest
    for (int k = tid; k < nns; k += blockDim.x) {
      const int i = nonsmall[k];
      wk->K[k] = i;
      wk->dK[k] = ds[i];
      wk->zK[k] = z[i];
    }
    if (tid == 0) {
      int nD = 0;
      for (int i = 0, k = 0; i < m; ++i) {
        if (k < nns && nonsmall[k] == i) {
          ++k;
          continue;
        }
        wk->D[nD] = i;
        wk->dD[nD++] = ds[i];
      }
      wk->nK = nns;
      wk->nD = nD;
    }
  } else if (tid == 0) {
    int nK = 0, nD = 0, prev = -1;
    for (int i = 0; i < m; ++i) {
      if (fabs(z[i]) * nz <= tol) {
        wk->D[nD] = i;
        wk->dD[nD++] = ds[i];
        continue;
      }
      if (prev < 0) {
        prev = i;
        continue;
      }
      const double t = hypot(z[prev], z[i]);
      const double c = z[i] / t, sn = z[prev] / t;
      if (fabs(c * sn * (ds[i] - ds[prev])) <= tol) {
        // fold z[prev] into z[i]; prev becomes an eigenpair
        const double dp = c * c * ds[prev] + sn * sn * ds[i];
        const double di = sn * sn * ds[prev] + c * c * ds[i];
        for (int a2 = 0; a2 < m; ++a2) {
          const double wp = Ws[prev * m + a2], wi = Ws[i * m + a2];
          Ws[prev * m + a2] = c * wp - sn * wi;
          Ws[i * m + a2] = sn * wp + c * wi;
        }
        z[prev] = 0.0;
        z[i] = t;
        ds[i] = di;
        wk->D[nD] = prev;
        wk->dD[nD++] = dp;
        prev = i;
      } else {
        wk->K[nK] = prev;
        wk->dK[nK] = ds[prev];
        wk->zK[nK++] = z[prev];
        prev = i;
      }
    }
    if (prev >= 0) {
      wk->K[nK] = prev;
      wk->dK[nK] = ds[prev];
      wk->zK[nK++] = z[prev];
    }
    wk->nK = nK;
    wk->nD = nD;
  }
  __syncthreads();
  for (int i = tid; i < m * m; i += blockDim.x) Wrot[i] = Ws[i];
}

// One warp per root (CTA j); Delta[i * 64 + j] = d_i - lambda_j.
__global__ void k_r1_roots(R1Work* wk, double* __restrict__ Delta) {
  const int j = blockIdx.x, lane = threadIdx.x;
  const int nK = wk->nK;
  if (j >= nK) return;
  double dv[2], z2[2];
  for (int u = 0; u < 2; ++u) {
    const int i = lane + 32 * u;
    dv[u] = i < nK ? wk->dK[i] : 0.0;
    const double zi = i < nK ? wk->zK[i] : 0.0;
    z2[u] = zi * zi;
  }
  double rho = warp_sum(z2[0] + z2[1]);
  const double dj = wk->dK[j];
  int o;
  double lo, hi;
  if (j == nK - 1) {
    o = j;
    lo = 0.0;
    hi = rho;
  } else {
    const double dn = wk->dK[j + 1];
    const double mid = 0.5 * (dj + dn);
    double f = 0.0;
    for (int u = 0; u < 2; ++u)
      if (lane + 32 * u < nK) f = f + z2[u] / (dv[u] - mid);
    f = 1.0 + warp_sum(f);
    if (f >= 0.0) {
      o = j;
      lo = 0.0;
      hi = mid - dj;
    } else {
      o = j + 1;
      lo = mid - dn;
      hi = 0.0;
    }
  }
  const double dorg = wk->dK[o];
  double del[2];
  for (int u = 0; u < 2; ++u) del[u] = dv[u] - dorg;
  // f(tau) = 1 + sum_i z_i^2 / (del_i - tau), increasing between the poles:
  // Newton steps kept inside a shrinking bracket (bisection when a step
  // leaves it); the iterate itself is the result once the step is below
  // 2 ulp or the bracket has collapsed.
  double t = (o == j) ? 0.5 * hi : 0.5 * lo;
  double tau = t;
  const double eps = 2.220446049250313e-16;
  for (int it = 0; it < 400; ++it) {
    if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
    tau = t;
    if (t <= lo || t >= hi) break;
    double f = 0.0, df = 0.0;
    for (int u = 0; u < 2; ++u)
      if (lane + 32 * u < nK) {
        const double r = 1.0 / (del[u] - t);
        f = f + z2[u] * r;
        df = df + z2[u] * r * r;
      }
    f = 1.0 + warp_sum(f);
    df = warp_sum(df);
    if (f == 0.0) break;
    if (f < 0.0)
      lo = t;
    else
      hi = t;
    if (hi - lo <= 2.0 * eps * fmax(fabs(hi), fabs(lo))) {
      tau = 0.5 * (lo + hi);
      break;
    }
    double nt = t - f / df;
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    if (fabs(nt - t) <= 2.0 * eps * fabs(t)) {
      tau = nt;
      break;
    }
    t = nt;
  }
  for (int u = 0; u < 2; ++u) {
    const int i = lane + 32 * u;
    if (i < nK) Delta[i * 64 + j] = del[u] - tau;
  }
  if (lane == 0) {
    wk->org[j] = o;
    wk->tau[j] = tau;
  }
}

// Eigenvector j of diag(dK) + z z^T (Loewner z), mapped back through W.
// CTA j writes column j of Wnew (m values) and lamnew[j].
__global__ void k_r1_vectors(const R1Work* __restrict__ wk, const double* __restrict__ Delta,
                             const double* __restrict__ Wrot, int m, double* __restrict__ Wnew,
                             double* __restrict__ lamnew) {
  __shared__ double zh[64], v[64];
  const int j = blockIdx.x, tid = threadIdx.x;
  const int nK = wk->nK;
  if (j >= nK) return;
  if (tid < nK) {
    const int i = tid;
    const double di = wk->dK[i];
    double pr = -Delta[i * 64 + i];  // lambda_i - d_i > 0
    for (int q = 0; q < nK; ++q)
      if (q != i) pr *= (-Delta[i * 64 + q]) / (wk->dK[q] - di);
    const double zz = sqrt(fmax(pr, 0.0));
    zh[i] = wk->zK[i] >= 0.0 ? zz : -zz;
  }
  __syncthreads();
  if (tid < nK) v[tid] = zh[tid] / Delta[tid * 64 + j];
  __syncthreads();
  double nrm = 0.0;
  if (tid < 64) nrm = tid < nK ? v[tid] * v[tid] : 0.0;
  nrm = block_sum(nrm);
  const double inv = 1.0 / sqrt(nrm);
  for (int a = tid; a < m; a += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nK; ++i) acc = fma(Wrot[wk->K[i] * m + a], v[i], acc);
    Wnew[j * m + a] = acc * inv;
  }
  if (tid == 0) lamnew[j] = wk->dK[wk->org[j]] + wk->tau[j];
}

// Merge deflated and new eigenpairs, ascending; reset the step's control.
__global__ void k_r1_merge(const R1Work* __restrict__ wk, const double* __restrict__ Wrot,
                           const double* __restrict__ Wnew, const double* __restrict__ lamnew,
                           int m, double* __restrict__ d_out, double* __restrict__ W_out,
                           OdCtl* ctl) {
  __shared__ double lv[64];
  __shared__ unsigned long long key[64];
  __shared__ int src[64];  // >= 0: new pair index; < 0: -(deflated idx)-1
  __shared__ int perm[64];
  const int tid = threadIdx.x;
  const int nK = wk->nK, nD = wk->nD;
  for (int j = tid; j < m; j += blockDim.x) {
    if (j < nK) {
      lv[j] = lamnew[j];
      src[j] = j;
    } else {
      lv[j] = wk->dD[j - nK];
      src[j] = -wk->D[j - nK] - 1;
    }
    key[j] = dkey(lv[j]);
  }
  __syncthreads();
  for (int j = tid; j < m; j += blockDim.x) {  // rank = position in ascending order
    int r = 0;
    for (int i = 0; i < m; ++i) r += (key[i] < key[j]) || (key[i] == key[j] && i < j);
    perm[r] = j;
  }
  __syncthreads();
  if (tid == 0) {
    ctl->lam1 = lv[perm[0]];
    ctl->lam2 = m > 1 ? lv[perm[1]] : INFINITY;
    ctl->lmax = lv[perm[m - 1]];
    ctl->smax = 0ull;
    ctl->lbest = 0ull;
    ctl->ubest = 0ull;
    ctl->argmin = 0x7fffffff;
    ctl->n_c = 0;
  }
  (void)nD;
  for (int i = tid; i < m; i += blockDim.x) d_out[i] = lv[perm[i]];
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int j = idx / m, a = idx % m;
    const int sidx = src[perm[j]];
    W_out[idx] = sidx >= 0 ? Wnew[sidx * m + a] : Wrot[(-sidx - 1) * m + a];
  }
}

__global__ void k_pad_sym2(const double* __restrict__ M, int m, int n, double* __restrict__ P) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int a = idx / n, b = idx % n;
    P[idx] = (a < m && b < m) ? M[a * m + b] : 0.0;
  }
}

// ---- driver -----------------------------------------------------------------

struct OdeimBufs {
  float* nrm;
  unsigned char* bkt;
  unsigned char* picked;
  int* ord;
  int* bcnt;
  int* bstart;
  int* bcur;
  unsigned int* bmax;
  double* scores;
  double* cvec;
  double* M;
  double* V;
  double* lam;
  double* lam_s;
  double* W_s;
  double* Mp;
  double* Wrot;
  double* Wnew;
  double* lamnew;
  double* Delta;
  double* lam_s2;
  double* W_s2;
  R1Work* r1;
  double* jbuf;
  double* jscale;
  int* jflag;
  double* Lf;
  double* Uf;
  double* yv;
  OdCtl* ctl;
};

size_t odeim_ws_bytes(int64_t N, int m) {
  size_t b = 0;
  b += N * sizeof(float) + N + N + N * sizeof(int) + N * sizeof(double);
  b += (3 * (kNB + 1) + kNB) * sizeof(int);
  b += sizeof(double) * (64 + 6 * (size_t)(m + 1) * (m + 1) + 4 * m + 64);
  b += 16 * 256;
  b += sizeof(double) * (5 * 64 * 64 + 3 * 64) + sizeof(R1Work) + 16 * 256;
  b += sizeof(double) * 2 * (m + 1) * (m + 1) + 3 * 256;
  b += sizeof(double) * (2 * 64 * 64 + 64) + 3 * 256;
  return b + 4096;
}

static OdeimBufs carve(void* ws, int64_t N, int m) {
  OdeimBufs o;
  char* p = (char*)ws;
  auto take = [&](size_t n) {
    char* r = p;
    p += (n + 255) & ~(size_t)255;
    return r;
  };
  o.ctl = (OdCtl*)take(256);
  o.scores = (double*)take(N * sizeof(double));
  o.nrm = (float*)take(N * sizeof(float));
  o.ord = (int*)take(N * sizeof(int));
  o.bkt = (unsigned char*)take(N);
  o.picked = (unsigned char*)take(N);
  o.bcnt = (int*)take((kNB + 1) * sizeof(int));
  o.bstart = (int*)take((kNB + 1) * sizeof(int));
  o.bcur = (int*)take((kNB + 1) * sizeof(int));
  o.bmax = (unsigned int*)take(kNB * sizeof(int));
  o.cvec = (double*)take(64 * sizeof(double));
  o.M = (double*)take((size_t)m * m * sizeof(double));
  o.V = (double*)take((size_t)(m + 1) * (m + 1) * sizeof(double));
  o.lam = (double*)take((m + 1) * sizeof(double));
  o.lam_s = (double*)take((m + 1) * sizeof(double));
  o.W_s = (double*)take((size_t)m * m * sizeof(double));
  o.Mp = (double*)take((size_t)(m + 1) * (m + 1) * sizeof(double));
  o.Wrot = (double*)take((size_t)64 * 64 * sizeof(double));
  o.Wnew = (double*)take((size_t)64 * 64 * sizeof(double));
  o.lamnew = (double*)take(64 * sizeof(double));
  o.Delta = (double*)take((size_t)64 * 64 * sizeof(double));
  o.lam_s2 = (double*)take(64 * sizeof(double));
  o.W_s2 = (double*)take((size_t)64 * 64 * sizeof(double));
  o.r1 = (R1Work*)take(sizeof(R1Work));
  o.jbuf = (double*)take((size_t)2 * (m + 1) * (m + 1) * sizeof(double));
  o.jscale = (double*)take(64);
  o.jflag = (int*)take(64);
  o.Lf = (double*)take((size_t)64 * 64 * sizeof(double));
  o.Uf = (double*)take((size_t)64 * 64 * sizeof(double));
  o.yv = (double*)take(64 * sizeof(double));
  return o;
}

template <typename T>
int launch_odeim(const T* phi, int64_t N, int m, int np, double tie_tol, int* pts, void* ws,
                 void* host_pinned, cudaStream_t s, void (*mark)(void*, int), void* mark_arg) {
  if (m <= 0) return 0;
  if (np > N) np = (int)N;
  OdeimBufs o = carve(ws, N, m);
  auto M_ = [&](int id) {
    if (mark) mark(mark_arg, id);
  };
  M_(12);
  cudaMemsetAsync(o.ctl, 0, sizeof(OdCtl), s);
  cudaMemsetAsync(o.picked, 0, N, s);
  cudaMemsetAsync(o.bcnt, 0, (kNB + 1) * sizeof(int), s);
  cudaMemsetAsync(o.bmax, 0, kNB * sizeof(int), s);
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_rownorm<T><<<(int)blocks, 256, 0, HY_S(s)>>>(phi, N, m, o.nrm, o.bkt, o.bcnt, o.bmax);
  k_bucket_scan<<<1, 32, 0, HY_S(s)>>>(o.bcnt, o.bstart, o.bcur);
  k_bucket_scatter<<<(int)blocks, 256, 0, HY_S(s)>>>(N, o.bkt, o.bcur, o.ord);
  const int probe = (int)(N < kProbe ? N : kProbe);
  M_(-13);
  // DEIM
  for (int l = 0; l < m; ++l) {
    k_deim_solve<T><<<1, 32, 0, HY_S(s)>>>(phi, N, l, pts, o.Lf, o.Uf, o.yv, o.cvec, o.ctl);
    k_deim_score<T><<<(probe + 255) / 256, 256, 0, HY_S(s)>>>(phi, N, l, o.cvec, o.ord, o.picked, 0,
                                                        probe, o.ctl, o.scores);
    k_deim_plan<<<1, 1, 0, HY_S(s)>>>(o.ctl, o.bmax, o.bstart, probe, tie_tol);
    k_deim_score<T><<<152 * 8, 256, 0, HY_S(s)>>>(phi, N, l, o.cvec, o.ord, o.picked, probe, -1,
                                            o.ctl, o.scores);
    k_argmin_tie<<<152 * 4, 256, 0, HY_S(s)>>>(o.scores, o.ord, o.ctl, tie_tol);
    k_commit<<<1, 1, 0, HY_S(s)>>>(o.ctl, l, pts, o.picked);
    if (l + 1 < m) k_deim_extend<T><<<1, 32, 0, HY_S(s)>>>(phi, N, l, o.ctl, o.Lf, o.Uf, o.yv);
  }
  if (mark) {  // DEIM ends, oversampling begins
    mark(mark_arg, -12);
    mark(mark_arg, 9);
  }
  if (np <= m) return 0;
  // ODEIM oversampling
  const int n = m % 2 ? m + 1 : m;  // Jacobi wants an even order
  k_odeim_gram<T><<<1, 256, 0, HY_S(s)>>>(phi, N, m, pts, m, o.M);
  const size_t smem = sizeof(double) * ((size_t)m * m + 64 + 64 * 8);
  cudaFuncSetAttribute(k_odeim_score<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_odeim_exact<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  M_(12);
  k_pad_sym2<<<1, 256, 0, HY_S(s)>>>(o.M, m, n, o.Mp);
  if (run_jacobi_multi(o.Mp, n, o.V, o.lam, o.jbuf, o.jflag, (int*)host_pinned, o.jscale,
                       (double*)host_pinned + 1, 60, s) < 0)
    return -1;
  k_odeim_sort<<<1, 256, 0, HY_S(s)>>>(o.lam, o.V, n, m, o.lam_s, o.W_s, o.ctl);
  M_(-13);
  for (int l = m; l < np; ++l) {
    M_(13);
    k_odeim_score<T><<<(probe + 7) / 8, 256, smem, HY_S(s)>>>(phi, N, m, o.lam_s, o.W_s, o.ord,
                                                        o.picked, 0, probe, 0, tie_tol, o.ctl,
                                                        o.scores);
    k_odeim_plan<<<1, 1, 0, HY_S(s)>>>(o.ctl, o.bmax, o.bstart, probe, tie_tol);
    M_(-14);
    M_(14);
    k_odeim_screen<T><<<152 * 8, 256, 0, HY_S(s)>>>(phi, N, m, o.W_s, o.lam_s, o.nrm, o.ord,
                                                    o.picked, probe, o.ctl, o.scores);
    k_odeim_probe_best<T><<<1, 64, 0, HY_S(s)>>>(phi, N, m, o.lam_s, o.W_s, o.ord, o.ctl,
                                                 o.scores);
    M_(-15);
    M_(15);
    k_odeim_exact<T><<<152 * 8, 256, smem, HY_S(s)>>>(phi, N, m, o.lam_s, o.W_s, o.ord, probe,
                                                      tie_tol, o.ctl, o.scores);
    M_(-16);
    M_(17);
    k_argmin_tie<<<152 * 4, 256, 0, HY_S(s)>>>(o.scores, o.ord, o.ctl, tie_tol);
    k_commit<<<1, 1, 0, HY_S(s)>>>(o.ctl, l, pts, o.picked);
    M_(-18);
    if (l + 1 < np) {
      M_(16);
      k_r1_prepare<T><<<1, 256, 0, HY_S(s)>>>(phi, N, m, o.ctl, o.lam_s, o.W_s, o.Wrot, o.r1);
      k_r1_roots<<<m, 32, 0, HY_S(s)>>>(o.r1, o.Delta);
      k_r1_vectors<<<m, 64, 0, HY_S(s)>>>(o.r1, o.Delta, o.Wrot, m, o.Wnew, o.lamnew);
      k_r1_merge<<<1, 256, 0, HY_S(s)>>>(o.r1, o.Wrot, o.Wnew, o.lamnew, m, o.lam_s2, o.W_s2,
                                         o.ctl);
      std::swap(o.lam_s, o.lam_s2);
      std::swap(o.W_s, o.W_s2);
      M_(-17);
    }
  }
  return 0;
}

template int launch_odeim<float>(const float*, int64_t, int, int, double, int*, void*, void*,
                                 cudaStream_t, void (*)(void*, int), void*);
template int launch_odeim<double>(const double*, int64_t, int, int, double, int*, void*, void*,
                                  cudaStream_t, void (*)(void*, int), void*);

}  // namespace hy
