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
  double lam1, lam2;        // two smallest eigenvalues of M (ODEIM)
};

size_t odeim_ctl_bytes() { return 256; }

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

__global__ void k_bucket_scatter(int64_t N, const unsigned char* __restrict__ bkt, int* bcur,
                                 int* __restrict__ ord) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    ord[atomicAdd(&bcur[bkt[i]], 1)] = (int)i;
}

// ---- DEIM -------------------------------------------------------------------

// c = (P^T Phi_{:, <l})^{-1} P^T phi_l by Gaussian elimination in pick order
// (no pivoting: the DEIM picks are the partial-pivoting order, so the
// multipliers are bounded by one).  Resets the step's control block.
template <typename T>
__global__ void k_deim_solve(const T* __restrict__ phi, int64_t N, int l,
                             const int* __restrict__ pts, double* __restrict__ cvec, OdCtl* ctl) {
  __shared__ double A[64 * 65];
  __shared__ double b[64];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < l * l; idx += nt) {
    const int r = idx / l, cc = idx % l;
    A[r * 65 + cc] = (double)phi[(int64_t)cc * N + pts[r]];
  }
  for (int r = tid; r < l; r += nt) b[r] = (double)phi[(int64_t)l * N + pts[r]];
  __syncthreads();
  for (int k = 0; k < l; ++k) {
    const double piv = A[k * 65 + k];
    for (int idx = tid; idx < (l - k - 1) * (l - k); idx += nt) {
      const int r = k + 1 + idx / (l - k), cc = k + idx % (l - k);
      if (cc == k) continue;
      A[r * 65 + cc] = A[r * 65 + cc] - (A[r * 65 + k] / piv) * A[k * 65 + cc];
    }
    __syncthreads();
    for (int r = k + 1 + tid; r < l; r += nt) b[r] = b[r] - (A[r * 65 + k] / piv) * b[k];
    __syncthreads();
  }
  if (tid == 0) {
    double cn = 1.0;
    for (int r = l - 1; r >= 0; --r) {
      double acc = b[r];
      for (int cc = r + 1; cc < l; ++cc) acc = fma(-A[r * 65 + cc], cvec[cc], acc);
      cvec[r] = acc / A[r * 65 + r];
    }
    for (int r = 0; r < l; ++r) cn = fma(cvec[r], cvec[r], cn);
    ctl->cn2 = cn;
    ctl->smax = 0ull;
    ctl->argmin = 0x7fffffff;
    ctl->n_c = 0;
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
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) perm[i] = i;
    for (int i = 0; i < m; ++i) {
      int b = i;
      for (int j = i + 1; j < m; ++j)
        if (lam[perm[j]] < lam[perm[b]]) b = j;
      const int t = perm[i];
      perm[i] = perm[b];
      perm[b] = t;
    }
    for (int i = 0; i < m; ++i) lam_s[i] = lam[perm[i]];
    ctl->lam1 = lam[perm[0]];
    ctl->lam2 = m > 1 ? lam[perm[1]] : INFINITY;
    ctl->smax = 0ull;
    ctl->argmin = 0x7fffffff;
    ctl->n_c = 0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int j = idx / m, a = idx % m;
    W_s[idx] = V[(int64_t)perm[j] * n + a];
  }
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
        double z0 = 0.0, z1 = 0.0;
        const int j0 = lane, j1 = lane + 32;
        if (j0 < m)
          for (int a = 0; a < m; ++a) z0 = fma(W[j0 * m + a], rb[a], z0);
        if (j1 < m)
          for (int a = 0; a < m; ++a) z1 = fma(W[j1 * m + a], rb[a], z1);
        const double q0 = z0 * z0, q1 = z1 * z1;
        const double zz = warp_sum(q0 + q1);
        if (m == 1) {
          sc = l1 + __shfl_sync(0xffffffffu, q0, 0);
        } else {
          double lo = l1, hi = fmin(l2, l1 + zz);
          for (int itr = 0; itr < 2000; ++itr) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            double f = 0.0;
            if (j0 < m) f = q0 / (lam[j0] - mid);
            if (j1 < m) f = f + q1 / (lam[j1] - mid);
            f = 1.0 + warp_sum(f);
            if (f < 0.0)
              lo = mid;
            else
              hi = mid;
          }
          sc = hi;
        }
        best = sc > best ? sc : best;
      }
      __syncwarp();
    }
    if (lane == 0) scores[pos] = sc;
  }
  best = block_max(best);
  if (threadIdx.x == 0) atomicMax(&ctl->smax, dbits(best));
}

__global__ void k_odeim_plan(OdCtl* ctl, const unsigned int* __restrict__ bmax,
                             const int* __restrict__ bstart, int probe_end, double tie_tol) {
  const double lim = bitsd(ctl->smax) * (1.0 - 2.0 * tie_tol);
  const double tau = (lim - ctl->lam1) / (1.0 + 1e-5);
  int blast = -1;
  for (int b = 0; b < kNB; ++b)
    if (bstart[b + 1] > bstart[b] && (double)__uint_as_float(bmax[b]) >= tau) blast = b;
  int n = blast >= 0 ? bstart[blast + 1] : 0;
  ctl->n_c = n > probe_end ? n : probe_end;
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
  OdCtl* ctl;
};

size_t odeim_ws_bytes(int64_t N, int m) {
  size_t b = 0;
  b += N * sizeof(float) + N + N + N * sizeof(int) + N * sizeof(double);
  b += (3 * (kNB + 1) + kNB) * sizeof(int);
  b += sizeof(double) * (64 + 6 * (size_t)(m + 1) * (m + 1) + 4 * m + 64);
  b += 16 * 256;
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
  return o;
}

template <typename T>
void launch_odeim(const T* phi, int64_t N, int m, int np, double tie_tol, int* pts, void* ws,
                  cudaStream_t s) {
  if (m <= 0) return;
  if (np > N) np = (int)N;
  OdeimBufs o = carve(ws, N, m);
  cudaMemsetAsync(o.picked, 0, N, s);
  cudaMemsetAsync(o.bcnt, 0, (kNB + 1) * sizeof(int), s);
  cudaMemsetAsync(o.bmax, 0, kNB * sizeof(int), s);
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_rownorm<T><<<(int)blocks, 256, 0, HY_S(s)>>>(phi, N, m, o.nrm, o.bkt, o.bcnt, o.bmax);
  k_bucket_scan<<<1, 32, 0, HY_S(s)>>>(o.bcnt, o.bstart, o.bcur);
  k_bucket_scatter<<<(int)blocks, 256, 0, HY_S(s)>>>(N, o.bkt, o.bcur, o.ord);
  const int probe = (int)(N < kProbe ? N : kProbe);
  // DEIM
  for (int l = 0; l < m; ++l) {
    k_deim_solve<T><<<1, 256, 0, HY_S(s)>>>(phi, N, l, pts, o.cvec, o.ctl);
    k_deim_score<T><<<(probe + 255) / 256, 256, 0, HY_S(s)>>>(phi, N, l, o.cvec, o.ord, o.picked, 0,
                                                        probe, o.ctl, o.scores);
    k_deim_plan<<<1, 1, 0, HY_S(s)>>>(o.ctl, o.bmax, o.bstart, probe, tie_tol);
    k_deim_score<T><<<152 * 8, 256, 0, HY_S(s)>>>(phi, N, l, o.cvec, o.ord, o.picked, probe, -1,
                                            o.ctl, o.scores);
    k_argmin_tie<<<152 * 4, 256, 0, HY_S(s)>>>(o.scores, o.ord, o.ctl, tie_tol);
    k_commit<<<1, 1, 0, HY_S(s)>>>(o.ctl, l, pts, o.picked);
  }
  if (np <= m) return;
  // ODEIM oversampling
  const int n = m % 2 ? m + 1 : m;  // Jacobi wants an even order
  k_odeim_gram<T><<<1, 256, 0, HY_S(s)>>>(phi, N, m, pts, m, o.M);
  const size_t smem = sizeof(double) * ((size_t)m * m + 64 + 64 * 8);
  cudaFuncSetAttribute(k_odeim_score<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int l = m; l < np; ++l) {
    launch_jacobi_padded(o.M, m, n, o.V, o.lam, o.Mp, s);
    k_odeim_sort<<<1, 256, 0, HY_S(s)>>>(o.lam, o.V, n, m, o.lam_s, o.W_s, o.ctl);
    k_odeim_score<T><<<(probe + 7) / 8, 256, smem, HY_S(s)>>>(phi, N, m, o.lam_s, o.W_s, o.ord,
                                                        o.picked, 0, probe, 0, tie_tol, o.ctl,
                                                        o.scores);
    k_odeim_plan<<<1, 1, 0, HY_S(s)>>>(o.ctl, o.bmax, o.bstart, probe, tie_tol);
    k_odeim_score<T><<<152 * 8, 256, smem, HY_S(s)>>>(phi, N, m, o.lam_s, o.W_s, o.ord, o.picked,
                                                probe, -1, 1, tie_tol, o.ctl, o.scores);
    k_argmin_tie<<<152 * 4, 256, 0, HY_S(s)>>>(o.scores, o.ord, o.ctl, tie_tol);
    k_commit<<<1, 1, 0, HY_S(s)>>>(o.ctl, l, pts, o.picked);
    k_odeim_rank1<T><<<1, 256, 0, HY_S(s)>>>(phi, N, m, o.ctl, o.M);
  }
}

template void launch_odeim<float>(const float*, int64_t, int, int, double, int*, void*,
                                  cudaStream_t);
template void launch_odeim<double>(const double*, int64_t, int, int, double, int*, void*,
                                   cudaStream_t);

}  // namespace hy
