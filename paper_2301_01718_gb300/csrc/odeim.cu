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
constexpr int kLdw = 65;       // odd leading dimension of W in shared memory
constexpr int kCompact = 524288;  // leading ordered rows kept row-major (FP32, 64 wide)

struct OdCtl {
  unsigned long long smax;  // bits of the best score so far (>= 0)
  int argmin;               // winning row (lowest index within the tie window)
  int n_c;                  // ordered rows to score
  double cn2;               // 1 + |c|^2            (DEIM)
  double lam1, lam2, lmax;  // eigenvalues of M (ODEIM)
  int n_list;                // rows passed on by the z_1 filter (ODEIM)
  int eig_sweeps;            // Jacobi sweeps of the first eigensystem (ODEIM)
  unsigned long long ubest;  // packed (upper bound bits, position) (ODEIM)
  // counters over one ODEIM call: DEIM rows scored, ODEIM rows given the
  // full FP32 bound, ODEIM exact scores, greedy steps
  unsigned long long stat[4];
};

size_t odeim_ctl_bytes() { return 256; }

// counters of the last ODEIM call (the control block heads the workspace)
void odeim_stats(const void* ws, unsigned long long* out4, cudaStream_t s) {
  const OdCtl* c = (const OdCtl*)ws;
  cudaMemcpyAsync(out4, c->stat, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
}

// Jacobi sweeps of the last ODEIM call's first eigensystem
void odeim_eig_sweeps(const void* ws, int* out, cudaStream_t s) {
  const OdCtl* c = (const OdCtl*)ws;
  cudaMemcpyAsync(out, &c->eig_sweeps, sizeof(int), cudaMemcpyDeviceToHost, s);
}

// ---- row norms and buckets --------------------------------------------------

static_assert(kNB == kNormBuckets, "row-norm buckets");

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
// Rows ord[0 .. C) of Phi copied once per call into a row-major FP32 array
// R (64 values per row, zero beyond m), so that the per-step scoring passes
// read each candidate row as 256 contiguous bytes instead of m scattered
// sectors of the column-major basis.  One warp per row.
template <typename T>
__global__ void k_gather_rows(const T* __restrict__ phi, int64_t N, int m,
                              const int* __restrict__ ord, int C, float* __restrict__ R) {
  const int lane = threadIdx.x & 31;
  for (int pos = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pos < C;
       pos += gridDim.x * (blockDim.x >> 5)) {
    const int i = ord[pos];
    const float x0 = lane < m ? (float)phi[(int64_t)lane * N + i] : 0.f;
    const float x1 = lane + 32 < m ? (float)phi[(int64_t)(lane + 32) * N + i] : 0.f;
    R[(int64_t)pos * 64 + lane] = x0;
    R[(int64_t)pos * 64 + lane + 32] = x1;
  }
}

template <typename T>
__global__ void k_deim_solve(const T* __restrict__ phi, int64_t N, int l,
                             const int* __restrict__ pts, const double* __restrict__ Lf,
                             const double* __restrict__ Uf, double* __restrict__ yv,
                             double* __restrict__ cvec, OdCtl* ctl) {
  pdl_enter();
  // L and U transposed into shared memory (stride 65: conflict-free), so
  // that both solves run column by column: after x_i is known every lane
  // updates its two right-hand-side entries (j = lane, lane + 32).
  extern __shared__ double dsm[];
  double* Lt = dsm;            // Lt[i * 65 + j] = L[j][i]
  double* Ut = dsm + 64 * 65;  // Ut[i * 65 + j] = U[j][i]
  // all threads stage (8 loads in flight each); warp 0 solves
  for (int base = threadIdx.x; base < l * l; base += blockDim.x * 8) {
    double lv[8], uv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      const int rr = idx / (l > 0 ? l : 1), cc = idx - rr * l;
      lv[u] = idx < l * l ? Lf[rr * 64 + cc] : 0.0;
      uv[u] = idx < l * l ? Uf[rr * 64 + cc] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < l * l) {
        const int rr = idx / l, cc = idx - rr * l;
        Lt[cc * 65 + rr] = lv[u];
        Ut[cc * 65 + rr] = uv[u];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double b0 = 0.0, b1 = 0.0;  // right-hand side, entries lane and lane + 32
  if (lane < l) b0 = (double)phi[(int64_t)l * N + pts[lane]];
  if (lane + 32 < l) b1 = (double)phi[(int64_t)l * N + pts[lane + 32]];
  __syncwarp();
  // forward: L y = b (unit diagonal)
  for (int i = 0; i < l; ++i) {
    const double yi = __shfl_sync(0xffffffffu, i < 32 ? b0 : b1, i & 31);
    const double* col = Lt + i * 65;
    if (lane > i && lane < l) b0 = fma(-col[lane], yi, b0);
    if (lane + 32 > i && lane + 32 < l) b1 = fma(-col[lane + 32], yi, b1);
  }
  const double y0 = b0, y1 = b1;
  // backward: U c = y, with the reciprocals of U's diagonal formed up front
  // (a division on every step of the dependent chain costs ~650 cycles)
  const double iu0 = lane < l ? 1.0 / Ut[lane * 65 + lane] : 0.0;
  const double iu1 = lane + 32 < l ? 1.0 / Ut[(lane + 32) * 65 + lane + 32] : 0.0;
  for (int i = l - 1; i >= 0; --i) {
    const double ci = __shfl_sync(0xffffffffu, i < 32 ? b0 : b1, i & 31) *
                      __shfl_sync(0xffffffffu, i < 32 ? iu0 : iu1, i & 31);
    if (lane == (i & 31)) {
      if (i < 32)
        b0 = ci;
      else
        b1 = ci;
    }
    const double* col = Ut + i * 65;
    if (lane < i) b0 = fma(-col[lane], ci, b0);
    if (lane + 32 < i) b1 = fma(-col[lane + 32], ci, b1);
  }
  double cn = 0.0;
  if (lane < l) {
    cvec[lane] = b0;
    yv[lane] = y0;
    cn = b0 * b0;
  }
  if (lane + 32 < l) {
    cvec[lane + 32] = b1;
    yv[lane + 32] = y1;
    cn = fma(b1, b1, cn);
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
  pdl_enter();
  // column-oriented solve of U^T ell = a with U^T's columns = U's rows
  __shared__ double Us[64 * 64];
  const int p = ctl->argmin;
  stage_copy(Us, Uf, l * 64);  // rows 0..l-1 (stride 64)
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double a0 = 0.0, a1 = 0.0;
  if (lane < l) a0 = (double)phi[(int64_t)lane * N + p];
  if (lane + 32 < l) a1 = (double)phi[(int64_t)(lane + 32) * N + p];
  const double pl = (double)phi[(int64_t)l * N + p];
  __syncwarp();
  const double iu0 = lane < l ? 1.0 / Us[lane * 64 + lane] : 0.0;
  const double iu1 = lane + 32 < l ? 1.0 / Us[(lane + 32) * 64 + lane + 32] : 0.0;
  for (int j = 0; j < l; ++j) {  // ell_j = (a_j - sum_{i<j} U_ij ell_i) / U_jj
    const double ej = __shfl_sync(0xffffffffu, j < 32 ? a0 : a1, j & 31) *
                      __shfl_sync(0xffffffffu, j < 32 ? iu0 : iu1, j & 31);
    if (lane == (j & 31)) {
      if (j < 32)
        a0 = ej;
      else
        a1 = ej;
    }
    const double* row = Us + j * 64;
    if (lane > j && lane < l) a0 = fma(-row[lane], ej, a0);
    if (lane + 32 > j && lane + 32 < l) a1 = fma(-row[lane + 32], ej, a1);
  }
  double dot = 0.0;
  if (lane < l) {
    Lf[l * 64 + lane] = a0;
    Uf[lane * 64 + l] = yv[lane];
    dot = a0 * yv[lane];
  }
  if (lane + 32 < l) {
    Lf[l * 64 + lane + 32] = a1;
    Uf[(lane + 32) * 64 + l] = yv[lane + 32];
    dot = fma(a1, yv[lane + 32], dot);
  }
  dot = warp_sum(dot);
  if (lane == 0) {
    Lf[l * 64 + l] = 1.0;
    Uf[l * 64 + l] = pl - dot;
  }
}

// exact |r_i| for the ordered rows [p0, p1) (p1 < 0: up to ctl->n_c)
template <typename T>
__global__ void k_deim_score(const T* __restrict__ phi, int64_t N, int l,
                             const double* __restrict__ cvec, const int* __restrict__ ord,
                             const unsigned char* __restrict__ picked, int p0, int p1,
                             OdCtl* ctl, double* __restrict__ scores, const float* __restrict__ R,
                             int C) {
  pdl_enter();
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
      double s4[4] = {0.0, 0.0, 0.0, 0.0};  // four chains
      if (sizeof(T) == 4 && pos < C) {  // the copy holds the FP32 values exactly
        const float* rr = R + (int64_t)pos * 64;
        for (int j = 0; j < l; ++j) s4[j & 3] = fma((double)rr[j], cs[j], s4[j & 3]);
        sc = fabs((double)rr[l] - ((s4[0] + s4[1]) + (s4[2] + s4[3])));
      } else {
        for (int j = 0; j < l; ++j)
          s4[j & 3] = fma((double)phi[(int64_t)j * N + i], cs[j], s4[j & 3]);
        sc = fabs((double)phi[(int64_t)l * N + i] - ((s4[0] + s4[1]) + (s4[2] + s4[3])));
      }
      best = sc > best ? sc : best;
    }
    scores[pos] = sc;
  }
  best = block_max(best);
  if (threadIdx.x == 0) atomicMax(&ctl->smax, dbits(best));
}

// one thread per bucket: the last non-empty bucket whose largest squared
// norm reaches tau bounds the rows still to score
__device__ void plan_rows(OdCtl* ctl, const unsigned int* __restrict__ bmax,
                          const int* __restrict__ bstart, int probe_end, double tau) {
  int blast = -1;
  for (int b = threadIdx.x; b < kNB; b += blockDim.x)
    if (bstart[b + 1] > bstart[b] && (double)__uint_as_float(bmax[b]) >= tau) blast = b;
  __shared__ int red[32];
  for (int o = 16; o > 0; o >>= 1) blast = max(blast, __shfl_xor_sync(0xffffffffu, blast, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = blast;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) blast = max(blast, red[w]);
    blast = max(blast, red[0]);
    const int n = blast >= 0 ? bstart[blast + 1] : 0;
    ctl->n_c = n > probe_end ? n : probe_end;
  }
}

// DEIM: |r_i| <= |phi_i| sqrt(1 + |c|^2), so rows need |phi_i|^2 >= lim^2 / cn2
__global__ void k_deim_plan(OdCtl* ctl, const unsigned int* __restrict__ bmax,
                            const int* __restrict__ bstart, int probe_end, double tie_tol) {
  pdl_enter();
  const double s = bitsd(ctl->smax);
  const double lim = s * (1.0 - 2.0 * tie_tol);
  plan_rows(ctl, bmax, bstart, probe_end, lim * lim / (ctl->cn2 * (1.0 + 1e-5)));
  if (threadIdx.x == 0) ctl->stat[0] += (unsigned long long)(ctl->n_c - probe_end);
}

// lowest row among the scored rows within the tie window of the best
__global__ void k_argmin_tie(const double* __restrict__ scores, const int* __restrict__ ord,
                             OdCtl* ctl, double tie_tol) {
  pdl_enter();
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
  pdl_enter();
  const int p = ctl->argmin;
  pts[l] = p;
  picked[p] = 1;
}

// ---- ODEIM oversampling -----------------------------------------------------

// M = A^T A over the first l points (m x m, FP64)
template <typename T>
__global__ void __launch_bounds__(256) k_odeim_gram(const T* __restrict__ phi, int64_t N, int m,
                                                    const int* __restrict__ pts, int l,
                                                    double* __restrict__ M) {
  // M = A^T A, A = the l sampled rows of Phi (l x m): every CTA stages A in
  // shared memory (eight loads in flight per thread), CTA c forms the rows
  // a = c, c + G, ... of M, one entry per thread, four chains over the l
  // terms (fma(x, y) = fma(y, x), so M is exactly symmetric)
  __shared__ double A[64][65];
  const int tid = threadIdx.x;
  for (int base = tid; base < l * m; base += blockDim.x * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      const int r = idx / m, a = idx - r * m;
      v[u] = idx < l * m ? (double)phi[(int64_t)a * N + pts[r]] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < l * m) A[idx / m][idx % m] = v[u];
    }
  }
  __syncthreads();
  for (int e = tid; e < 4 * 64; e += blockDim.x) {
    const int a = blockIdx.x + gridDim.x * (e >> 6), b = e & 63;
    if (a >= m || b >= m) continue;
    double p4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r = 0; r < l; ++r) p4[r & 3] = fma(A[r][a], A[r][b], p4[r & 3]);
    M[a * m + b] = (p4[0] + p4[1]) + (p4[2] + p4[3]);
  }
}

// sort the Jacobi eigenpairs ascending: lam_s, W_s (m x m column-major);
// reset the step's control block
// The screens read the eigensystem in FP32, written once per step where it
// changes: wt32[a * 64 + j] = W_ja (zero for j >= m), then dn[64] and du[64]
// at wt32 + 4096: d_j = lam_j - lam_1 (sorted) rounded to nearest and upward
// for 1 <= j < m, +inf otherwise (slot 0 carries z_1 itself).  One CTA.
HY_DEV void w32_tail(const double* __restrict__ lam_sorted, int m, float* __restrict__ wt32) {
  for (int idx = threadIdx.x; idx < m * (64 - m); idx += blockDim.x) {
    const int a = idx / (64 - m), j = m + idx % (64 - m);
    wt32[a * 64 + j] = 0.f;
  }
  float* dn = wt32 + 64 * 64;
  float* du = dn + 64;
  const double l1 = lam_sorted[0];
  for (int j = threadIdx.x; j < 64; j += blockDim.x) {
    if (j >= 1 && j < m) {
      dn[j] = (float)(lam_sorted[j] - l1);
      du[j] = __double2float_ru(__dsub_ru(lam_sorted[j], l1));
    } else {
      dn[j] = INFINITY;
      du[j] = INFINITY;
    }
  }
}

__global__ void k_odeim_sort(const double* __restrict__ lam, const double* __restrict__ V, int n,
                             int m, double* __restrict__ lam_s, double* __restrict__ W_s,
                             OdCtl* ctl, float* __restrict__ wt32) {
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
    ctl->n_list = 0;
    ctl->ubest = 0ull;
    ctl->argmin = 0x7fffffff;
    ctl->n_c = 0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int j = idx / m, a = idx % m;
    const double v = V[(int64_t)perm[j] * n + a];
    W_s[idx] = v;
    wt32[a * 64 + j] = (float)v;
  }
  w32_tail(lam_s, m, wt32);
}

// Smallest root of 1 + sum_j z_j^2 / (lam_j - mu) (lam ascending): with
// mu = l1 + tau and d_j = lam_j - l1 it is the root in (0, min(d_2, |z|^2)] of
//   h(tau) = tau (1 + g(tau)) - z_1^2,   g(tau) = sum_{j>=2} z_j^2 / (d_j - tau),
// which is increasing and has no pole at tau = 0 (the secular equation
// multiplied by tau).  Each step solves the two-pole model of the secular
// equation: the pole at 0 exactly, and g replaced by a + b / (d_2 - tau)
// with a and b matching g and g' at the current iterate (the "middle way"
// of Li's secular-equation solver, as in LAPACK's dlaed4); the model's
// smaller root is
//   tau' = 2 z_1^2 d_2 / (B + sqrt(B^2 - 4 C z_1^2 d_2)),
//   C = 1 + a,  B = C d_2 + z_1^2 + b.
// These steps run in FP32 (an FP64 divide or square root costs ~650
// cycles on this GPU, an FP32 reciprocal ~85), from tau = 0 until the step is
// at FP32 rounding; FP64 Newton steps on h then finish inside a shrinking
// bracket (bisection otherwise).  Stop when |h| is within the rounding error
// of its evaluation, the step is below 2 ulp, or the bracket has collapsed.  One warp; z in shared
// memory (lane j takes z_j and z_{j+32}).
__device__ double secular_root_warp(const double* __restrict__ z, const double* __restrict__ lam,
                                    int m, double l1, double l2) {
  const int lane = threadIdx.x & 31;
  const int j0 = lane, j1 = lane + 32;
  const double z0 = j0 < m ? z[j0] : 0.0, z1 = j1 < m ? z[j1] : 0.0;
  const double q0 = z0 * z0, q1 = z1 * z1;
  const double zz = warp_sum(q0 + q1);
  const double zf = __shfl_sync(0xffffffffu, q0, 0);  // z_1^2
  if (m == 1) return l1 + zf;
  // shifted poles of the other terms (lane 0's first slot is the pole itself)
  const double d0 = lam[j0 < m ? j0 : 0] - l1, d1 = j1 < m ? lam[j1] - l1 : 0.0;
  const double w0 = (j0 >= 1 && j0 < m) ? q0 : 0.0, w1 = j1 < m ? q1 : 0.0;
  const double d2 = l2 - l1;
  double hi = fmin(d2, zz), lo = 0.0;
  if (!(hi > 0.0) || zf == 0.0) return l1;  // z_1 = 0 or a double eigenvalue
  const double eps = 2.220446049250313e-16;
  // FP32 two-pole model steps (cheap) to a starting point for FP64 Newton
  double tau;
  {
    const float fd0 = (float)d0, fd1 = (float)d1, fw0 = (float)w0, fw1 = (float)w1;
    const float fzf = (float)zf, fd2 = (float)d2;
    float t = 0.f, flo = 0.f, fhi = (float)hi;
    for (int it = 0; it < 12; ++it) {
      float g = 0.f, dg = 0.f;
      if (fw0 > 0.f) {
        const float r = __frcp_rn(fd0 - t);
        g = fw0 * r;
        dg = g * r;
      }
      if (fw1 > 0.f) {
        const float r = __frcp_rn(fd1 - t);
        const float q = fw1 * r;
        g += q;
        dg = fmaf(q, r, dg);
      }
      g = warp_sum(g);
      dg = warp_sum(dg);
      if (it > 0) {
        const float h = fmaf(t, 1.f + g, -fzf);
        if (h < 0.f)
          flo = t;
        else
          fhi = t;
      }
      const float gap = fd2 - t;
      const float C = 1.f + (g - dg * gap);
      const float B = C * fd2 + fzf + dg * gap * gap;
      const float nt = 2.f * fzf * fd2 / (B + sqrtf(fmaxf(B * B - 4.f * C * fzf * fd2, 0.f)));
      const bool done = it > 0 && fabsf(nt - t) <= 4.f * 1.1920929e-7f * t;
      t = (nt > flo && nt < fhi) ? nt : 0.5f * (flo + fhi);
      if (done) break;
    }
    tau = (double)t;
    if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
  }
  // FP64 Newton steps on h inside the bracket
  for (int itr = 0; itr < 60; ++itr) {
    double g = 0.0, dg = 0.0;
    if (w0 > 0.0) {
      const double r = rcp64(d0 - tau);
      g = w0 * r;
      dg = g * r;
    }
    if (w1 > 0.0) {
      const double r = rcp64(d1 - tau);
      const double q = w1 * r;
      g = g + q;
      dg = fma(q, r, dg);
    }
    g = warp_sum(g);
    dg = warp_sum(dg);
    const double h = tau * (1.0 + g) - zf;
    if (fabs(h) <= 16.0 * eps * (tau * (1.0 + g) + zf)) break;
    if (h < 0.0)
      lo = tau;
    else
      hi = tau;
    if (hi - lo <= 2.0 * eps * hi) {
      tau = hi;
      break;
    }
    const double nt = tau - h / fma(tau, dg, 1.0 + g);
    if (fabs(nt - tau) <= 2.0 * eps * tau) {
      tau = nt;
      break;
    }
    tau = (nt > lo && nt < hi) ? nt : 0.5 * (lo + hi);
  }
  return l1 + tau;
}

// z = W^T rb for the m x m eigenvector block W (column j at W + j ldw) by the
// whole CTA (blockDim a multiple of 64): thread t forms component t % 64 over
// one of blockDim / 64 contiguous parts of the m terms (four chains), the
// parts are then added in a fixed order.  A warp-wide FP64 instruction
// occupies an SM sub-partition for 64 cycles, so the 64 x 64 product is
// spread over all the CTA's warps.  Synchronises the CTA on entry and exit.
HY_DEV void z_block(const double* W, int ldw, const double* rb, int m, double* zp, double* z) {
  const int t = threadIdx.x, j = t & 63, h = t >> 6, parts = blockDim.x >> 6;
  const int len = (m + parts - 1) / parts;
  const int a0 = h * len, a1 = a0 + len < m ? a0 + len : m;
  __syncthreads();
  double p[4] = {0.0, 0.0, 0.0, 0.0};
  if (j < m) {
    const double* w = W + j * ldw;
    int a = a0;
    for (; a + 3 < a1; a += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) p[u] = fma(w[a + u], rb[a + u], p[u]);
    }
    for (; a < a1; ++a) p[0] = fma(w[a], rb[a], p[0]);
  }
  zp[h * 64 + j] = (p[0] + p[1]) + (p[2] + p[3]);
  __syncthreads();
  if (t < 64) {
    double sm = 0.0;
    for (int q = 0; q < parts; ++q) sm += zp[q * 64 + t];
    z[t] = t < m ? sm : 0.0;
  }
  __syncthreads();
}

// ---- ODEIM scoring: certified FP32 bounds, then exact FP64 scores ---------
//
// With z = W^T phi, d_j = l_j - l1 and mu = l1 + tau, tau is the root in
// [0, d_2) of the increasing function
//   h(tau) = tau (1 + sum_{j>=2} z_j^2 / (d_j - tau)) - z_1^2,
// so tau <= z_1^2 and tau <= d_2 (interlacing).  FP32 dot products of m <= 64
// terms on operands rounded to FP32 are within dl = 8e-6 |phi| of the exact
// components ((m + 2) 2^-24 |W_j| |phi| = 3.9e-6 |phi|; the factor 2 covers
// the rounding of the stored norm), so with b1 = |z~_1| + dl and
// a_j = max(|z~_j| - dl, 0) the function
//   h_L(t) = t (1 + sum_{j>=2} a_j^2 / (d_j - t)) - b1^2  <=  h(t),
// and h_L(t) >= 0 proves tau <= t.  Every bound below is evaluated with
// directed rounding, so it stays an upper bound of the exact score.

// Stage 1, one thread per ordered row in [p0, ctl->n_c): the bound
// U1 = min(l1 + b1^2, l2) from z_1 alone (one m-term dot product).  Rows
// with U1 >= lim = smax (1 - 2 tie) are appended to `list` for stage 2.
template <typename T>
__global__ void __launch_bounds__(256) k_odeim_z1(
    const T* __restrict__ phi, int64_t N, int m, const double* __restrict__ W_s,
    const float* __restrict__ nrm, const int* __restrict__ ord,
    const unsigned char* __restrict__ picked, int p0, double tie_tol, OdCtl* ctl,
    double* __restrict__ scores, int* __restrict__ list, const float* __restrict__ R, int C) {
  pdl_enter();
  __shared__ float w1[64];
  for (int a = threadIdx.x; a < 64; a += blockDim.x) w1[a] = a < m ? (float)W_s[a] : 0.f;
  __syncthreads();
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  const double lim = bitsd(ctl->smax) * (1.0 - 2.0 * tie_tol);
  const int end = ctl->n_c;
  const int lane = threadIdx.x & 31;
  for (int base = p0 + blockIdx.x * blockDim.x; base < end; base += gridDim.x * blockDim.x) {
    const int pos = base + threadIdx.x;
    bool pass = false;
    if (pos < end) {
      const int i = ord[pos];
      double U = -1.0;
      if (!picked[i]) {
        float z1 = 0.f;
        if (pos < C) {  // contiguous copy (zero beyond m: same sum)
          const float4* rp = reinterpret_cast<const float4*>(R + (int64_t)pos * 64);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float4 v = rp[q];
            z1 = fmaf(w1[4 * q], v.x, z1);
            z1 = fmaf(w1[4 * q + 1], v.y, z1);
            z1 = fmaf(w1[4 * q + 2], v.z, z1);
            z1 = fmaf(w1[4 * q + 3], v.w, z1);
          }
        } else {
          for (int a = 0; a < 64; ++a)
            z1 = fmaf(w1[a], a < m ? (float)phi[(int64_t)a * N + i] : 0.f, z1);
        }
        const float dl = __fmul_ru(8e-6f, __fsqrt_ru(nrm[i]));
        const float b1 = __fadd_ru(fabsf(z1), dl);
        U = fmin(__dadd_ru(l1, (double)__fmul_ru(b1, b1)), l2);
        pass = U >= lim;
      }
      scores[pos] = U;
    }
    // warp-aggregated append
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    if (bal) {
      int first = 0;
      if (lane == 0) first = atomicAdd(&ctl->n_list, __popc(bal));
      first = __shfl_sync(0xffffffffu, first, 0);
      if (pass) list[first + __popc(bal & ((1u << lane) - 1u))] = pos;
    }
  }
}

// Stage 2, one warp per row (rows [p0, p1) of the order, or with list !=
// NULL the ctl->n_list positions in list): the bound from all m components,
// lane j holding z_j and z_{j+32}.  The root of h_L is approached with the
// two-pole model steps of secular_min_warp in FP32 (first step from t = 0)
// until |h_L| is at its rounding level; h_L(t') >= 0 is then checked, in
// directed rounding, at t' slightly above the iterate.  Rows whose check
// fails keep U = min(U1, l2).  The row with the largest bound is packed into
// ctl->ubest for the exact probe.
HY_DEV float warp_sum_rd(float v) {
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rd(v, __shfl_xor_sync(0xffffffffu, v, o));
  return __shfl_sync(0xffffffffu, v, 0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_odeim_screen(
    const T* __restrict__ phi, int64_t N, int m, const float* __restrict__ wt32,
    const float* __restrict__ nrm, const int* __restrict__ ord,
    const unsigned char* __restrict__ picked, int p0, int p1, const int* __restrict__ list,
    OdCtl* ctl, double* __restrict__ scores, const float* __restrict__ R, int C) {
  pdl_enter();
  __shared__ __align__(16) float Wt[64][64];  // Wt[a][j] = W_ja in FP32, zero padded
  __shared__ float dn[64], du[64];
  __shared__ float ph[8][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  {  // the step's FP32 eigensystem: rows a < m of Wt, then the shifts
    const float4* src = reinterpret_cast<const float4*>(wt32);
    float4* dst = reinterpret_cast<float4*>(&Wt[0][0]);
    for (int i = threadIdx.x; i < m * 16; i += blockDim.x) dst[i] = src[i];
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
      dn[j] = wt32[4096 + j];
      du[j] = wt32[4096 + 64 + j];
    }
  }
  __syncthreads();
  const float d2n = m > 1 ? dn[1] : INFINITY, d2u = m > 1 ? du[1] : INFINITY;
  const float dn0 = dn[lane], dn1 = dn[lane + 32], du0 = du[lane], du1 = du[lane + 32];
  const int count = list ? ctl->n_list : (p1 >= 0 ? p1 : ctl->n_c) - p0;
  float* pr = ph[wid];
  unsigned long long bestU = 0ull, cnt = 0;
  for (int t0 = blockIdx.x * nw + wid; t0 < count; t0 += gridDim.x * nw) {
    const int pos = list ? list[t0] : p0 + t0;
    const int i = ord[pos];
    if (picked[i]) {
      if (lane == 0) scores[pos] = -1.0;
      continue;
    }
    if (pos < C) {
      pr[lane] = R[(int64_t)pos * 64 + lane];
      pr[lane + 32] = R[(int64_t)pos * 64 + lane + 32];
    } else {
      pr[lane] = lane < m ? (float)phi[(int64_t)lane * N + i] : 0.f;
      pr[lane + 32] = lane + 32 < m ? (float)phi[(int64_t)(lane + 32) * N + i] : 0.f;
    }
    __syncwarp();
    float z0 = 0.f, z1 = 0.f;
#pragma unroll 8
    for (int a = 0; a < m; ++a) {
      const float x = pr[a];
      z0 = fmaf(Wt[a][lane], x, z0);
      z1 = fmaf(Wt[a][lane + 32], x, z1);
    }
    __syncwarp();
    const float dl = __fmul_ru(8e-6f, __fsqrt_ru(nrm[i]));
    const float zf = __shfl_sync(0xffffffffu, z0, 0);
    const float b1 = __fadd_ru(fabsf(zf), dl);
    const float b1s = __fmul_ru(b1, b1);
    // lower bounds of z_j^2 (j >= 2); lane 0's first slot is z_1 itself
    float a0 = lane == 0 ? 0.f : fmaxf(__fsub_rd(fabsf(z0), dl), 0.f);
    float a1 = fmaxf(__fsub_rd(fabsf(z1), dl), 0.f);
    a0 = __fmul_rd(a0, a0);
    a1 = __fmul_rd(a1, a1);
    double U = fmin(__dadd_ru(l1, (double)b1s), l2);
    if (m == 1 || !(d2n > 0.f)) {
      // U already exact up to rounding (m = 1) or the interlacing bound l2
    } else {
      float t = 0.f, lo = 0.f, hi = fminf(d2n, b1s);
      float g = warp_sum(a0 / dn0 + a1 / dn1);
      float dg = warp_sum(a0 / (dn0 * dn0) + a1 / (dn1 * dn1));
      for (int it = 0; it < 16; ++it) {
        if (it > 0) {
          const float r0 = __frcp_rn(dn0 - t), r1 = __frcp_rn(dn1 - t);
          const float q0 = a0 * r0, q1 = a1 * r1;
          g = warp_sum(q0 + q1);
          dg = warp_sum(fmaf(q0, r0, q1 * r1));
          const float h = fmaf(t, 1.f + g, -b1s);
          if (fabsf(h) <= 32.f * 1.1920929e-7f * (t * (1.f + g) + b1s)) break;
          if (h < 0.f)
            lo = t;
          else
            hi = t;
        }
        const float gap = d2n - t;
        const float C = 1.f + (g - dg * gap);
        const float B = C * d2n + b1s + dg * gap * gap;
        const float nt = 2.f * b1s * d2n / (B + sqrtf(fmaxf(B * B - 4.f * C * b1s * d2n, 0.f)));
        if (it > 0 && fabsf(nt - t) <= 4.f * 1.1920929e-7f * t) {
          t = nt;
          break;
        }
        t = (nt > lo && nt < hi) ? nt : 0.5f * (lo + hi);
      }
      // certify h_L(t') >= 0: t' 3e-5 above the iterate, else 5e-4
      for (int tr = 0; tr < 2; ++tr) {
        const float tu = __fmul_ru(t, tr == 0 ? 1.f + 1.0f / 32768.f : 1.f + 1.0f / 2048.f);
        if (!(tu < d2u)) break;
        const float S = warp_sum_rd(__fadd_rd(__fmul_rd(a0, __frcp_rd(__fsub_ru(du0, tu))),
                                              __fmul_rd(a1, __frcp_rd(__fsub_ru(du1, tu)))));
        const float hl = __fsub_rd(__fmul_rd(tu, __fadd_rd(1.f, S)), b1s);
        if (hl >= 0.f) {
          U = fmin(U, __dadd_ru(l1, (double)tu));
          break;
        }
      }
    }
    if (lane == 0) {
      scores[pos] = U;
      ++cnt;
      const unsigned long long kU =
          ((unsigned long long)(__double_as_longlong(U) >> 20) << 32) | (unsigned)pos;
      bestU = kU > bestU ? kU : bestU;
    }
  }
  if (lane == 0) {
    if (bestU) atomicMax(&ctl->ubest, bestU);
    if (cnt) atomicAdd(&ctl->stat[1], cnt);
  }
}

// stage a CTA's copy of W (m x m, column j = eigenvector j) with an odd
// leading dimension, and the eigenvalues
HY_DEV void stage_w(const double* __restrict__ W_s, const double* __restrict__ lam_s, int m,
                    double* W, double* lam) {
  for (int base = threadIdx.x; base < m * m; base += blockDim.x * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * blockDim.x;
      v[u] = i < m * m ? W_s[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * blockDim.x;
      if (i < m * m) {
        const int j = i / m, a = i - j * m;
        W[j * kLdw + a] = v[u];
      }
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = lam_s[i];
}

// exact score of the row with the largest screen bound -> raise smax to it
// (z by the whole CTA, the root by warp 0)
template <typename T>
__global__ void __launch_bounds__(256) k_odeim_probe_best(
    const T* __restrict__ phi, int64_t N, int m, const double* __restrict__ lam_s,
    const double* __restrict__ W_s, const int* __restrict__ ord, OdCtl* ctl) {
  pdl_enter();
  extern __shared__ double sh[];
  double* W = sh;               // 64 x kLdw
  double* lam = W + 64 * kLdw;  // 64
  double* rb = lam + 64;        // 64
  double* zp = rb + 64;         // 4 x 64
  double* zs = zp + 4 * 64;     // 64
  const unsigned long long key = ctl->ubest;
  if (!key) return;
  const int row = ord[(int)(key & 0xffffffffull)];
  stage_w(W_s, lam_s, m, W, lam);
  for (int i = threadIdx.x; i < m; i += blockDim.x) rb[i] = (double)phi[(int64_t)i * N + row];
  z_block(W, kLdw, rb, m, zp, zs);
  if (threadIdx.x < 32) {
    const double mu = secular_root_warp(zs, lam, m, ctl->lam1, ctl->lam2);
    if (threadIdx.x == 0) atomicMax(&ctl->smax, dbits(mu));
  }
}

// exact scores of the rows whose bound reaches smax (1 - 2 tie); the others
// get -1.  Only the probe positions [0, probe) and the ctl->n_list positions
// in `list` (the rows the z_1 bound passed to the full screen) can reach it:
// every other row keeps its z_1 bound, which is below the limit of that
// time and so below every later one.  One CTA of 128 threads per SM walks
// tiles of 128 of these, interleaved over the CTAs (entry c + G (128 k + t)
// for CTA c of G) because the rows that reach the limit are the largest-norm
// ones at the front of the order: the tile's rows that reach it are listed in shared
// memory, W is staged at the CTA's first such row, and the rows are scored
// four at a time — z by the whole CTA for each, then warp w solves the
// secular equation of the w-th row.  Before each group the limit is raised
// to the best exact score any CTA has found so far; rows whose bound no
// longer reaches it get -1 (they cannot reach the tie window of the best).
constexpr int kExactThreads = 128;
template <typename T>
__global__ void __launch_bounds__(kExactThreads) k_odeim_exact(
    const T* __restrict__ phi, int64_t N, int m, const double* __restrict__ lam_s,
    const double* __restrict__ W_s, const int* __restrict__ ord, int probe,
    const int* __restrict__ list, double tie_tol, OdCtl* ctl, double* __restrict__ scores) {
  pdl_enter();
  extern __shared__ double sh[];
  double* W = sh;               // 64 x kLdw
  double* lam = W + 64 * kLdw;  // 64
  double* rb = lam + 64;        // 4 x 64: rows of the group
  double* zp = rb + 4 * 64;     // 2 x 64
  double* zs = zp + 2 * 64;     // 4 x 64
  __shared__ int surv[kExactThreads];
  __shared__ int nlist;
  __shared__ int grp[4];  // the group's positions still to score (-1: none)
  __shared__ int ngrp;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  const double lim = bitsd(ctl->smax) * (1.0 - 2.0 * tie_tol);
  const int end = probe + ctl->n_list;  // entries: probe positions, then the list
  double best = 0.0;
  unsigned long long cnt = 0;
  bool staged = false;
  if (tid == 0) nlist = 0;
  __syncthreads();
  const int G = gridDim.x;
  for (int base = 0; (int)blockIdx.x + G * base < end; base += kExactThreads) {
    const int e = blockIdx.x + G * (base + tid);
    if (e < end) {
      const int pos = e < probe ? e : list[e - probe];
      const double U = scores[pos];
      if (U < lim) {
        if (U >= 0.0) scores[pos] = -1.0;
      } else {
        surv[atomicAdd(&nlist, 1)] = pos;
      }
    }
    __syncthreads();
    const int n = nlist;
    if (n > 0 && !staged) {
      stage_w(W_s, lam_s, m, W, lam);
      staged = true;
    }
    for (int g = 0; g < n; g += 4) {
      const int nq = n - g < 4 ? n - g : 4;
      if (tid == 0) {
        const double lnow =
            fmax(lim, bitsd(*(volatile unsigned long long*)&ctl->smax) * (1.0 - 2.0 * tie_tol));
        int k = 0;
        for (int q = 0; q < nq; ++q) {
          const int pos = surv[g + q];
          if (scores[pos] >= lnow)
            grp[k++] = pos;
          else
            scores[pos] = -1.0;
        }
        ngrp = k;
      }
      __syncthreads();
      const int ng = ngrp;
      for (int idx = tid; idx < ng * 64; idx += kExactThreads) {
        const int q = idx >> 6, a = idx & 63;
        rb[idx] = a < m ? (double)phi[(int64_t)a * N + ord[grp[q]]] : 0.0;
      }
      for (int q = 0; q < ng; ++q) z_block(W, kLdw, rb + 64 * q, m, zp, zs + 64 * q);
      if (wid < ng) {
        const double mu = secular_root_warp(zs + 64 * wid, lam, m, l1, l2);
        if (lane == 0) {
          scores[grp[wid]] = mu;
          atomicMax(&ctl->smax, dbits(mu));  // raises the limit of later groups
        }
        best = mu > best ? mu : best;
        ++cnt;
      }
      __syncthreads();
    }
    if (tid == 0) nlist = 0;
    __syncthreads();
  }
  best = block_max(best);
  if (tid == 0) atomicMax(&ctl->smax, dbits(best));
  if (lane == 0 && cnt) atomicAdd(&ctl->stat[2], cnt);
}

// ODEIM: mu - l1 <= z_1^2 <= |phi_i|^2, so rows need |phi_i|^2 >= lim - l1
__global__ void k_odeim_plan(OdCtl* ctl, const unsigned int* __restrict__ bmax,
                             const int* __restrict__ bstart, int probe_end, double tie_tol) {
  pdl_enter();
  if (threadIdx.x == 0) ctl->stat[3] += 1;
  const double lim = bitsd(ctl->smax) * (1.0 - 2.0 * tie_tol);
  plan_rows(ctl, bmax, bstart, probe_end, (lim - ctl->lam1) / (1.0 + 1e-5));
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
  double zh[64];   // Loewner z of the non-deflated components
};

template <typename T>
__global__ void k_r1_prepare(const T* __restrict__ phi, int64_t N, int m, const OdCtl* ctl,
                             const double* __restrict__ d, const double* __restrict__ W,
                             double* __restrict__ Wrot, R1Work* wk) {
  pdl_enter();
  __shared__ double Ws[64 * 64];
  __shared__ double ph[64], z[64], ds[64];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int p = ctl->argmin;
  for (int a = tid; a < m; a += blockDim.x) {
    ph[a] = (double)phi[(int64_t)a * N + p];
    ds[a] = d[a];
  }
  stage_copy(Ws, W, m * m);
  __shared__ double zp[4][64];
  {  // z = W^T phi: thread t forms component t % 64 over a quarter of the terms
    __syncthreads();
    const int j = tid & 63, h = tid >> 6;
    const int len = (m + 3) / 4, a0 = h * len, a1 = a0 + len < m ? a0 + len : m;
    double p0 = 0.0, p1 = 0.0;
    if (j < m && h < 4) {
      int a = a0;
      for (; a + 1 < a1; a += 2) {
        p0 = fma(Ws[j * m + a], ph[a], p0);
        p1 = fma(Ws[j * m + a + 1], ph[a + 1], p1);
      }
      if (a < a1) p0 = fma(Ws[j * m + a], ph[a], p0);
    }
    if (h < 4) zp[h][j] = p0 + p1;
    __syncthreads();
    if (tid < m) z[tid] = (zp[0][tid] + zp[1][tid]) + (zp[2][tid] + zp[3][tid]);
    __syncthreads();
  }
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
  if (tid < 64) {  // ordered list of the non-negligible z (two warps, ballots)
    const bool keep = tid < m && !(fabs(z[tid]) * nz <= tol);
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    __shared__ int wcnt[2];
    if (lane == 0) wcnt[wid] = __popc(b);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    const int off = (wid == 1 ? wcnt[0] : 0) + __popc(b & ((1u << lane) - 1u));
    if (keep) nonsmall[off] = tid;
    if (tid == 0) nns = wcnt[0] + wcnt[1];
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
// Root j lies in (d_j, d_{j+1}) (the last one in (d_n, d_n + |z|^2)); it is
// computed as tau in coordinates shifted to the nearer pole o, so that
// d_i - lambda_j = (d_i - d_o) - tau keeps full relative accuracy.  Each
// step solves the two-pole model of f(tau) = 1 + sum_i z_i^2 / (del_i - tau)
// (the "middle way" of Li's secular solver, as in LAPACK's dlaed4): with
// psi the terms with poles at or left of d_j and phi the rest,
//   f ~ c + s / (del_j - tau') + S / (del_{j+1} - tau'),
//   s = psi' (del_j - tau)^2, S = phi' (del_{j+1} - tau)^2,
//   c = f - psi' (del_j - tau) - phi' (del_{j+1} - tau),
// a quadratic in the correction whose root in the interval is taken
// (the last root has no right pole: tau' = del_n + s / c).  Steps are kept
// inside a shrinking bracket (bisection otherwise); the iteration stops once
// |f| is within the rounding error of its evaluation, the step is below
// 2 ulp, or the bracket has collapsed.
__global__ void k_r1_roots(R1Work* wk, double* __restrict__ Delta) {
  pdl_enter();
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
  const double rho = warp_sum(z2[0] + z2[1]);
  const double dj = wk->dK[j];
  const bool last = j == nK - 1;
  int o;
  double lo, hi;
  if (last) {
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
  const double delj = dj - dorg, deln = last ? 0.0 : wk->dK[j + 1] - dorg;
  double t = (o == j) ? 0.5 * hi : 0.5 * lo;
  const double eps = 2.220446049250313e-16;
  {  // the same model steps in FP32 (cheap) to a start for the FP64 ones,
     // which keep their own bracket
    const float fe = 1.1920929e-7f;
    float fdel[2], fz2[2];
    for (int u = 0; u < 2; ++u) {
      fdel[u] = (float)del[u];
      fz2[u] = (float)z2[u];
    }
    const float fdelj = (float)delj, fdeln = (float)deln;
    float ft = (float)t, flo = (float)lo, fhi = (float)hi;
    for (int it = 0; it < 16; ++it) {
      float f = 0.f, fa = 0.f, dps = 0.f, dph = 0.f;
      for (int u = 0; u < 2; ++u) {
        const int i = lane + 32 * u;
        if (i < nK) {
          const float r = __frcp_rn(fdel[u] - ft);
          const float q = fz2[u] * r;
          f += q;
          fa += fabsf(q);
          if (i <= j)
            dps = fmaf(q, r, dps);
          else
            dph = fmaf(q, r, dph);
        }
      }
      f = 1.f + warp_sum(f);
      fa = warp_sum(fa);
      dps = warp_sum(dps);
      dph = warp_sum(dph);
      if (fabsf(f) <= 8.f * fe * (1.f + fa + fabsf(ft) * (dps + dph))) break;
      if (f < 0.f)
        flo = ft;
      else
        fhi = ft;
      if (fhi - flo <= 2.f * fe * fmaxf(fabsf(fhi), fabsf(flo))) {
        ft = 0.5f * (flo + fhi);
        break;
      }
      const float Dj = fdelj - ft;
      float eta = NAN;
      if (last) {
        const float sL = dps * Dj * Dj, cq = f - dps * Dj;
        if (cq > 0.f) eta = Dj + sL / cq;
      } else {
        const float Dn = fdeln - ft;
        const float sL = dps * Dj * Dj, sR = dph * Dn * Dn;
        const float A = f - dps * Dj - dph * Dn;
        const float B = A * (Dj + Dn) + sL + sR;
        const float Cq = f * Dj * Dn;
        if (A == 0.f) {
          if (B != 0.f) eta = Cq / B;
        } else {
          const float qq = 0.5f * (B + copysignf(sqrtf(fmaxf(B * B - 4.f * A * Cq, 0.f)), B));
          const float e1 = qq / A, e2 = qq != 0.f ? Cq / qq : NAN;
          if (e1 > Dj && e1 < Dn) eta = e1;
          if (e2 > Dj && e2 < Dn) eta = e2;
        }
      }
      float nt = ft + eta;
      if (fabsf(nt - ft) <= 2.f * fe * fabsf(ft)) {
        ft = nt;
        break;
      }
      if (!(nt > flo && nt < fhi)) nt = 0.5f * (flo + fhi);
      ft = nt;
    }
    const double tc = (double)ft;
    if (tc > lo && tc < hi) t = tc;
  }
  for (int it = 0; it < 100; ++it) {
    double f = 0.0, fa = 0.0, dps = 0.0, dph = 0.0;
    for (int u = 0; u < 2; ++u) {
      const int i = lane + 32 * u;
      if (i < nK) {
        const double r = rcp64(del[u] - t);
        const double q = z2[u] * r;
        f = f + q;
        fa = fa + fabs(q);
        if (i <= j)
          dps = dps + q * r;
        else
          dph = dph + q * r;
      }
    }
    f = 1.0 + warp_sum(f);
    fa = warp_sum(fa);
    dps = warp_sum(dps);
    dph = warp_sum(dph);
    if (fabs(f) <= 8.0 * eps * (1.0 + fa + fabs(t) * (dps + dph))) break;
    if (f < 0.0)
      lo = t;
    else
      hi = t;
    if (hi - lo <= 2.0 * eps * fmax(fabs(hi), fabs(lo))) {
      t = 0.5 * (lo + hi);
      break;
    }
    const double Dj = delj - t;  // < 0
    double eta = NAN;
    if (last) {
      const double sL = dps * Dj * Dj, c = f - dps * Dj;
      if (c > 0.0) eta = Dj + sL / c;
    } else {
      const double Dn = deln - t;  // > 0
      const double sL = dps * Dj * Dj, sR = dph * Dn * Dn;
      const double A = f - dps * Dj - dph * Dn;
      const double B = A * (Dj + Dn) + sL + sR;
      const double Cq = f * Dj * Dn;
      // A eta^2 - B eta + Cq = 0: the root in (Dj, Dn)
      if (A == 0.0) {
        if (B != 0.0) eta = Cq / B;
      } else {
        const double q = 0.5 * (B + copysign(sqrt(fmax(B * B - 4.0 * A * Cq, 0.0)), B));
        const double e1 = q / A, e2 = q != 0.0 ? Cq / q : NAN;
        if (e1 > Dj && e1 < Dn) eta = e1;
        if (e2 > Dj && e2 < Dn) eta = e2;
      }
    }
    double nt = t + eta;
    if (fabs(nt - t) <= 2.0 * eps * fabs(t)) {  // before the bracket test: a
      t = nt;                                    // converged step may sit on it
      break;
    }
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    t = nt;
  }
  for (int u = 0; u < 2; ++u) {
    const int i = lane + 32 * u;
    if (i < nK) Delta[i * 64 + j] = del[u] - t;
  }
  if (lane == 0) {
    wk->org[j] = o;
    wk->tau[j] = t;
  }
}

// Loewner's z (Gu & Eisenstat): with Delta_iq = d_i - lambda_q,
//   zh_i^2 = (lambda_i - d_i) prod_{q != i} (lambda_q - d_i) / (d_q - d_i),
// signed like z_i.  One warp per component i (lane: q and q + 32), a product
// tree over the lanes.
__global__ void __launch_bounds__(128) k_r1_loewner(R1Work* wk, const double* __restrict__ Delta) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nK = wk->nK;
  if (i >= nK) return;
  const double di = wk->dK[i];
  double pr = 1.0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = lane + 32 * u;
    if (q < nK) {
      const double lq = -Delta[i * 64 + q];  // lambda_q - d_i
      pr *= q == i ? lq : lq * rcp64(wk->dK[q] - di);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pr *= __shfl_xor_sync(0xffffffffu, pr, o);
  if (lane == 0) {
    const double zz = sqrt(fmax(pr, 0.0));
    wk->zh[i] = wk->zK[i] >= 0.0 ? zz : -zz;
  }
}

// Eigenvector j of diag(dK) + z z^T, v_i = zh_i / (d_i - lambda_j), mapped
// back through W.  CTA j writes column j of Wnew (m values) and lamnew[j];
// the product with W is split over the CTA's eight warps (thread t: row
// a = t % 64 over a quarter of the components).
__global__ void __launch_bounds__(256) k_r1_vectors(const R1Work* __restrict__ wk,
                                                    const double* __restrict__ Delta,
                                                    const double* __restrict__ Wrot, int m,
                                                    double* __restrict__ Wnew,
                                                    double* __restrict__ lamnew) {
  pdl_enter();
  __shared__ double v[64];
  __shared__ double Wk[64 * 65];  // rows K[i] of Wrot, stride 65
  __shared__ double part[4][64];
  __shared__ int Ks[64];
  const int j = blockIdx.x, tid = threadIdx.x;
  const int nK = wk->nK;
  if (j >= nK) return;
  for (int i = tid; i < nK; i += blockDim.x) Ks[i] = wk->K[i];
  __syncthreads();
  for (int base = tid; base < nK * 64; base += blockDim.x * 8) {
    double wv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      const int i = idx >> 6, a = idx & 63;
      wv[u] = idx < nK * 64 && a < m ? Wrot[Ks[i] * m + a] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < nK * 64) Wk[(idx >> 6) * 65 + (idx & 63)] = wv[u];
    }
  }
  double vi = 0.0;
  if (tid < 64) {
    if (tid < nK) vi = wk->zh[tid] * rcp64(Delta[tid * 64 + j]);
    v[tid] = vi;
  }
  __syncthreads();
  double nrm = tid < 64 ? vi * vi : 0.0;
  nrm = block_sum(nrm);
  const double inv = 1.0 / sqrt(nrm);
  {
    const int a = tid & 63, h = tid >> 6;
    const int i0 = h * 16, i1 = i0 + 16 < nK ? i0 + 16 : nK;
    double acc0 = 0.0, acc1 = 0.0;
    int i = i0;
    for (; i + 1 < i1; i += 2) {
      acc0 = fma(Wk[i * 65 + a], v[i], acc0);
      acc1 = fma(Wk[(i + 1) * 65 + a], v[i + 1], acc1);
    }
    if (i < i1) acc0 = fma(Wk[i * 65 + a], v[i], acc0);
    part[h][a] = acc0 + acc1;
  }
  __syncthreads();
  if (tid < m) Wnew[j * m + tid] = ((part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid])) * inv;
  if (tid == 0) lamnew[j] = wk->dK[wk->org[j]] + wk->tau[j];
}

// Merge deflated and new eigenpairs, ascending; reset the step's control.
__global__ void k_r1_merge(const R1Work* __restrict__ wk, const double* __restrict__ Wrot,
                           const double* __restrict__ Wnew, const double* __restrict__ lamnew,
                           int m, double* __restrict__ d_out, double* __restrict__ W_out,
                           OdCtl* ctl, float* __restrict__ wt32) {
  pdl_enter();
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
    ctl->n_list = 0;
    ctl->ubest = 0ull;
    ctl->argmin = 0x7fffffff;
    ctl->n_c = 0;
  }
  (void)nD;
  for (int i = tid; i < m; i += blockDim.x) d_out[i] = lv[perm[i]];
  // eight loads in flight per thread before any store
  for (int base = tid; base < m * m; base += blockDim.x * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      v[u] = 0.0;
      if (idx < m * m) {
        const int j = idx / m, a = idx - j * m;
        const int sidx = src[perm[j]];
        v[u] = sidx >= 0 ? Wnew[sidx * m + a] : Wrot[(-sidx - 1) * m + a];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < m * m) {
        W_out[idx] = v[u];
        const int j = idx / m, a = idx - j * m;
        wt32[a * 64 + j] = (float)v[u];
      }
    }
  }
  __syncthreads();  // d_out complete
  w32_tail(d_out, m, wt32);
}

__global__ void k_pad_sym2(const double* __restrict__ M, int m, int n, double* __restrict__ P) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int a = idx / n, b = idx % n;
    P[idx] = (a < m && b < m) ? M[a * m + b] : 0.0;
  }
}

// ---- driver -----------------------------------------------------------------

struct OdeimBufs {
  int* list;
  float* rows;
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
  float* wt32;  // the step's eigensystem in FP32 for the screens (4096 + 128)
};

size_t odeim_ws_bytes(int64_t N, int m) {
  size_t b = 0;
  b += N * sizeof(float) + N + N + 2 * N * sizeof(int) + N * sizeof(double) + 256;
  b += (size_t)(N < kCompact ? N : kCompact) * 64 * sizeof(float) + 256;
  b += (3 * (kNB + 1) + kNB) * sizeof(int);
  b += sizeof(double) * (64 + 6 * (size_t)(m + 1) * (m + 1) + 4 * m + 64);
  b += 16 * 256;
  b += sizeof(double) * (5 * 64 * 64 + 3 * 64) + sizeof(R1Work) + 16 * 256;
  b += sizeof(double) * (2 * (m + 1) * (m + 1) + 512) + 3 * 256;
  b += sizeof(double) * (2 * 64 * 64 + 64) + 3 * 256;
  b += sizeof(float) * (64 * 64 + 128) + 256;
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
  o.list = (int*)take(N * sizeof(int));
  o.rows = (float*)take((size_t)(N < kCompact ? N : kCompact) * 64 * sizeof(float));
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
  o.jbuf = (double*)take(((size_t)2 * (m + 1) * (m + 1) + 512) * sizeof(double));
  o.jscale = (double*)take(64);
  o.jflag = (int*)take(64);
  o.Lf = (double*)take((size_t)64 * 64 * sizeof(double));
  o.Uf = (double*)take((size_t)64 * 64 * sizeof(double));
  o.yv = (double*)take(64 * sizeof(double));
  o.wt32 = (float*)take((64 * 64 + 128) * sizeof(float));
  return o;
}

OdeimNorms odeim_norm_bufs(void* ws, int64_t N) {
  const OdeimBufs o = carve(ws, N, 1);  // these buffers precede every m-dependent one
  return OdeimNorms{o.nrm, o.bkt, o.bcnt, o.bmax};
}

void odeim_graphs_free(OdeimGraphs* g) {
  graph_slot_free(&g->deim);
  graph_slot_free(&g->over);
  g->N = -1;
  g->m = g->np = -1;
}

// Launch with programmatic stream serialization (the kernel starts with
// pdl_enter(), which keeps stream order); where the attribute is refused,
// an ordinary launch.  The arguments are converted to the kernel's
// parameter types as in a triple-chevron launch.
template <typename... KArgs, typename... Args>
void pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
         Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  if (cudaLaunchKernelEx(&cfg, kern, args...) != cudaSuccess) {
    cudaGetLastError();
    cfg.numAttrs = 0;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  }
}

template <typename T>
int launch_odeim(const T* phi, int64_t N, int m, int np, double tie_tol, int* pts, void* ws,
                 void* host_pinned, cudaStream_t s, void (*mark)(void*, int), void* mark_arg,
                 bool norms_ready, OdeimGraphs* graphs) {
  if (m <= 0) return 0;
  if (np > N) np = (int)N;
  OdeimBufs o = carve(ws, N, m);
  if (graphs && (graphs->N != N || graphs->m != m || graphs->np != np)) {
    odeim_graphs_free(graphs);
    graphs->N = N;
    graphs->m = m;
    graphs->np = np;
  }
  auto M_ = [&](int id) {
    if (mark) mark(mark_arg, id);
  };
  M_(12);
  cudaMemsetAsync(o.ctl, 0, sizeof(OdCtl), s);
  cudaMemsetAsync(o.picked, 0, N, s);
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (!norms_ready) {  // else the basis product's epilogue formed them
    cudaMemsetAsync(o.bcnt, 0, (kNB + 1) * sizeof(int), s);
    cudaMemsetAsync(o.bmax, 0, kNB * sizeof(int), s);
    k_rownorm<T><<<(int)blocks, 256, 0, HY_S(s)>>>(phi, N, m, o.nrm, o.bkt, o.bcnt, o.bmax);
  }
  k_bucket_scan<<<1, 32, 0, HY_S(s)>>>(o.bcnt, o.bstart, o.bcur);
  k_bucket_scatter<<<(int)blocks, 256, 0, HY_S(s)>>>(N, o.bkt, o.bcur, o.ord);
  const int C = (int)(N < kCompact ? N : kCompact);
  if (m <= 64) {
    k_gather_rows<T><<<152 * 8, 256, 0, HY_S(s)>>>(phi, N, m, o.ord, C, o.rows);
  }
  const int probe = (int)(N < kProbe ? N : kProbe);
  M_(-13);
  // DEIM.  The kernels of both greedy loops start with pdl_enter() and are
  // launched with programmatic stream serialization (pdl()): each is
  // scheduled while its predecessor runs and waits for it on the device.
  const size_t dsmem = sizeof(double) * 2 * 64 * 65;
  smem_at_least((const void*)k_deim_solve<T>, dsmem);
  auto deim_loop = [&]() {
  for (int l = 0; l < m; ++l) {
    pdl(k_deim_solve<T>, 1, 256, dsmem, s, phi, N, l, pts, o.Lf, o.Uf, o.yv, o.cvec, o.ctl);
    pdl(k_deim_score<T>, (probe + 255) / 256, 256, 0, s, phi, N, l, o.cvec, o.ord, o.picked, 0,
        probe, o.ctl, o.scores, o.rows, C);
    pdl(k_deim_plan, 1, 256, 0, s, o.ctl, o.bmax, o.bstart, probe, tie_tol);
    pdl(k_deim_score<T>, 152 * 8, 256, 0, s, phi, N, l, o.cvec, o.ord, o.picked, probe, -1,
        o.ctl, o.scores, o.rows, C);
    pdl(k_argmin_tie, 152 * 4, 256, 0, s, o.scores, o.ord, o.ctl, tie_tol);
    pdl(k_commit, 1, 1, 0, s, o.ctl, l, pts, o.picked);
    if (l + 1 < m) pdl(k_deim_extend<T>, 1, 256, 0, s, phi, N, l, o.ctl, o.Lf, o.Uf, o.yv);
  }
  };
  if (graphs)
    run_graphed(&graphs->deim, s, deim_loop);
  else
    deim_loop();
  if (mark) {  // DEIM ends, oversampling begins
    mark(mark_arg, -12);
    mark(mark_arg, 9);
  }
  if (np <= m) return 0;
  // ODEIM oversampling
  const int n = m % 2 ? m + 1 : m;  // Jacobi wants an even order
  k_odeim_gram<T><<<(m + 3) / 4, 256, 0, HY_S(s)>>>(phi, N, m, pts, m, o.M);
  const size_t smem_pb = sizeof(double) * ((size_t)64 * kLdw + 64 + 64 + 4 * 64 + 64);
  const size_t smem_ex = sizeof(double) * ((size_t)64 * kLdw + 64 + 4 * 64 + 2 * 64 + 4 * 64);
  M_(12);
  // eigensystem of M: pivoted Cholesky + one-sided Jacobi; two-sided
  // Jacobi if M is numerically rank deficient (its null space is needed)
  int rank_m = 0;
  if (run_psd_eig(o.M, m, o.V, o.lam, o.jbuf, o.jflag, (int*)host_pinned, 60, s,
                  (int*)host_pinned + 2) < 0)
    return -1;
  rank_m = ((int*)host_pinned)[2];
  cudaMemcpyAsync(&o.ctl->eig_sweeps, o.jflag + 4, sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (rank_m == m) {
    k_odeim_sort<<<1, 256, 0, HY_S(s)>>>(o.lam, o.V, m, m, o.lam_s, o.W_s, o.ctl, o.wt32);
  } else {
    k_pad_sym2<<<1, 256, 0, HY_S(s)>>>(o.M, m, n, o.Mp);
    if (run_jacobi_multi(o.Mp, n, o.V, o.lam, o.jbuf, o.jflag, (int*)host_pinned, o.jscale,
                         (double*)host_pinned + 1, 60, s) < 0)
      return -1;
    k_odeim_sort<<<1, 256, 0, HY_S(s)>>>(o.lam, o.V, n, m, o.lam_s, o.W_s, o.ctl, o.wt32);
  }
  M_(-13);
  // sub-stage marks only where the loop is not replayed from a graph
  auto ML_ = [&](int id) {
    if (mark && !graphs) mark(mark_arg, id);
  };
  auto over_loop = [&]() {
  for (int l = m; l < np; ++l) {
    ML_(13);
    // full FP32 bounds of the largest-norm rows, exact score of the best
    pdl(k_odeim_screen<T>, (probe + 7) / 8, 256, 0, s, phi, N, m, o.wt32, o.nrm, o.ord, o.picked,
        0, probe, (const int*)nullptr, o.ctl, o.scores, o.rows, C);
    pdl(k_odeim_probe_best<T>, 1, 256, smem_pb, s, phi, N, m, o.lam_s, o.W_s, o.ord, o.ctl);
    pdl(k_odeim_plan, 1, 256, 0, s, o.ctl, o.bmax, o.bstart, probe, tie_tol);
    ML_(-14);
    ML_(14);
    // the other rows whose norm can reach the best score: the z_1 bound for
    // all, the full bound for those it does not exclude
    pdl(k_odeim_z1<T>, 152 * 8, 256, 0, s, phi, N, m, o.W_s, o.nrm, o.ord, o.picked, probe,
        tie_tol, o.ctl, o.scores, o.list, o.rows, C);
    pdl(k_odeim_screen<T>, 152 * 8, 256, 0, s, phi, N, m, o.wt32, o.nrm, o.ord, o.picked, 0, -1,
        (const int*)o.list, o.ctl, o.scores, o.rows, C);
    pdl(k_odeim_probe_best<T>, 1, 256, smem_pb, s, phi, N, m, o.lam_s, o.W_s, o.ord, o.ctl);
    ML_(-15);
    ML_(15);
    pdl(k_odeim_exact<T>, 152, kExactThreads, smem_ex, s, phi, N, m, o.lam_s, o.W_s, o.ord, probe,
        o.list, tie_tol, o.ctl, o.scores);
    ML_(-16);
    ML_(17);
    pdl(k_argmin_tie, 152 * 4, 256, 0, s, o.scores, o.ord, o.ctl, tie_tol);
    pdl(k_commit, 1, 1, 0, s, o.ctl, l, pts, o.picked);
    ML_(-18);
    if (l + 1 < np) {
      ML_(16);
      pdl(k_r1_prepare<T>, 1, 256, 0, s, phi, N, m, o.ctl, o.lam_s, o.W_s, o.Wrot, o.r1);
      pdl(k_r1_roots, m, 32, 0, s, o.r1, o.Delta);
      pdl(k_r1_loewner, (m + 3) / 4, 128, 0, s, o.r1, o.Delta);
      pdl(k_r1_vectors, m, 256, 0, s, o.r1, o.Delta, o.Wrot, m, o.Wnew, o.lamnew);
      pdl(k_r1_merge, 1, 256, 0, s, o.r1, o.Wrot, o.Wnew, o.lamnew, m, o.lam_s2, o.W_s2, o.ctl,
          o.wt32);
      std::swap(o.lam_s, o.lam_s2);
      std::swap(o.W_s, o.W_s2);
      ML_(-17);
    }
  }
  };
  if (graphs)
    run_graphed(&graphs->over, s, over_loop);
  else
    over_loop();
  return 0;
}

template int launch_odeim<float>(const float*, int64_t, int, int, double, int*, void*, void*,
                                 cudaStream_t, void (*)(void*, int), void*, bool, OdeimGraphs*);
template int launch_odeim<double>(const double*, int64_t, int, int, double, int*, void*, void*,
                                  cudaStream_t, void (*)(void*, int), void*, bool, OdeimGraphs*);

}  // namespace hy
