// Sample-row form of the reduced solve (Sec. 2.2, reduced coordinates, with
// every dof row of the sample cells S-hat as regression rows instead of the
// ODEIM rows P, which S-hat contains):
//   y = argmin || (Phi y - (v - psi))_S ||_2,
// solved through the normal equations
//   (Phi_S^T Phi_S) y = Phi_S^T (v - psi)_S.
// The m x m normal matrix is formed once per basis and sample set (at the
// rebuild) and Cholesky-factored in FP64; each solve forms the right-hand
// side (one pass over the sample rows of Phi, v and psi) and substitutes.
// Rows are variable-major: row r = (v, cell) with v = r / n_s and cell the
// (r % n_s)-th sample cell in ascending order.
//
// The normal matrix comes in four precisions (the reduced-precision form of
// the sample-row solve): FP32 products accumulated in FP32 within a CTA and
// in FP64 across CTAs (FP64 throughout for FP64 states), or on the tensor
// cores (reduced_tc.cu) TF32 or BF16 products, or FP32-level products of a
// TF32 hi/lo split, accumulated in FP32 within a CTA and in FP64 across.
// fail[0] = 1: a Cholesky pivot is not positive; fail[1] = 1: a bounded wait
// of the tensor-core kernel gave up.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace hy {
namespace {

constexpr int kRowsChunk = 64;  // rows staged per iteration
constexpr int kPad = 68;        // staged row stride (floats or doubles)

HY_DEV int64_t sample_dof(const int* __restrict__ cells, int ns, int64_t nc, int64_t r) {
  const int v = (int)(r / ns);
  return (int64_t)v * nc + cells[r - (int64_t)v * ns];
}

// CTA b accumulates the rows [b * rpc, (b + 1) * rpc): thread t owns the 4 x 4
// block (t / 16, t % 16) of the 64 x 64 matrix (columns >= m are zero).
// A: accumulator type (float for FP32 states, double for FP64).  FP64
// partials go to part[b * 64 * 64 ...].
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_sample_moments(
    const T* __restrict__ phi, int64_t N, int m, const int* __restrict__ cells, int ns, int nvar,
    int64_t nc, int64_t rpc, double* __restrict__ part) {
  __shared__ A xs[kRowsChunk][kPad];
  const int tid = threadIdx.x;
  const int bi = tid >> 4, bj = tid & 15;
  A acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = A(0);
  const int64_t nrows = (int64_t)ns * nvar;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = r0 + rpc < nrows ? r0 + rpc : nrows;
  for (int64_t base = r0; base < r1; base += kRowsChunk) {
    __syncthreads();
    // stage 64 rows x 64 columns: consecutive threads take consecutive rows
    // of one column (coalesced along the sorted cells)
#pragma unroll 4
    for (int idx = tid; idx < kRowsChunk * 64; idx += 256) {
      const int rr = idx & (kRowsChunk - 1), j = idx >> 6;
      const int64_t r = base + rr;
      A x = A(0);
      if (r < r1 && j < m) x = (A)phi[(int64_t)j * N + sample_dof(cells, ns, nc, r)];
      xs[rr][j] = x;
    }
    __syncthreads();
    for (int rr = 0; rr < kRowsChunk; ++rr) {
      A x4[4], y4[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        x4[a] = xs[rr][4 * bi + a];
        y4[a] = xs[rr][4 * bj + a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(x4[a], y4[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
      part[(int64_t)blockIdx.x * 4096 + (4 * bi + a) * 64 + 4 * bj + b] = (double)acc[a][b];
}

// Right-hand side Phi_S^T (v - psi)_S: CTA b takes the rows [b * rpc,
// (b + 1) * rpc) in 32-row blocks, one block per warp at a time; lane = row,
// which loads its m basis entries (coalesced across the warp along the
// sorted cells) and accumulates them, times (v - psi) at its dof, in
// registers.  Warp sums by shuffles, CTA sums in shared memory, FP64
// partials to part[b * 64 ...].
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_sample_rhs(
    const T* __restrict__ phi, int64_t N, int m, const int* __restrict__ cells, int ns,
    int nvar, int64_t nc, int64_t rpc, const T* __restrict__ v, const T* __restrict__ psi,
    double* __restrict__ part) {
  __shared__ A red[8][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nrows = (int64_t)ns * nvar;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = r0 + rpc < nrows ? r0 + rpc : nrows;
  A acc[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) acc[j] = A(0);
  for (int64_t base = r0 + 32 * warp; base < r1; base += 256) {
    const int64_t r = base + lane;
    if (r < r1) {
      const int64_t dof = sample_dof(cells, ns, nc, r);
      const A d = (A)v[dof] - (A)psi[dof];
#pragma unroll
      for (int j = 0; j < 64; ++j)
        if (j < m) acc[j] = fma((A)phi[(int64_t)j * N + dof], d, acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    if (j < m) {
      A x = acc[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[warp][j] = x;
    }
  }
  __syncthreads();
  if (threadIdx.x < 64) {
    const int j = threadIdx.x;
    double t = 0.0;
    if (j < m)
      for (int w = 0; w < 8; ++w) t += (double)red[w][j];
    part[(int64_t)blockIdx.x * 64 + j] = t;
  }
}

// out[e] = sum over nb partials of part[b * len + e] (FP64).  A CTA takes
// 64 consecutive e; its blockDim / 64 thread groups take every (blockDim /
// 64)-th partial with eight independent chains each, then the groups' sums
// are added in a fixed order.
__global__ void k_sum_partials(const double* __restrict__ part, int nb, int len,
                               double* __restrict__ out) {
  __shared__ double red[16][64];
  const int el = threadIdx.x & 63, grp = threadIdx.x >> 6, ngrp = blockDim.x >> 6;
  const int e = blockIdx.x * 64 + el;
  double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (e < len) {
    int b = grp;
    for (; b + 7 * ngrp < nb; b += 8 * ngrp)
#pragma unroll
      for (int u = 0; u < 8; ++u) s[u] += part[(int64_t)(b + u * ngrp) * len + e];
    for (; b < nb; b += ngrp) s[0] += part[(int64_t)b * len + e];
  }
  red[grp][el] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
  __syncthreads();
  if (grp == 0 && e < len) {
    double t = 0.0;
    for (int g = 0; g < ngrp; ++g) t += red[g][el];
    out[e] = t;
  }
}

// FP64 Cholesky G = L L^T of the m x m normal matrix (stored 64 x 64), one
// CTA of 256 threads, right-looking.  The lower triangle is packed by
// columns from the last one (column j holds rows j..m-1; with c = m-1-j,
// entry (j + q, j) has index c (c + 1) / 2 + q), and thread t owns the
// indices t + 256 u in registers, so the entries right of column k are the
// first (m-1-k)(m-k)/2 indices and the warps past them sit out.  Per column
// k the owners scale it by the pivot's reciprocal into a shared column
// buffer, then every owner of an entry right of k subtracts l_ik l_jk, and
// the owner of (k + 1, k + 1) forms the next pivot.
// L (lower, 64 x 64) and the inverse diagonal to Lout / dinv; *fail = 1 if a
// pivot is not positive (the sample rows do not determine y).
__global__ void __launch_bounds__(256, 1) k_sample_chol(const double* __restrict__ G, int m,
                                                     double* __restrict__ Lout,
                                                     double* __restrict__ dinv,
                                                     int* __restrict__ fail) {
  constexpr int kOwn = 9;  // ceil(64 * 65 / 2 / 256)
  __shared__ double col[64];
  __shared__ double piv[2];  // sqrt(a_kk), 1 / sqrt(a_kk)
  const int t = threadIdx.x;
  int ii[kOwn], jj[kOwn];
  double a[kOwn];
  const int ntri = m * (m + 1) / 2;
#pragma unroll
  for (int u = 0; u < kOwn; ++u) {
    const int idx = t + 256 * u;
    int i = -1, j = 0;
    if (idx < ntri) {
      int c = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
      while (c * (c + 1) / 2 > idx) --c;
      while ((c + 1) * (c + 2) / 2 <= idx) ++c;
      j = m - 1 - c;
      i = j + (idx - c * (c + 1) / 2);
    }
    ii[u] = i;
    jj[u] = j;
    a[u] = i >= 0 ? G[i * 64 + j] : 0.0;
  }
  // 1 / sqrt(x) from an FP32 seed and two FP64 Newton steps
  auto pivot = [&](double x) {
    if (!(x > 0.0)) {
      *fail = 1;
      piv[0] = 0.0;
      piv[1] = 0.0;
      return;
    }
    const double y = rsqrt64(x);
    piv[0] = x * y;
    piv[1] = y;
  };
  // entry (0, 0) opens the last column's segment, at index m (m - 1) / 2
  const int idx00 = m * (m - 1) / 2;
  if (m > 0 && t == idx00 % 256) {
#pragma unroll
    for (int u = 0; u < kOwn; ++u)
      if (t + 256 * u == idx00) pivot(a[u]);
  }
  for (int idx = t; idx < 64 * 64; idx += 256) {
    const int i = idx >> 6, j = idx & 63;
    if (i >= m || j > i) Lout[idx] = 0.0;
  }
  for (int i = m + t; i < 64; i += 256) dinv[i] = 0.0;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    const double r = piv[1];
#pragma unroll
    for (int u = 0; u < kOwn; ++u) {
      if (jj[u] == k && ii[u] > k) {
        a[u] *= r;
        col[ii[u]] = a[u];
      } else if (jj[u] == k && ii[u] == k) {
        a[u] = piv[0];
        dinv[k] = r;
      }
    }
    __syncthreads();
    const int nact = (m - 1 - k) * (m - k) / 2;  // entries right of column k
#pragma unroll
    for (int u = 0; u < kOwn; ++u) {
      if (256 * u + (t & ~31) < nact && t + 256 * u < nact) {  // whole warps skip
        a[u] = fma(-col[ii[u]], col[jj[u]], a[u]);
        if (ii[u] == k + 1 && jj[u] == k + 1) pivot(a[u]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kOwn; ++u)
    if (ii[u] >= 0) Lout[ii[u] * 64 + jj[u]] = a[u];
}

// y = L^{-T} L^{-1} b by one warp (column-oriented, reciprocal diagonal);
// with y_prev, *dy = ||y - y_prev||_2.
__global__ void k_sample_solve(const double* __restrict__ L, const double* __restrict__ dinv,
                               const double* __restrict__ b, int m, double* __restrict__ y,
                               const double* __restrict__ y_prev, double* __restrict__ dy) {
  __shared__ double Ls[64][65];
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) Ls[idx >> 6][idx & 63] = L[idx];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double x0 = lane < m ? b[lane] : 0.0, x1 = lane + 32 < m ? b[lane + 32] : 0.0;
  const double i0 = dinv[lane], i1 = dinv[lane + 32];
  for (int k = 0; k < m; ++k) {  // forward: L z = b
    const double zk = __shfl_sync(0xffffffffu, k < 32 ? x0 : x1, k & 31) *
                      __shfl_sync(0xffffffffu, k < 32 ? i0 : i1, k & 31);
    if (lane == (k & 31)) {
      if (k < 32)
        x0 = zk;
      else
        x1 = zk;
    }
    if (lane > k && lane < m) x0 = fma(-Ls[lane][k], zk, x0);
    if (lane + 32 > k && lane + 32 < m) x1 = fma(-Ls[lane + 32][k], zk, x1);
  }
  for (int k = m - 1; k >= 0; --k) {  // backward: L^T y = z
    const double yk = __shfl_sync(0xffffffffu, k < 32 ? x0 : x1, k & 31) *
                      __shfl_sync(0xffffffffu, k < 32 ? i0 : i1, k & 31);
    if (lane == (k & 31)) {
      if (k < 32)
        x0 = yk;
      else
        x1 = yk;
    }
    if (lane < k) x0 = fma(-Ls[k][lane], yk, x0);
    if (lane + 32 < k) x1 = fma(-Ls[k][lane + 32], yk, x1);
  }
  double d = 0.0;
  if (lane < m) {
    if (y_prev) d = (x0 - y_prev[lane]) * (x0 - y_prev[lane]);
    y[lane] = x0;
  }
  if (lane + 32 < m) {
    if (y_prev) d = fma(x1 - y_prev[lane + 32], x1 - y_prev[lane + 32], d);
    y[lane + 32] = x1;
  }
  d = warp_sum(d);
  if (lane == 0 && y_prev && dy) *dy = sqrt(d);
}

int nblocks_for(int64_t nrows) {
  int64_t nb = (nrows + 2047) / 2048;
  if (nb > 152 * 2) nb = 152 * 2;
  return (int)(nb < 1 ? 1 : nb);
}

}  // namespace

size_t sample_part_doubles() { return (size_t)152 * 2 * 4096; }

template <typename T>
void launch_sample_normal(const T* phi, int64_t N, int m, const int* cells, int ns, int nvar,
                          int64_t nc, int red, double* part, double* G, double* L, double* dinv,
                          int* fail, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (red != 0) {
      const int nbt = launch_sample_gram_tc(phi, N, m, cells, ns, nvar, nc, red, part, fail + 1, s);
      k_sum_partials<<<64, 256, 0, HY_S(s)>>>(part, nbt, 4096, G);
      k_sample_chol<<<1, 256, 0, HY_S(s)>>>(G, m, L, dinv, fail);
      return;
    }
  }
  const int64_t nrows = (int64_t)ns * nvar;
  const int nb = nblocks_for(nrows);
  const int64_t rpc = (nrows + nb - 1) / nb;
  using A = typename std::conditional<sizeof(T) == 4, float, double>::type;
  k_sample_moments<T, A><<<nb, 256, 0, HY_S(s)>>>(phi, N, m, cells, ns, nvar, nc, rpc, part);
  k_sum_partials<<<64, 256, 0, HY_S(s)>>>(part, nb, 4096, G);
  k_sample_chol<<<1, 256, 0, HY_S(s)>>>(G, m, L, dinv, fail);
}

template <typename T>
void launch_sample_solve(const T* phi, int64_t N, int m, const int* cells, int ns, int nvar,
                         int64_t nc, const T* v, const T* psi, double* part, double* b,
                         const double* L, const double* dinv, double* y, const double* y_prev,
                         double* dy, cudaStream_t s) {
  const int64_t nrows = (int64_t)ns * nvar;
  // rows per CTA a multiple of the 256 rows its 8 warps take per sweep
  int64_t nb = (nrows + 1023) / 1024;
  if (nb > 152 * 4) nb = 152 * 4;
  if (nb < 1) nb = 1;
  const int64_t rpc = ((nrows + nb - 1) / nb + 255) / 256 * 256;
  nb = (nrows + rpc - 1) / rpc;
  using A = typename std::conditional<sizeof(T) == 4, float, double>::type;
  k_sample_rhs<T, A><<<(int)nb, 256, 0, HY_S(s)>>>(phi, N, m, cells, ns, nvar, nc, rpc, v, psi,
                                                    part);
  k_sum_partials<<<1, 1024, 0, HY_S(s)>>>(part, (int)nb, 64, b);
  k_sample_solve<<<1, 256, 0, HY_S(s)>>>(L, dinv, b, m, y, y_prev, dy);
}

#define HY_INST(T)                                                                            \
  template void launch_sample_normal<T>(const T*, int64_t, int, const int*, int, int, int64_t, \
                                        int, double*, double*, double*, double*, int*,         \
                                        cudaStream_t);                                         \
  template void launch_sample_solve<T>(const T*, int64_t, int, const int*, int, int, int64_t,  \
                                       const T*, const T*, double*, double*, const double*,    \
                                       const double*, double*, const double*, double*,         \
                                       cudaStream_t);
HY_INST(float)
HY_INST(double)
#undef HY_INST

}  // namespace hy
