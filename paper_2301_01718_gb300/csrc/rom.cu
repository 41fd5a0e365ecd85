// Reduced-basis kernels: Sec. 2.3.1 of the paper.
//
//  * gappy coordinates y = (P^T Phi)^+ P^T (v - psi) (Eq. red_coord): the
//    pseudo-inverse of the n_p x m sampled basis is formed once per basis
//    (Householder QR in FP64, one CTA) and applied per solve (an m x n_p
//    FP64 GEMV).
//  * reconstruction psi + Phi y on S-breve (Algorithm 1) and the
//    pointwise reconstruction error per cell (Sec. 2.3.3): HBM-bound GEMVs
//    over Phi (column-major, so each column read is coalesced).
//  * POD_m (Eq. pod), two implementations:
//      FP64 states: one-sided (Hestenes) Jacobi SVD of the centred window,
//        one CTA per column pair per round; relative accuracy of the small
//        singular values is that of the data.
//      FP32 states: the snapshot-ring Gram matrix H_ij = gamma_i . gamma_j is
//        kept up to date with one new row per snapshot (float-float
//        accumulation of exact FP32 products), centred by the identity
//        (X - psi 1^T)^T (X - psi 1^T) = H - h 1^T - 1 h^T + (psi.psi) 1 1^T
//        with psi the mean of ring slots, diagonalised in FP64 by pivoted
//        Cholesky and one-sided Jacobi (one thread-block cluster), and
//        Phi = X_c V_m Sigma_m^{-1} is formed in one pass over the window
//        that also produces the next reference state psi (Eq. mean).
#include <cooperative_groups.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace hy {

// ---------------------------------------------------------------------------
// gappy least squares
// ---------------------------------------------------------------------------

// Pseudo-inverse of A = Phi[points, 0:m] (n_p x m, full column rank) as
// pinv (m x n_p, row-major) = R^{-1} Q^T from a Householder QR.  Dynamic
// shared memory: A and Q (n_p*m each) + R (m*m) + beta (m) doubles.
template <typename T>
__global__ void k_gappy_pinv(const T* __restrict__ phi, int64_t N, int m,
                             const int* __restrict__ pts, int np, double* __restrict__ pinv,
                             int* status) {
  extern __shared__ double sm[];
  double* A = sm;                  // column-major n_p x m
  double* Q = A + (size_t)np * m;  // column-major n_p x m
  double* R = Q + (size_t)np * m;  // row-major m x m
  double* beta = R + (size_t)m * m;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int idx = tid; idx < np * m; idx += nt) {
    const int i = idx % np, j = idx / np;
    A[idx] = (double)phi[(int64_t)j * N + pts[i]];
  }
  __syncthreads();
  // Householder QR: reflector j stored in A[j:, j] with v_j = 1 implied off
  for (int j = 0; j < m; ++j) {
    double s = 0.0;
    for (int i = j + tid; i < np; i += nt) s = fma(A[j * np + i], A[j * np + i], s);
    s = block_sum(s);
    const double ajj = A[j * np + j];
    const double nrm = sqrt(s);
    const double alpha = ajj >= 0.0 ? -nrm : nrm;  // R_jj
    const double v0 = ajj - alpha;
    // v = [1, A[j+1:, j] / v0], beta = -v0 / alpha
    __syncthreads();
    if (tid == 0) {
      beta[j] = (nrm == 0.0) ? 0.0 : -v0 / alpha;
      A[j * np + j] = alpha;
    }
    const double iv0 = (v0 == 0.0) ? 0.0 : rcp64(v0);
    for (int i = j + 1 + tid; i < np; i += nt) A[j * np + i] *= iv0;
    __syncthreads();
    const double bj = beta[j];
    // apply (I - beta v v^T) to columns j+1..m-1, one warp per column
    for (int col = j + 1 + wid; col < m; col += nw) {
      double d = 0.0;
      for (int i = j + lane; i < np; i += 32) {
        const double vi = i == j ? 1.0 : A[j * np + i];
        d = fma(vi, A[col * np + i], d);
      }
      d = warp_sum(d) * bj;
      for (int i = j + lane; i < np; i += 32) {
        const double vi = i == j ? 1.0 : A[j * np + i];
        A[col * np + i] = fma(-d, vi, A[col * np + i]);
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < m * m; idx += nt) {
    const int r = idx / m, cc = idx % m;
    R[idx] = cc >= r ? A[cc * np + r] : 0.0;
  }
  // Q = H_0 ... H_{m-1} [I; 0]
  for (int idx = tid; idx < np * m; idx += nt) {
    const int i = idx % np, j = idx / np;
    Q[idx] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = m - 1; j >= 0; --j) {
    const double bj = beta[j];
    for (int col = j + wid; col < m; col += nw) {
      double d = 0.0;
      for (int i = j + lane; i < np; i += 32) {
        const double vi = i == j ? 1.0 : A[j * np + i];
        d = fma(vi, Q[col * np + i], d);
      }
      d = warp_sum(d) * bj;
      for (int i = j + lane; i < np; i += 32) {
        const double vi = i == j ? 1.0 : A[j * np + i];
        Q[col * np + i] = fma(-d, vi, Q[col * np + i]);
      }
    }
    __syncthreads();
  }
  // numerical rank: pivot j counts as zero when |R_jj| <= 64 n_p eps
  // max_i |R_ii| (a QR without pivoting of a rank-deficient matrix, e.g. one
  // with two equal rows and n_p = m, leaves a pivot of a few eps there); its
  // reciprocal is taken as 0 below (a truncated solve) and *status is
  // incremented
  double rmax = 0.0;
  for (int j = 0; j < m; ++j) rmax = fmax(rmax, fabs(R[j * m + j]));
  const double rtol = 64.0 * (double)np * 2.220446049250313e-16 * rmax;
  bool bad = rmax == 0.0;
  for (int j = 0; j < m; ++j) bad |= !(fabs(R[j * m + j]) > rtol);
  if (bad && tid == 0) atomicAdd(status, 1);
  // pinv = R^{-1} Q^T: back substitution in shared memory (X, m x n_p, in
  // the reflectors' space, free once Q is formed), one thread per column i
  // of Q^T, four chains, reciprocal diagonal; then one coalesced store
  double* X = A;
  for (int i = tid; i < np; i += nt) {
    for (int r = m - 1; r >= 0; --r) {
      double p4[4] = {Q[r * np + i], 0.0, 0.0, 0.0};
      int cc = r + 1;
      for (; cc + 3 < m; cc += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) p4[u] = fma(-R[r * m + cc + u], X[(cc + u) * np + i], p4[u]);
      }
      for (; cc < m; ++cc) p4[0] = fma(-R[r * m + cc], X[cc * np + i], p4[0]);
      const double rr = R[r * m + r];
      X[r * np + i] = ((p4[0] + p4[1]) + (p4[2] + p4[3])) * (fabs(rr) > rtol ? rcp64(rr) : 0.0);
    }
  }
  __syncthreads();
  for (int idx = tid; idx < m * np; idx += nt) pinv[idx] = X[idx];
}

// The same pseudo-inverse by a thread-block cluster of C = min(16, m) CTAs
// of 128 threads, CTA c owning the columns [c cpc, (c + 1) cpc) of A (and of
// Q), so that the FP64 work of each step spreads over C SMs:
//   * QR: at step j the owner of column j forms the reflector; after a
//     cluster barrier every CTA copies it (and beta_j) from the owner's
//     shared memory and applies it to its own columns beyond j;
//   * every CTA then gathers the whole factored A (reflectors and R) and
//     forms its own columns of Q = H_0 ... H_{m-1} [I; 0];
//   * row r of R^{-1} for each of its own rows r, by forward substitution
//     in R^T (one warp per row; pivots at or below the rank tolerance
//     contribute zero, as in the one-CTA kernel's truncated solve);
//   * after a second barrier, the whole Q gathered, and its rows of
//     pinv = R^{-1} Q^T.
// Shared memory: the whole A or Q (n_p m), own A and Q columns (2 n_p cpc),
// the reflector (n_p), R^{-1} rows (cpc m) doubles.
constexpr int kPinvThreads = 128;
constexpr int kPinvMaxC = 16;

template <typename T>
__global__ void __launch_bounds__(kPinvThreads, 1)
    k_gappy_pinv_cl(const T* __restrict__ phi, int64_t N, int m, const int* __restrict__ pts,
                    int np, double* __restrict__ pinv, int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), me = (int)cl.block_rank();
  const int cpc = (m + C - 1) / C;
  const int c0 = me * cpc, nc = c0 < m ? (c0 + cpc <= m ? cpc : m - c0) : 0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kPinvThreads >> 5;
  extern __shared__ double psm[];
  double* Full = psm;                      // n_p x m, column-major
  double* Aloc = Full + (size_t)np * m;    // n_p x cpc: own columns of A
  double* Qloc = Aloc + (size_t)np * cpc;  // n_p x cpc: own columns of Q
  double* vloc = Qloc + (size_t)np * cpc;  // n_p: the step's reflector
  double* Y = vloc + np;                   // cpc x m: own rows of R^{-1}
  __shared__ double beta_own[64];
  __shared__ double vbeta;
  for (int idx = tid; idx < np * nc; idx += kPinvThreads) {
    const int i = idx % np, jj = idx / np;
    Aloc[idx] = (double)phi[(int64_t)(c0 + jj) * N + pts[i]];
  }
  cl.sync();
  // Householder QR: reflector j stored in column j (rows > j), v_j = 1 implied
  for (int j = 0; j < m; ++j) {
    const int o = j / cpc, jo = j - o * cpc;
    if (me == o) {
      double* a = Aloc + (size_t)jo * np;
      double s = 0.0;
      for (int i = j + tid; i < np; i += kPinvThreads) s = fma(a[i], a[i], s);
      s = block_sum(s);
      const double ajj = a[j];
      const double nrm = sqrt(s);
      const double alpha = ajj >= 0.0 ? -nrm : nrm;  // R_jj
      const double v0 = ajj - alpha;
      __syncthreads();
      if (tid == 0) {
        beta_own[jo] = (nrm == 0.0) ? 0.0 : -v0 / alpha;
        a[j] = alpha;
      }
      const double iv0 = (v0 == 0.0) ? 0.0 : 1.0 / v0;
      for (int i = j + 1 + tid; i < np; i += kPinvThreads) a[i] *= iv0;
    }
    cl.sync();
    // the reflector from its owner, then applied to the own columns beyond j
    if (nc > 0 && c0 + nc - 1 > j) {
      const double* ao = cl.map_shared_rank(Aloc, (unsigned)o) + (size_t)jo * np;
      for (int i = j + 1 + tid; i < np; i += kPinvThreads) vloc[i] = ao[i];
      if (tid == 0) vbeta = cl.map_shared_rank(beta_own, (unsigned)o)[jo];
      __syncthreads();
      const double bj = vbeta;
      for (int jj = wid; jj < nc; jj += nw) {
        if (c0 + jj <= j) continue;
        double* col = Aloc + (size_t)jj * np;
        double d = 0.0;
        for (int i = j + lane; i < np; i += 32) d = fma(i == j ? 1.0 : vloc[i], col[i], d);
        d = warp_sum(d) * bj;
        for (int i = j + lane; i < np; i += 32) col[i] = fma(-d, i == j ? 1.0 : vloc[i], col[i]);
      }
    }
    __syncthreads();
  }
  cl.sync();
  // the whole factored A, and the betas
  __shared__ double betas[64];
  for (int idx = tid; idx < np * m; idx += kPinvThreads) {
    const int i = idx % np, j = idx / np, o = j / cpc, jo = j - o * cpc;
    Full[idx] = cl.map_shared_rank(Aloc, (unsigned)o)[(size_t)jo * np + i];
  }
  for (int j = tid; j < m; j += kPinvThreads) {
    const int o = j / cpc;
    betas[j] = cl.map_shared_rank(beta_own, (unsigned)o)[j - o * cpc];
  }
  __syncthreads();
  // numerical rank (the same rule and tolerance as the one-CTA kernel)
  double rmax = 0.0;
  for (int j = 0; j < m; ++j) rmax = fmax(rmax, fabs(Full[(size_t)j * np + j]));
  const double rtol = 64.0 * (double)np * 2.220446049250313e-16 * rmax;
  bool bad = rmax == 0.0;
  for (int j = 0; j < m; ++j) bad |= !(fabs(Full[(size_t)j * np + j]) > rtol);
  if (bad && me == 0 && tid == 0) atomicAdd(status, 1);
  __shared__ double rdiag[64];  // 1 / R_kk, 0 for a pivot at or below the tolerance
  for (int k = tid; k < m; k += kPinvThreads) {
    const double d = Full[(size_t)k * np + k];
    rdiag[k] = fabs(d) > rtol ? 1.0 / d : 0.0;
  }
  // own columns of Q = H_0 ... H_{m-1} [I; 0]
  for (int idx = tid; idx < np * nc; idx += kPinvThreads) {
    const int i = idx % np, jj = idx / np;
    Qloc[idx] = i == c0 + jj ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = m - 1; j >= 0; --j) {
    const double bj = betas[j];
    const double* v = Full + (size_t)j * np;
    for (int jj = wid; jj < nc; jj += nw) {
      if (c0 + jj < j) continue;
      double* col = Qloc + (size_t)jj * np;
      double d = 0.0;
      for (int i = j + lane; i < np; i += 32) d = fma(i == j ? 1.0 : v[i], col[i], d);
      d = warp_sum(d) * bj;
      for (int i = j + lane; i < np; i += 32) col[i] = fma(-d, i == j ? 1.0 : v[i], col[i]);
    }
    __syncthreads();
  }
  // own rows r of R^{-1}: y^T R = e_r^T, i.e. y_k = -(sum_{r<=l<k} R_lk y_l) / R_kk
  // (R_lk = Full[k np + l] for l <= k)
  for (int rr = wid; rr < nc; rr += nw) {
    const int r = c0 + rr;
    double* y = Y + (size_t)rr * m;
    for (int k = lane; k < m; k += 32) y[k] = 0.0;
    __syncwarp();
    if (lane == 0) y[r] = rdiag[r];
    __syncwarp();
    for (int k = r + 1; k < m; ++k) {
      double acc = 0.0;
      for (int l = r + lane; l < k; l += 32) acc = fma(Full[(size_t)k * np + l], y[l], acc);
      acc = warp_sum(acc);
      if (lane == 0) y[k] = -acc * rdiag[k];
      __syncwarp();
    }
  }
  cl.sync();
  // the whole Q (its own columns from every CTA), then own rows of pinv
  for (int idx = tid; idx < np * m; idx += kPinvThreads) {
    const int i = idx % np, j = idx / np, o = j / cpc, jo = j - o * cpc;
    Full[idx] = cl.map_shared_rank(Qloc, (unsigned)o)[(size_t)jo * np + i];
  }
  cl.sync();  // no CTA leaves while another still reads its Q columns
  for (int idx = tid; idx < nc * np; idx += kPinvThreads) {
    const int rr = idx / np, i = idx % np, r = c0 + rr;
    const double* y = Y + (size_t)rr * m;
    double p4[4] = {0.0, 0.0, 0.0, 0.0};
    int k = r;
    for (; k + 3 < m; k += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) p4[u] = fma(y[k + u], Full[(size_t)(k + u) * np + i], p4[u]);
    }
    for (; k < m; ++k) p4[0] = fma(y[k], Full[(size_t)k * np + i], p4[0]);
    pinv[(size_t)r * np + i] = (p4[0] + p4[1]) + (p4[2] + p4[3]);
  }
}

template <typename T>
void launch_gappy_pinv(const T* phi, int64_t N, int m, const int* pts, int np, double* pinv,
                       int* status, cudaStream_t s) {
  if (m <= 0) return;
  // the cluster version where its shared memory fits, else one CTA
  const int cpc = (m + kPinvMaxC - 1) / kPinvMaxC, C = (m + cpc - 1) / cpc;
  const size_t smem_cl =
      sizeof(double) * ((size_t)np * m + (size_t)2 * np * cpc + np + (size_t)cpc * m);
  if (C > 1 && m <= 64 && smem_cl <= 200 * 1024) {
    cudaFuncSetAttribute(k_gappy_pinv_cl<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    smem_at_least((const void*)k_gappy_pinv_cl<T>, smem_cl);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(C);
    lc.blockDim = dim3(kPinvThreads);
    lc.dynamicSmemBytes = smem_cl;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    ::hy::count_launch();
    if (cudaLaunchKernelEx(&lc, k_gappy_pinv_cl<T>, phi, N, m, pts, np, pinv, status) ==
        cudaSuccess)
      return;
    cudaGetLastError();
  }
  const size_t smem = sizeof(double) * ((size_t)2 * np * m + (size_t)m * m + m);
  smem_at_least((const void*)k_gappy_pinv<T>, smem);
  k_gappy_pinv<T><<<1, 256, smem, HY_S(s)>>>(phi, N, m, pts, np, pinv, status);
}

size_t gappy_pinv_smem(int m, int np) {
  return sizeof(double) * ((size_t)2 * np * m + (size_t)m * m + m);
}

// y = pinv (v[P] - psi[P]); also |y - y_prev|_2 into *dy when y_prev given.
// With rank_flag given and non-zero (the QR found P^T Phi rank-deficient)
// every y_j is set to NaN instead.
template <typename T>
__global__ void k_gappy_apply(const double* __restrict__ pinv, int m, int np,
                              const int* __restrict__ pts, const T* __restrict__ v,
                              const T* __restrict__ psi, double* __restrict__ y,
                              const double* __restrict__ y_prev, double* dy,
                              const int* __restrict__ rank_flag) {
  __shared__ double b[1024];
  __shared__ double ynew[256];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < np; i += blockDim.x) b[i] = (double)v[pts[i]] - (double)psi[pts[i]];
  __syncthreads();
  for (int j = wid; j < m; j += nw) {
    double acc = 0.0;
    for (int i = lane; i < np; i += 32) acc = fma(pinv[(int64_t)j * np + i], b[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) ynew[j] = acc;
  }
  __syncthreads();
  double d2 = 0.0;
  for (int j = tid; j < m; j += blockDim.x) {
    if (y_prev) {
      const double d = ynew[j] - y_prev[j];
      d2 = fma(d, d, d2);
    }
  }
  d2 = block_sum(d2);
  const bool deficient = rank_flag && *rank_flag != 0;
  for (int j = tid; j < m; j += blockDim.x) y[j] = deficient ? __longlong_as_double(0x7ff8000000000000ll) : ynew[j];
  if (dy && tid == 0) *dy = sqrt(d2);
}

template <typename T>
void launch_gappy_apply(const double* pinv, int m, int np, const int* pts, const T* v,
                        const T* psi, double* y, const double* y_prev, double* dy,
                        cudaStream_t s, const int* rank_flag) {
  k_gappy_apply<T><<<1, 256, 0, HY_S(s)>>>(pinv, m, np, pts, v, psi, y, y_prev, dy, rank_flag);
}

// ---------------------------------------------------------------------------
// reconstruction and pointwise error
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_reconstruct(const T* __restrict__ phi, int64_t N, int64_t nc, int m,
                              const double* __restrict__ y, const T* __restrict__ psi,
                              const uint32_t* __restrict__ s_hat, int only_set,
                              T* __restrict__ q) {
  __shared__ T ys[256];
  for (int j = threadIdx.x; j < m; j += blockDim.x) ys[j] = (T)y[j];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (s_hat && bit_get(s_hat, r % nc) != (bool)only_set) continue;
    T acc = (T)0;
    for (int j = 0; j < m; ++j) acc = fma(phi[(int64_t)j * N + r], ys[j], acc);
    q[r] = psi[r] + acc;
  }
}

template <typename T>
void launch_reconstruct(const T* phi, int64_t N, int64_t nc, int m, const double* y,
                        const T* psi, const uint32_t* s_hat, int only_set, T* q, cudaStream_t s) {
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_reconstruct<T><<<(int)blocks, 256, 0, HY_S(s)>>>(phi, N, nc, m, y, psi, s_hat, only_set, q);
}

template <typename T>
__global__ void k_cell_error(const T* __restrict__ g, const T* __restrict__ psi,
                             const T* __restrict__ phi, int64_t nc, int nvar, int m,
                             const double* __restrict__ y, T* __restrict__ eps) {
  __shared__ T ys[256];
  for (int j = threadIdx.x; j < m; j += blockDim.x) ys[j] = (T)y[j];
  __syncthreads();
  const int64_t N = nc * nvar;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    T e = (T)0;
    for (int v = 0; v < nvar; ++v) {
      const int64_t r = v * nc + c;
      T acc = (T)0;
      for (int j = 0; j < m; ++j) acc = fma(phi[(int64_t)j * N + r], ys[j], acc);
      const T d = (g[r] - psi[r]) - acc;
      e = v == 0 ? d * d : e + d * d;
    }
    eps[c] = e;
  }
}

template <typename T>
void launch_cell_error(const T* g, const T* psi, const T* phi, int64_t nc, int nvar, int m,
                       const double* y, T* eps, cudaStream_t s) {
  int64_t blocks = (nc + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_cell_error<T><<<(int)blocks, 256, 0, HY_S(s)>>>(g, psi, phi, nc, nvar, m, y, eps);
}

// ---------------------------------------------------------------------------
// snapshot-ring Gram matrix (FP32 path)
// ---------------------------------------------------------------------------

// part[j * nchunk + chunk] = sum over the chunk's rows of ring[s][r]*ring[j][r]
// Grid: x = ring slot j (fastest, so the CTAs in flight share the chunk of
// slot s through L2), y = row chunk.
// Dot product accumulated exactly enough for the centring identity: each
// product a*b is split exactly into p + e (p = fl(a*b), e = fma(a, b, -p)),
// and the running sum is a float-float pair (hi, lo) updated with the
// error-free TwoSum of Knuth; lo also collects the product errors.  The
// per-thread pair is combined in FP64.  FP32 data only (FP64 data uses FP64).
HY_DEV void ff_add(float& hi, float& lo, float p, float e) {
  const float s = hi + p;
  const float bb = s - hi;
  const float t = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo = lo + (t + e);
}

template <typename T>
__global__ void k_gram_row(const T* __restrict__ ring, int64_t N, int s, int64_t chunk,
                           double* __restrict__ part) {
  const int j = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * chunk;
  int64_t r1 = r0 + chunk;
  if (r1 > N) r1 = N;
  const T* a = ring + (int64_t)s * N;
  const T* b = ring + (int64_t)j * N;
  double acc = 0.0;
  if (sizeof(T) == 4) {
    float hi = 0.f, lo = 0.f;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      const float x = (float)a[r], y = (float)b[r];
      const float p = x * y;
      const float e = fmaf(x, y, -p);
      ff_add(hi, lo, p, e);
    }
    acc = (double)hi + (double)lo;
  } else {
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
      acc = fma((double)a[r], (double)b[r], acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[(int64_t)j * gridDim.y + blockIdx.y] = acc;
}

// Two rows at once, s1 and s2, in one pass over the ring: each block reads
// its chunk of slot j once for both dot products.  Each dot product is
// accumulated exactly as k_gram_row accumulates it (same rows per thread,
// same order), so the rows are the same bits as two k_gram_row passes.
// part: row s1's partials at [j * nchunk + y], row s2's at
// [(nslot + j) * nchunk + y].
template <typename T>
__global__ void k_gram_row2(const T* __restrict__ ring, int64_t N, int s1, int s2, int64_t chunk,
                            double* __restrict__ part) {
  const int j = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * chunk;
  int64_t r1 = r0 + chunk;
  if (r1 > N) r1 = N;
  const T* a1 = ring + (int64_t)s1 * N;
  const T* a2 = ring + (int64_t)s2 * N;
  const T* b = ring + (int64_t)j * N;
  double acc1 = 0.0, acc2 = 0.0;
  if (sizeof(T) == 4) {
    float hi1 = 0.f, lo1 = 0.f, hi2 = 0.f, lo2 = 0.f;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      const float y = (float)b[r];
      const float x1 = (float)a1[r], x2 = (float)a2[r];
      const float p1 = x1 * y, p2 = x2 * y;
      const float e1 = fmaf(x1, y, -p1), e2 = fmaf(x2, y, -p2);
      ff_add(hi1, lo1, p1, e1);
      ff_add(hi2, lo2, p2, e2);
    }
    acc1 = (double)hi1 + (double)lo1;
    acc2 = (double)hi2 + (double)lo2;
  } else {
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      const double y = (double)b[r];
      acc1 = fma((double)a1[r], y, acc1);
      acc2 = fma((double)a2[r], y, acc2);
    }
  }
  acc1 = block_sum(acc1);
  acc2 = block_sum(acc2);
  if (threadIdx.x == 0) {
    part[(int64_t)j * gridDim.y + blockIdx.y] = acc1;
    part[((int64_t)gridDim.x + j) * gridDim.y + blockIdx.y] = acc2;
  }
}

__global__ void k_gram_finalize(const double* __restrict__ part, int nslot, int nchunk, int s,
                                double* __restrict__ H) {
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nchunk; i += blockDim.x) acc += part[(int64_t)j * nchunk + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    H[(int64_t)s * nslot + j] = acc;
    H[(int64_t)j * nslot + s] = acc;
  }
}

template <typename T>
void launch_gram_row(const T* ring, int64_t N, int nslot, int s, double* part, int max_chunks,
                     double* H, cudaStream_t st) {
  int64_t chunk = (N + max_chunks - 1) / max_chunks;
  if (chunk < 1024) chunk = 1024;
  const int nchunk = (int)((N + chunk - 1) / chunk);
  dim3 grid(nslot, nchunk);
  k_gram_row<T><<<grid, 256, 0, HY_S(st)>>>(ring, N, s, chunk, part);
  k_gram_finalize<<<nslot, 256, 0, HY_S(st)>>>(part, nslot, nchunk, s, H);
}

template <typename T>
void launch_gram_rows2(const T* ring, int64_t N, int nslot, int s1, int s2, double* part,
                       int max_chunks, double* H, cudaStream_t st) {
  int64_t chunk = (N + max_chunks - 1) / max_chunks;
  if (chunk < 1024) chunk = 1024;
  const int nchunk = (int)((N + chunk - 1) / chunk);
  dim3 grid(nslot, nchunk);
  k_gram_row2<T><<<grid, 256, 0, HY_S(st)>>>(ring, N, s1, s2, chunk, part);
  k_gram_finalize<<<nslot, 256, 0, HY_S(st)>>>(part, nslot, nchunk, s1, H);
  k_gram_finalize<<<nslot, 256, 0, HY_S(st)>>>(part + (size_t)nslot * nchunk, nslot, nchunk, s2,
                                               H);
}

// Centred Gram of the window from the ring Gram H (nslot x nslot):
// G[a][b] = H[wa][wb] - h[a] - h[b] + pp, with h[a] = (sum_{j in ps} H[wa][j])/npsi and
// pp = (sum_{j,l in ps} H[j][l]) / (npsi*npsi).  Also xraw2 = sum_a H[wa][wa].
__global__ void k_gram_center(const double* __restrict__ H, int nslot, const int* __restrict__ win,
                              int w, const int* __restrict__ ps, int npsi, double* __restrict__ G,
                              int ldg, double* xraw2) {
  __shared__ double h[256];
  __shared__ double pp;
  const int tid = threadIdx.x;
  for (int a = tid; a < w; a += blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < npsi; ++j) acc += H[(int64_t)win[a] * nslot + ps[j]];
    h[a] = acc / npsi;
  }
  double acc = 0.0;
  for (int idx = tid; idx < npsi * npsi; idx += blockDim.x)
    acc += H[(int64_t)ps[idx / npsi] * nslot + ps[idx % npsi]];
  acc = block_sum(acc);
  double xr = 0.0;
  for (int a = tid; a < w; a += blockDim.x) xr += H[(int64_t)win[a] * nslot + win[a]];
  xr = block_sum(xr);
  if (tid == 0) {
    pp = acc / ((double)npsi * npsi);
    *xraw2 = xr;
  }
  __syncthreads();
  for (int idx = tid; idx < ldg * ldg; idx += blockDim.x) {
    const int a = idx / ldg, b = idx % ldg;
    double v = 0.0;
    if (a < w && b < w) v = ((H[(int64_t)win[a] * nslot + win[b]] - h[a]) - h[b]) + pp;
    G[idx] = v;
  }
}

void launch_gram_center(const double* H, int nslot, const int* win, int w, const int* ps,
                        int npsi, double* G, int ldg, double* xraw2, cudaStream_t s) {
  k_gram_center<<<1, 256, 0, HY_S(s)>>>(H, nslot, win, w, ps, npsi, G, ldg, xraw2);
}

// Same with psi given by its dots hp[j] = psi . ring[j] (all nslot slots)
// and pp = psi . psi (for a psi that is not a mean of ring slots).
__global__ void k_gram_center_explicit(const double* __restrict__ H, int nslot,
                                       const int* __restrict__ win, int w,
                                       const double* __restrict__ hp, const double* __restrict__ pp,
                                       double* __restrict__ G, int ldg, double* xraw2) {
  const int tid = threadIdx.x;
  double xr = 0.0;
  for (int a = tid; a < w; a += blockDim.x) xr += H[(int64_t)win[a] * nslot + win[a]];
  xr = block_sum(xr);
  if (tid == 0) *xraw2 = xr;
  const double p2 = *pp;
  for (int idx = tid; idx < ldg * ldg; idx += blockDim.x) {
    const int a = idx / ldg, b = idx % ldg;
    double v = 0.0;
    if (a < w && b < w) v = ((H[(int64_t)win[a] * nslot + win[b]] - hp[win[a]]) - hp[win[b]]) + p2;
    G[idx] = v;
  }
}

void launch_gram_center_explicit(const double* H, int nslot, const int* win, int w,
                                 const double* hp, const double* pp, double* G, int ldg,
                                 double* xraw2, cudaStream_t s) {
  k_gram_center_explicit<<<1, 256, 0, HY_S(s)>>>(H, nslot, win, w, hp, pp, G, ldg, xraw2);
}

// out[j] = a . ring[j] for all nslot slots (same two-level order as the
// ring Gram rows).
template <typename T>
__global__ void k_dots(const T* __restrict__ a, const T* __restrict__ ring, int64_t N,
                       int64_t chunk, double* __restrict__ part) {
  const int j = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * chunk;
  int64_t r1 = r0 + chunk;
  if (r1 > N) r1 = N;
  const T* b = ring + (int64_t)j * N;
  double acc = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
    acc = fma((double)a[r], (double)b[r], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[(int64_t)j * gridDim.y + blockIdx.y] = acc;
}

__global__ void k_dots_finalize(const double* __restrict__ part, int nchunk,
                                double* __restrict__ out) {
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nchunk; i += blockDim.x) acc += part[(int64_t)j * nchunk + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[j] = acc;
}

template <typename T>
void launch_dots(const T* a, const T* ring, int64_t N, int nslot, double* part, int max_chunks,
                 double* out, cudaStream_t st) {
  int64_t chunk = (N + max_chunks - 1) / max_chunks;
  if (chunk < 1024) chunk = 1024;
  const int nchunk = (int)((N + chunk - 1) / chunk);
  dim3 grid(nslot, nchunk);
  k_dots<T><<<grid, 256, 0, HY_S(st)>>>(a, ring, N, chunk, part);
  k_dots_finalize<<<nslot, 256, 0, HY_S(st)>>>(part, nchunk, out);
}
template void launch_dots<float>(const float*, const float*, int64_t, int, double*, int, double*,
                                 cudaStream_t);
template void launch_dots<double>(const double*, const double*, int64_t, int, double*, int,
                                  double*, cudaStream_t);

__global__ void k_identity(double* V, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x)
    V[i] = (i / n == i % n) ? 1.0 : 0.0;
}

void launch_identity(double* V, int n, cudaStream_t s) { k_identity<<<16, 256, 0, HY_S(s)>>>(V, n); }

// ---------------------------------------------------------------------------
// two-sided cyclic Jacobi (FP64) spread over n/2 CTAs: A (n x n, n even),
// V (n x n column-major) in global memory.  Round-robin ordering: n/2
// disjoint rotations per round, pair b of round r given by rr_pair.
// ---------------------------------------------------------------------------

HY_DEV void rr_pair(int n, int r, int b, int& p, int& q) {
  int a, c;
  if (b == 0) {
    a = r;
    c = n - 1;
  } else {
    a = (r + b) % (n - 1);
    c = (r - b + (n - 1)) % (n - 1);
  }
  p = a < c ? a : c;
  q = a < c ? c : a;
}

// Grid barrier for a cooperative launch (all CTAs co-resident).  The spin is
// bounded: after ~2^22 polls (about a second) the waiting CTA sets *err and
// returns false, and every caller leaves the kernel.
struct GridBar {
  unsigned count;
  unsigned gen;
};

__device__ bool grid_sync_bounded(GridBar* bar, unsigned nblocks, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = &bar->gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      unsigned i = 0;
      while (*vgen == g) {
        if (++i > (1u << 22) || *((volatile int*)err)) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// One full sweep (n - 1 rounds) of the multi-CTA Jacobi in one cooperative
// launch; A ping-pongs between A0 and A1 every round (the result ends in A0
// when n - 1 is even, else in A1).
__global__ void k_jacobi_sweep(double* A0, double* A1, int n, double* __restrict__ V,
                               double floor_abs, int* rotated, GridBar* bar, int* err) {
  __shared__ double cs[2 * 128];
  __shared__ double rp[128], rq[128];
  const int half = n / 2, tid = threadIdx.x, nm1 = n - 1;
  for (int r = 0; r < n - 1; ++r) {
    const double* Ain = (r % 2 == 0) ? A0 : A1;
    double* Aout = (r % 2 == 0) ? A1 : A0;
    for (int b = tid; b < half; b += blockDim.x) {
      int p, q;
      rr_pair(n, r, b, p, q);
      const double apq = __ldcg(Ain + p * n + q), app = __ldcg(Ain + p * n + p),
                   aqq = __ldcg(Ain + q * n + q);
      double c = 1.0, sn = 0.0;
      if (fabs(apq) > floor_abs && fabs(apq) > 1e-14 * sqrt(fabs(app * aqq))) {
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        c = 1.0 / sqrt(1.0 + t * t);
        sn = t * c;
      }
      cs[2 * b] = c;
      cs[2 * b + 1] = sn;
    }
    __syncthreads();
    int p, q;
    rr_pair(n, r, blockIdx.x, p, q);
    const double c = cs[2 * blockIdx.x], sn = cs[2 * blockIdx.x + 1];
    for (int k = tid; k < n; k += blockDim.x) {
      const double ap = __ldcg(Ain + p * n + k), aq = __ldcg(Ain + q * n + k);
      rp[k] = c * ap - sn * aq;
      rq[k] = sn * ap + c * aq;
      if (sn != 0.0) {
        const double vp = __ldcg(V + (int64_t)p * n + k), vq = __ldcg(V + (int64_t)q * n + k);
        V[(int64_t)p * n + k] = c * vp - sn * vq;
        V[(int64_t)q * n + k] = sn * vp + c * vq;
      }
    }
    __syncthreads();
    for (int k = tid; k < n; k += blockDim.x) {
      int partner, b2;
      if (k == nm1 || k == r) {
        partner = k == nm1 ? r : nm1;
        b2 = 0;
      } else {
        partner = ((2 * r - k) % nm1 + nm1) % nm1;
        const int b1 = ((k - r) % nm1 + nm1) % nm1;
        b2 = b1 <= half - 1 ? b1 : nm1 - b1;
      }
      const int p2 = k < partner ? k : partner, q2 = k < partner ? partner : k;
      const double c2 = cs[2 * b2], s2 = cs[2 * b2 + 1];
      double np_, nq_;
      if (k == p2) {
        np_ = c2 * rp[p2] - s2 * rp[q2];
        nq_ = c2 * rq[p2] - s2 * rq[q2];
      } else {
        np_ = s2 * rp[p2] + c2 * rp[q2];
        nq_ = s2 * rq[p2] + c2 * rq[q2];
      }
      // the entry this rotation annihilates is zero, not rounding noise of
      // size eps |A| that would keep later sweeps rotating
      if (sn != 0.0 && k == q) np_ = 0.0;
      if (sn != 0.0 && k == p) nq_ = 0.0;
      Aout[p * n + k] = np_;
      Aout[q * n + k] = nq_;
    }
    if (tid == 0 && sn != 0.0) *rotated = 1;
    if (!grid_sync_bounded(bar, gridDim.x, err)) return;
  }
}

__global__ void k_diag_max(const double* __restrict__ A, int n, double* out) {
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(A[i * n + i]));
  mx = block_max(mx);
  if (threadIdx.x == 0) *out = mx;
}

__global__ void k_copy_diag(const double* __restrict__ A, int n, double* __restrict__ lam) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = A[i * n + i];
}

// Multi-CTA Jacobi: A (n x n, n even, n <= 128) is copied into the ping-pong
// pair (buf, buf + n*n); V starts at the identity.  The host reads one flag
// per sweep (through `host_flag`, pinned) and stops after a sweep without
// rotation or after max_sweeps.  Returns the sweeps run, or -1 on a CUDA error.
int run_jacobi_multi(const double* A, int n, double* V, double* lam, double* buf, int* flag,
                     int* host_flag, double* scale_dev, double* host_scale, int max_sweeps,
                     cudaStream_t s) {
  double* A0 = buf;
  double* A1 = buf + (size_t)n * n;
  cudaMemcpyAsync(A0, A, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s);
  k_identity<<<16, 256, 0, HY_S(s)>>>(V, n);
  k_diag_max<<<1, 128, 0, HY_S(s)>>>(A0, n, scale_dev);
  cudaMemcpyAsync(host_scale, scale_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  const double floor_abs = 1e-16 * host_scale[0];
  // flag[0]: rotated in this sweep; flag[1]: barrier timeout; flag[2..3]: barrier
  GridBar* bar = (GridBar*)(flag + 2);
  int* err = flag + 1;
  cudaMemsetAsync(flag, 0, 4 * sizeof(int), s);
  int sw = 0;
  const int nb = n / 2;
  for (; sw < max_sweeps; ++sw) {
    cudaMemsetAsync(flag, 0, sizeof(int), s);
    void* args[] = {(void*)&A0, (void*)&A1, (void*)&n, (void*)&V, (void*)&floor_abs,
                    (void*)&flag, (void*)&bar, (void*)&err};
    ::hy::count_launch();
    if (cudaLaunchCooperativeKernel((void*)k_jacobi_sweep, dim3(nb), dim3(128), args, 0, s) !=
        cudaSuccess)
      return -1;
    if ((n - 1) % 2 == 1) {  // the result of the last round is in A1
      double* t = A0;
      A0 = A1;
      A1 = t;
    }
    cudaMemcpyAsync(host_flag, flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    if (host_flag[1]) return -2;
    if (!host_flag[0]) break;
  }
  k_copy_diag<<<1, 128, 0, HY_S(s)>>>(A0, n, lam);
  return sw;
}

// ---------------------------------------------------------------------------
// Eigenpairs of a symmetric positive semidefinite G (n x n, n <= 136) by
// pivoted Cholesky and one-sided Jacobi (the preconditioned Jacobi SVD of
// Drmac and Veselic, SIAM J. Matrix Anal. Appl. 29, 2008):
// Pi^T G Pi = R^T R with the pivot the largest remaining diagonal entry, to
// the numerical rank r where that entry drops below n eps max(diag G); the r
// columns of B = R^T (n x r) are then made mutually orthogonal by plane
// rotations, B V = U S, so that G = (Pi U) S^2 (Pi U)^T.  The pivoting grades
// the columns of B and the rotations converge in a few sweeps (two-sided
// Jacobi on G needs about one sweep per decade of its spectrum).  Eigenvalue
// j is |b_j|^2 and its eigenvector Pi b_j / |b_j|; no rotation is
// accumulated.
// ---------------------------------------------------------------------------

constexpr int kEigMaxN = 136;

// Pivoted Cholesky in one CTA, the lower triangle of G in shared memory;
// the pivot exchange swaps rows and columns in place (O(n) entries), so the
// trailing update walks contiguous rows.  Row k of R is kept in the upper
// triangle of the same array (row k, columns >= k: free once column k is
// eliminated), so the loop touches no global memory.  FP64 throughput
// bounds this kernel: the update is s (s + 1) / 2 explicit FMAs at trailing
// size s.  B (column k = row k of R over the pivoted order), piv and r go to
// global memory at the end.
__global__ void __launch_bounds__(1024) k_pchol(const double* __restrict__ G, int ldg, int n,
                                                double* __restrict__ B, int* __restrict__ piv_out,
                                                int* __restrict__ rank_out) {
  extern __shared__ double A[];  // n x n, lower triangle used
  __shared__ int piv[kEigMaxN];
  __shared__ double rk[kEigMaxN];
  __shared__ double rk_s[2];
  __shared__ int pk_s, stop_s;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx - i * n;
    A[idx] = G[(int64_t)i * ldg + j];
  }
  for (int i = tid; i < n; i += nt) piv[i] = i;
  __syncthreads();
  double m0 = 0.0;
  for (int i = tid; i < n; i += nt) m0 = fmax(m0, A[i * n + i]);
  m0 = block_max(m0);
  const double tol = n * 2.220446049250313e-16 * m0;
  int r = n;
  for (int k = 0; k < n; ++k) {
    // largest remaining diagonal entry (lowest index on ties), one warp
    if (wid == 0) {
      double best = -1.0;
      int bidx = k;
      for (int i = k + lane; i < n; i += 32) {
        const double v = A[i * n + i];
        if (v > best) {
          best = v;
          bidx = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ov > best || (ov == best && oi < bidx)) {
          best = ov;
          bidx = oi;
        }
      }
      if (lane == 0) {
        pk_s = bidx;
        stop_s = !(best > tol);
        if (!stop_s && bidx != k) {
          const int t = piv[k];
          piv[k] = piv[bidx];
          piv[bidx] = t;
        }
      }
    }
    __syncthreads();
    if (stop_s) {
      r = k;
      break;
    }
    const int p = pk_s;
    if (p != k) {
      // symmetric exchange of k and p on the trailing lower triangle, and of
      // columns k and p of the rows of R already formed
      if (tid == 0) {
        const double t = A[k * n + k];
        A[k * n + k] = A[p * n + p];
        A[p * n + p] = t;
      }
      for (int i = k + 1 + tid; i < n; i += nt) {
        if (i < p) {  // (i, k) <-> (p, i)
          const double t = A[i * n + k];
          A[i * n + k] = A[p * n + i];
          A[p * n + i] = t;
        } else if (i > p) {  // (i, k) <-> (i, p)
          const double t = A[i * n + k];
          A[i * n + k] = A[i * n + p];
          A[i * n + p] = t;
        }
      }
      for (int i = tid; i < k; i += nt) {  // rows of R already formed
        const double t = A[i * n + k];
        A[i * n + k] = A[i * n + p];
        A[i * n + p] = t;
      }
    }
    if (tid == 0) {  // sqrt and 1 / sqrt from an FP32 seed and two Newton steps
      const double a = A[k * n + k];
      const double y = rsqrt64(a);
      rk_s[0] = a * y;
      rk_s[1] = y;
    }
    __syncthreads();
    for (int j = k + tid; j < n; j += nt) {
      const double v = j == k ? rk_s[0] : A[j * n + k] * rk_s[1];
      rk[j] = v;
    }
    __syncthreads();
    for (int j = k + tid; j < n; j += nt) A[k * n + j] = rk[j];  // row k of R
    // trailing lower triangle: rows i > k, columns k < j <= i
    for (int i = k + 1 + wid; i < n; i += nt >> 5) {
      const double ri = rk[i];
      for (int j = k + 1 + lane; j <= i; j += 32) A[i * n + j] = fma(-ri, rk[j], A[i * n + j]);
    }
    __syncthreads();
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx - i * n;
    B[idx] = (i < r && j >= i) ? A[idx] : 0.0;
  }
  if (tid == 0) *rank_out = r;
  for (int i = tid; i < n; i += nt) piv_out[i] = piv[i];
}

// One-sided Jacobi on the columns of B (n <= 128), all sweeps in one launch
// of one thread-block cluster of C = ceil(n / 8) CTAs, by blocks: the
// columns form nb = 2 C blocks of four, block j held in CTA j % C (slot
// j / C).  A sweep is a round-robin tournament of the blocks (nb - 1
// rounds); in a round, CTA c takes the pair of blocks rr_pair(nb, rd, c),
// copies both into its own shared memory through distributed shared
// memory, rotates the 16 pairs across the two blocks (and, in the sweep's
// first round, the 6 pairs within each block) in warp-local inner rounds of
// 4 disjoint pairs, 8 lanes per pair, and writes the blocks back; one
// cluster barrier ends the round.  Every column pair meets once per sweep.
// The squared column norms are formed at the start of each sweep and carried
// through the rotations (a' = cs^2 a - 2 cs sn g + sn^2 c, and likewise c'),
// so a pair costs one inner product.  Every CTA runs the same number of
// rounds and barriers: after a sweep all read the same rotation flag (kept
// in CTA 0, one per sweep parity) and stop together; at most max_sweeps.
constexpr int kBjCols = 4;     // columns per block
constexpr int kBjMaxN = 128;   // rows (and columns) at most
constexpr int kBjThreads = kBjMaxN;  // one thread per row when blocks move; 4 warps

// Rotate columns X, Y (length n, in this CTA's shared memory) with carried
// squared norms *na, *nc by one warp (lane l holds rows l + 32 u); returns
// whether a rotation was applied.  A warp-wide FP64 instruction occupies an
// SM sub-partition for 64 cycles, so each of the CTA's four warps takes one
// pair and the scalar work per pair is kept to a few FP64 instructions.
HY_DEV bool bj_rotate(double* X, double* Y, double* na, double* nc, int n, int lane, double tol) {
  constexpr int kPer = kBjMaxN / 32;
  double xv[kPer], yv[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = lane + 32 * u;
    xv[u] = i < n ? X[i] : 0.0;
    yv[u] = i < n ? Y[i] : 0.0;
  }
  const double a = *na, c = *nc;
  double g = xv[0] * yv[0];
#pragma unroll
  for (int u = 1; u < kPer; ++u) g = fma(xv[u], yv[u], g);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
  if (!(g * g > tol * tol * (a * c) && a > 0.0 && c > 0.0)) return false;
  // Angle in FP32 (any angle near the optimum converges): t = tan(theta),
  // cs = (1 + t^2)^{-1/2}, sn = cs t.  The rotation is made orthogonal to
  // FP64 precision by scaling (cs, sn) with q^{-1/2}, q = cs^2 + sn^2 =
  // 1 + e (|e| < 1e-6, exact squares of FP32 values): q^{-1/2} = 1 - e/2 +
  // 3e^2/8 to within e^3.
  const float df = (float)(c - a), g2 = (float)(2.0 * g);
  const float sc = fmaxf(fabsf(df), fabsf(g2));
  const float uu = df / sc, vv = g2 / sc;
  const float tf = copysignf(1.f, uu) * vv / (fabsf(uu) + sqrtf(fmaf(uu, uu, vv * vv)));
  double cs, sn, tt;
  if (tf != 0.f && isfinite(tf)) {
    tt = (double)tf;
    const float c32 = rsqrtf(fmaf(tf, tf, 1.f));
    const double c0 = (double)c32, s0 = (double)(c32 * tf);
    const double e = fma(c0, c0, s0 * s0) - 1.0;
    const double rq = 1.0 + fma(0.375 * e, e, -0.5 * e);
    cs = c0 * rq;
    sn = s0 * rq;
  } else {  // out of FP32 range: FP64 formulas
    const double zeta = (c - a) / (2.0 * g);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
    cs = 1.0 / sqrt(fma(t, t, 1.0));
    sn = cs * t;
    tt = t;
  }
#pragma unroll
  for (int u2 = 0; u2 < kPer; ++u2) {
    const int i = lane + 32 * u2;
    if (i < n) {
      X[i] = fma(cs, xv[u2], -sn * yv[u2]);
      Y[i] = fma(sn, xv[u2], cs * yv[u2]);
    }
  }
  // squared norms after the rotation, a - t g and c + t g: exact for the
  // optimal angle, within the FP32 angle's error otherwise; they only steer
  // the rest of the sweep (recomputed at each sweep, and the eigenvalues are
  // formed from the final columns)
  if (lane == 0) {
    *na = fma(-tt, g, a);
    *nc = fma(tt, g, c);
  }
  return true;
}

__global__ void __launch_bounds__(kBjThreads, 1) k_osj_block(double* __restrict__ B, int n,
                                                          const int* __restrict__ rank,
                                                          double tol, int max_sweeps,
                                                          int* __restrict__ sweeps_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double hcol[2][kBjCols][kBjMaxN];  // home blocks me (slot 0), me + C (slot 1)
  __shared__ double hnrm[2][kBjCols];
  __shared__ double wcol[2][kBjCols][kBjMaxN];  // the round's pair of blocks
  __shared__ double wnrm[2][kBjCols];
  __shared__ int rot_flag[2];
  __shared__ int rot_local;
  const int C = (int)cl.num_blocks(), me = (int)cl.block_rank();
  const int nb = 2 * C;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = blockDim.x >> 5;
  const int r = *rank;
  // thread t owns row t of every block it moves (blockDim = kBjMaxN rows)
  const int row = tid;
#pragma unroll
  for (int k = 0; k < 2 * kBjCols; ++k) {
    const int sl = k / kBjCols, c = k % kBjCols;
    const int j = kBjCols * (me + C * sl) + c;
    hcol[sl][c][row] = (j < r && row < n) ? B[(int64_t)j * n + row] : 0.0;
  }
  if (tid < 2) rot_flag[tid] = 0;
  cl.sync();
  int* flag0 = cl.map_shared_rank(&rot_flag[0], 0);
  int sw = 0;
  for (; sw < max_sweeps; ++sw) {
    // squared norms of the home columns (one warp per column)
    for (int k = wid; k < 2 * kBjCols; k += nw) {
      const int sl = k / kBjCols, c = k % kBjCols;
      double a = 0.0;
      for (int i = lane; i < n; i += 32) a = fma(hcol[sl][c][i], hcol[sl][c][i], a);
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) hnrm[sl][c] = a;
    }
    if (tid == 0) rot_local = 0;
    cl.sync();
    for (int rd = 0; rd < nb - 1; ++rd) {
      int pb, qb;
      rr_pair(nb, rd, me, pb, qb);
      // the two blocks (and their norms) in their home CTAs
      double(*hp)[kBjMaxN] = cl.map_shared_rank(hcol[pb / C], (unsigned)(pb % C));
      double(*hq)[kBjMaxN] = cl.map_shared_rank(hcol[qb / C], (unsigned)(qb % C));
      double* np_ = cl.map_shared_rank(hnrm[pb / C], (unsigned)(pb % C));
      double* nq_ = cl.map_shared_rank(hnrm[qb / C], (unsigned)(qb % C));
      {  // gather: all eight remote loads of a thread are issued before any is used
        double v[2 * kBjCols];
#pragma unroll
        for (int c = 0; c < kBjCols; ++c) {
          v[c] = hp[c][row];
          v[kBjCols + c] = hq[c][row];
        }
#pragma unroll
        for (int c = 0; c < kBjCols; ++c) {
          wcol[0][c][row] = v[c];
          wcol[1][c][row] = v[kBjCols + c];
        }
      }
      if (tid < 2 * kBjCols) {
        const int s2 = tid / kBjCols, c = tid % kBjCols;
        wnrm[s2][c] = s2 == 0 ? np_[c] : nq_[c];
      }
      __syncthreads();
      // inner rounds of four disjoint pairs, one per warp
      bool rot = false;
      if (rd == 0) {
        // pairs within each block: (0,1)(2,3), (0,2)(1,3), (0,3)(1,2); warp
        // w takes block w / 2, pair w % 2
        const int wx[3][2] = {{0, 2}, {0, 1}, {0, 1}}, wy[3][2] = {{1, 3}, {2, 3}, {3, 2}};
        const int s2 = wid >> 1, h = wid & 1;
        for (int t = 0; t < 3; ++t) {
          const int x = wx[t][h], y = wy[t][h];
          rot |= bj_rotate(wcol[s2][x], wcol[s2][y], &wnrm[s2][x], &wnrm[s2][y], n, lane, tol);
          __syncthreads();
        }
      }
      // pairs across the two blocks: warp w takes column w of the first and
      // column (w + t) mod 4 of the second, t = 0..3
      for (int t = 0; t < kBjCols; ++t) {
        const int y = (wid + t) % kBjCols;
        rot |= bj_rotate(wcol[0][wid], wcol[1][y], &wnrm[0][wid], &wnrm[1][y], n, lane, tol);
        __syncthreads();
      }
      if (rot && lane == 0) rot_local = 1;
      __syncthreads();
      // write the two blocks back to their homes
#pragma unroll
      for (int c = 0; c < kBjCols; ++c) {
        hp[c][row] = wcol[0][c][row];
        hq[c][row] = wcol[1][c][row];
      }
      if (tid < 2 * kBjCols) {
        const int s2 = tid / kBjCols, c = tid % kBjCols;
        (s2 == 0 ? np_ : nq_)[c] = wnrm[s2][c];
      }
      cl.sync();
    }
    if (tid == 0 && rot_local) atomicOr(flag0 + (sw & 1), 1);
    cl.sync();
    const int rotated = *((volatile int*)(flag0 + (sw & 1)));
    cl.sync();  // everyone has read this sweep's flag before it is reused
    if (me == 0 && tid == 0) rot_flag[(sw + 1) & 1] = 0;
    cl.sync();
    if (!rotated) break;
  }
#pragma unroll
  for (int k = 0; k < 2 * kBjCols; ++k) {
    const int sl = k / kBjCols, c = k % kBjCols;
    const int j = kBjCols * (me + C * sl) + c;
    if (j < r && row < n) B[(int64_t)j * n + row] = hcol[sl][c][row];
  }
  if (sweeps_out && me == 0 && tid == 0) *sweeps_out = sw < max_sweeps ? sw + 1 : max_sweeps;
}

// ---- FP32 preconditioning sweeps of the block one-sided Jacobi -------------
//
// Most of the Jacobi sweeps only bring the columns near orthogonality, which
// FP32 does as well as FP64 at a fraction of the cost: a warp-wide FP64
// instruction holds an SM sub-partition for 64 cycles, an FP32 one about
// one.  So B (the columns of R^T) is first rotated in FP32, with the
// rotations accumulated in J (n x n, FP32, from the identity), until no
// pair rotates at the FP32 tolerance; J is then made orthogonal to FP64
// precision by two Newton-Schulz steps J <- J (3 I - J^T J) / 2 (from
// |J^T J - I| ~ 1e-6: 1e-12, then rounding), B <- B J in FP64, and the FP64
// sweeps finish from there (typically two, and the one that finds no
// rotation).  B J has the same Gram B B^T up to the rounding of the product
// (eps |B| absolute), so the eigenvectors and eigenvalues are those of the
// same matrix.
HY_DEV bool bj_rotate32(float* X, float* Y, float* JX, float* JY, float* na, float* nc, int n,
                        int lane, float tol) {
  constexpr int kPer = kBjMaxN / 32;
  float xv[kPer], yv[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = lane + 32 * u;
    xv[u] = i < n ? X[i] : 0.f;
    yv[u] = i < n ? Y[i] : 0.f;
  }
  const float a = *na, c = *nc;
  float g = xv[0] * yv[0];
#pragma unroll
  for (int u = 1; u < kPer; ++u) g = fmaf(xv[u], yv[u], g);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
  if (!(g * g > tol * tol * (a * c) && a > 0.f && c > 0.f)) return false;
  const float df = c - a, g2 = 2.f * g;
  const float sc = fmaxf(fabsf(df), fabsf(g2));
  const float uu = df / sc, vv = g2 / sc;
  const float t = copysignf(1.f, uu) * vv / (fabsf(uu) + sqrtf(fmaf(uu, uu, vv * vv)));
  const float cs = rsqrtf(fmaf(t, t, 1.f)), sn = cs * t;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = lane + 32 * u;
    if (i < n) {
      X[i] = fmaf(cs, xv[u], -sn * yv[u]);
      Y[i] = fmaf(sn, xv[u], cs * yv[u]);
      const float jx = JX[i], jy = JY[i];
      JX[i] = fmaf(cs, jx, -sn * jy);
      JY[i] = fmaf(sn, jx, cs * jy);
    }
  }
  if (lane == 0) {
    *na = fmaf(-t, g, a);
    *nc = fmaf(t, g, c);
  }
  return true;
}

// The FP32 sweeps in one thread-block cluster, with the same layout and
// tournament as k_osj_block: B32 and J32 (n x n, column j at + j n, FP32)
// in, rotated in place.
__global__ void __launch_bounds__(kBjThreads, 1) k_osj_block32(float* __restrict__ B32,
                                                            float* __restrict__ J32, int n,
                                                            const int* __restrict__ rank,
                                                            float tol, int max_sweeps) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ float hcol[2][2 * kBjCols][kBjMaxN];  // home blocks: X columns, then J columns
  __shared__ float hnrm[2][kBjCols];
  __shared__ float wcol[2][2 * kBjCols][kBjMaxN];  // the round's pair of blocks
  __shared__ float wnrm[2][kBjCols];
  __shared__ int rot_flag[2];
  __shared__ int rot_local;
  const int C = (int)cl.num_blocks(), me = (int)cl.block_rank();
  const int nb = 2 * C;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = blockDim.x >> 5;
  const int r = *rank;
  const int row = tid;
#pragma unroll
  for (int k = 0; k < 2 * kBjCols; ++k) {
    const int sl = k / kBjCols, c = k % kBjCols;
    const int j = kBjCols * (me + C * sl) + c;
    hcol[sl][c][row] = (j < r && row < n) ? B32[(int64_t)j * n + row] : 0.f;
    hcol[sl][kBjCols + c][row] = (j < n && row < n) ? J32[(int64_t)j * n + row] : 0.f;
  }
  if (tid < 2) rot_flag[tid] = 0;
  cl.sync();
  int* flag0 = cl.map_shared_rank(&rot_flag[0], 0);
  for (int sw = 0; sw < max_sweeps; ++sw) {
    for (int k = wid; k < 2 * kBjCols; k += nw) {
      const int sl = k / kBjCols, c = k % kBjCols;
      float a = 0.f;
      for (int i = lane; i < n; i += 32) a = fmaf(hcol[sl][c][i], hcol[sl][c][i], a);
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) hnrm[sl][c] = a;
    }
    if (tid == 0) rot_local = 0;
    cl.sync();
    for (int rd = 0; rd < nb - 1; ++rd) {
      int pb, qb;
      rr_pair(nb, rd, me, pb, qb);
      float(*hp)[kBjMaxN] = cl.map_shared_rank(hcol[pb / C], (unsigned)(pb % C));
      float(*hq)[kBjMaxN] = cl.map_shared_rank(hcol[qb / C], (unsigned)(qb % C));
      float* np_ = cl.map_shared_rank(hnrm[pb / C], (unsigned)(pb % C));
      float* nq_ = cl.map_shared_rank(hnrm[qb / C], (unsigned)(qb % C));
      {
        float v[4 * kBjCols];
#pragma unroll
        for (int c = 0; c < 2 * kBjCols; ++c) {
          v[c] = hp[c][row];
          v[2 * kBjCols + c] = hq[c][row];
        }
#pragma unroll
        for (int c = 0; c < 2 * kBjCols; ++c) {
          wcol[0][c][row] = v[c];
          wcol[1][c][row] = v[2 * kBjCols + c];
        }
      }
      if (tid < 2 * kBjCols) {
        const int s2 = tid / kBjCols, c = tid % kBjCols;
        wnrm[s2][c] = s2 == 0 ? np_[c] : nq_[c];
      }
      __syncthreads();
      bool rot = false;
      if (rd == 0) {
        const int wx[3][2] = {{0, 2}, {0, 1}, {0, 1}}, wy[3][2] = {{1, 3}, {2, 3}, {3, 2}};
        const int s2 = wid >> 1, h = wid & 1;
        for (int t = 0; t < 3; ++t) {
          const int x = wx[t][h], y = wy[t][h];
          rot |= bj_rotate32(wcol[s2][x], wcol[s2][y], wcol[s2][kBjCols + x],
                             wcol[s2][kBjCols + y], &wnrm[s2][x], &wnrm[s2][y], n, lane, tol);
          __syncthreads();
        }
      }
      for (int t = 0; t < kBjCols; ++t) {
        const int y = (wid + t) % kBjCols;
        rot |= bj_rotate32(wcol[0][wid], wcol[1][y], wcol[0][kBjCols + wid], wcol[1][kBjCols + y],
                           &wnrm[0][wid], &wnrm[1][y], n, lane, tol);
        __syncthreads();
      }
      if (rot && lane == 0) rot_local = 1;
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 2 * kBjCols; ++c) {
        hp[c][row] = wcol[0][c][row];
        hq[c][row] = wcol[1][c][row];
      }
      if (tid < 2 * kBjCols) {
        const int s2 = tid / kBjCols, c = tid % kBjCols;
        (s2 == 0 ? np_ : nq_)[c] = wnrm[s2][c];
      }
      cl.sync();
    }
    if (tid == 0 && rot_local) atomicOr(flag0 + (sw & 1), 1);
    cl.sync();
    const int rotated = *((volatile int*)(flag0 + (sw & 1)));
    cl.sync();
    if (me == 0 && tid == 0) rot_flag[(sw + 1) & 1] = 0;
    cl.sync();
    if (!rotated) break;
  }
#pragma unroll
  for (int k = 0; k < 2 * kBjCols; ++k) {
    const int sl = k / kBjCols, c = k % kBjCols;
    const int j = kBjCols * (me + C * sl) + c;
    if (j < n && row < n) {
      B32[(int64_t)j * n + row] = hcol[sl][c][row];
      J32[(int64_t)j * n + row] = hcol[sl][kBjCols + c][row];
    }
  }
}

// B32 = (float) B on the first r columns (zero beyond), J32 = I (n x n)
__global__ void k_osj32_init(const double* __restrict__ B, float* __restrict__ B32,
                             float* __restrict__ J32, int n, const int* __restrict__ rank) {
  const int r = *rank;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += gridDim.x * blockDim.x) {
    B32[idx] = idx / n < r ? (float)B[idx] : 0.f;
    J32[idx] = (idx % n) == (idx / n) ? 1.f : 0.f;
  }
}

// B = (columns < r of) B kept, beyond r zeroed, for the product B J
__global__ void k_zero_beyond_rank(double* __restrict__ B, int n, const int* __restrict__ rank) {
  const int r = *rank;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += gridDim.x * blockDim.x)
    if (idx / n >= r) B[idx] = 0.0;
}

// C = op(A) B for n x n column-major FP64 matrices (op: A or A^T; A may be
// FP32), each thread one entry, the sum in four chains; plus alpha I when
// asked (C = alpha I + beta op(A) B).
template <typename TA, bool TRANS>
__global__ void k_gemm_nn64(const TA* __restrict__ A, const double* __restrict__ B,
                            double* __restrict__ Cm, int n, double alpha, double beta) {
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  if (i >= n || j >= n) return;
  double p[4] = {0.0, 0.0, 0.0, 0.0};
  int k = 0;
  for (; k + 3 < n; k += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double a = TRANS ? (double)A[(int64_t)i * n + k + u] : (double)A[(int64_t)(k + u) * n + i];
      p[u] = fma(a, B[(int64_t)j * n + k + u], p[u]);
    }
  }
  for (; k < n; ++k) {
    const double a = TRANS ? (double)A[(int64_t)i * n + k] : (double)A[(int64_t)k * n + i];
    p[0] = fma(a, B[(int64_t)j * n + k], p[0]);
  }
  Cm[(int64_t)j * n + i] = (i == j ? alpha : 0.0) + beta * ((p[0] + p[1]) + (p[2] + p[3]));
}

__global__ void k_f32_to_f64(const float* __restrict__ a, double* __restrict__ b, int n) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
    b[idx] = (double)a[idx];
}

// lam[j] = |b_j|^2 and V[:, j] = Pi b_j / |b_j| for j < r; zero beyond.
__global__ void k_osj_finish(const double* __restrict__ B, int n, const int* __restrict__ rank,
                             const int* __restrict__ piv, double* __restrict__ lam,
                             double* __restrict__ V) {
  const int j = blockIdx.x;
  const int r = *rank;
  double s = 0.0;
  if (j < r)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double x = B[(int64_t)j * n + i];
      s = fma(x, x, s);
    }
  s = block_sum(s);
  const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  if (threadIdx.x == 0) lam[j] = j < r ? s : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    V[(int64_t)j * n + piv[i]] = j < r ? B[(int64_t)j * n + i] * inv : 0.0;
}

// G (n x n, ld n) -> lam (n), V (n x n column-major).  buf: n * n doubles
// and 2 * kEigMaxN ints.  flag (device, 5 ints, nullable): flag[4] = the
// sweeps the one-sided Jacobi ran.  With host_rank (pinned) the numerical
// rank is read back (one synchronisation).  Returns 0, or -1 on a CUDA error.
size_t psd_eig_scratch_doubles(int n) { return (size_t)5 * n * n + kEigMaxN + 64; }

int run_psd_eig(const double* G, int n, double* V, double* lam, double* buf, int* flag,
                int* host_flag, int max_sweeps, cudaStream_t s, int* host_rank, bool fp32_pre) {
  if (n > kEigMaxN) return -1;
  double* B = buf;
  int* piv = reinterpret_cast<int*>(buf + (size_t)n * n);
  int* rank = piv + kEigMaxN;
  const size_t smem = sizeof(double) * (size_t)n * n;
  smem_at_least((const void*)k_pchol, smem);
  k_pchol<<<1, 1024, smem, HY_S(s)>>>(G, n, n, B, piv, rank);
  (void)host_flag;
  const double tol = 1e-14;
  if (n > kBjMaxN) return -1;
  const int C = (n + 2 * kBjCols - 1) / (2 * kBjCols);  // two blocks of four per CTA
  if (fp32_pre && n >= 32) {
    // FP32 sweeps with the rotations accumulated, J made orthogonal in FP64
    // (two Newton-Schulz steps), B <- B J; the FP64 sweeps finish below
    float* B32 = reinterpret_cast<float*>(buf + (size_t)n * n + kEigMaxN);
    float* J32 = B32 + (size_t)n * n;
    double* J = reinterpret_cast<double*>(J32 + (size_t)n * n);
    double* T1 = J + (size_t)n * n;
    double* T2 = T1 + (size_t)n * n;
    const int g = (n * n + 255) / 256;
    k_osj32_init<<<g, 256, 0, HY_S(s)>>>(B, B32, J32, n, rank);
    cudaFuncSetAttribute(k_osj_block32, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(C);
    lc.blockDim = dim3(kBjThreads);
    lc.dynamicSmemBytes = 0;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    ::hy::count_launch();
    if (cudaLaunchKernelEx(&lc, k_osj_block32, B32, J32, n, (const int*)rank, 1e-5f, 12) !=
        cudaSuccess)
      return -1;
    k_f32_to_f64<<<g, 256, 0, HY_S(s)>>>(J32, J, n * n);
    const dim3 gb((n + 15) / 16, (n + 15) / 16), tb(16, 16);
    for (int it = 0; it < 2; ++it) {
      k_gemm_nn64<double, true><<<gb, tb, 0, HY_S(s)>>>(J, J, T1, n, 1.5, -0.5);
      k_gemm_nn64<double, false><<<gb, tb, 0, HY_S(s)>>>(J, T1, T2, n, 0.0, 1.0);
      double* t = J;
      J = T2;
      T2 = t;
    }
    k_zero_beyond_rank<<<g, 256, 0, HY_S(s)>>>(B, n, rank);
    k_gemm_nn64<double, false><<<gb, tb, 0, HY_S(s)>>>(B, J, T1, n, 0.0, 1.0);
    cudaMemcpyAsync(B, T1, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, s);
  }
  cudaFuncSetAttribute(k_osj_block, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(C);
  lc.blockDim = dim3(kBjThreads);
  lc.dynamicSmemBytes = 0;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  ::hy::count_launch();
  if (cudaLaunchKernelEx(&lc, k_osj_block, B, n, (const int*)rank, tol, max_sweeps,
                         flag ? flag + 4 : (int*)nullptr) != cudaSuccess)
    return -1;
  const int sw = 0;
  k_osj_finish<<<n, 128, 0, HY_S(s)>>>(B, n, rank, piv, lam, V);
  if (host_rank) {
    cudaMemcpyAsync(host_rank, rank, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  }
  return sw;
}

// Order eigenpairs (lam[0..n), columns of V; V = NULL means the identity)
// by descending eigenvalue into
// sig (sqrt(max(lam, 0))) and perm; m_eff by the rank rule
// sigma_j > pod_tol*sigma_1 and sigma_j > pod_abs*sqrt(xraw2); coefficient
// matrix C (w x m_eff, row-major ldc = m) = V_perm / sigma.
template <typename T>
__global__ void k_pod_coeffs(const double* __restrict__ lam, const double* __restrict__ V, int n,
                             int w, int m, double pod_tol, double pod_abs,
                             const double* __restrict__ xraw2, double* __restrict__ sig_out,
                             int* m_eff_out, T* __restrict__ C) {
  __shared__ int perm[256];
  __shared__ double sg[256];
  __shared__ unsigned long long key[256];
  __shared__ int me;
  for (int i = threadIdx.x; i < w; i += blockDim.x) key[i] = dkey(lam[i]);
  __syncthreads();
  for (int j = threadIdx.x; j < w; j += blockDim.x) {  // descending rank, ties by index
    int r = 0;
    for (int i = 0; i < w; ++i) r += (key[i] > key[j]) || (key[i] == key[j] && i < j);
    perm[r] = j;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < w; i += blockDim.x) {
    const double l = lam[perm[i]];
    sg[i] = sqrt(l > 0.0 ? l : 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double floor_abs = pod_abs * sqrt(*xraw2);
    int k = 0;
    for (int i = 0; i < m && i < w; ++i)
      if (sg[i] > pod_tol * sg[0] && sg[i] > floor_abs) ++k;
    me = k;
    *m_eff_out = k;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < w; i += blockDim.x)
    if (sig_out) sig_out[i] = sg[i];
  for (int idx = threadIdx.x; idx < w * m; idx += blockDim.x) {
    const int i = idx / m, j = idx % m;
    const double vij = V ? V[(int64_t)perm[j] * n + i] : (perm[j] == i ? 1.0 : 0.0);
    C[idx] = j < me ? (T)(vij / sg[j]) : (T)0;
  }
}

template <typename T>
void launch_pod_coeffs(const double* lam, const double* V, int n, int w, int m, double pod_tol,
                       double pod_abs, const double* xraw2, double* sig_out, int* m_eff_out,
                       T* C, cudaStream_t s) {
  k_pod_coeffs<T><<<1, 256, 0, HY_S(s)>>>(lam, V, n, w, m, pod_tol, pod_abs, xraw2, sig_out, m_eff_out,
                                    C);
}

// Phi[:, j] = sum_i (ring[win[i]] - psi) C[i][j]  (j < m_eff), and
// psi_next = mean of the window slots, in one pass over the window.  One
// row per thread; the snapshot values of 16 window slots are loaded before
// they are used, so each thread keeps 16 independent loads in flight (the
// kernel is otherwise latency-bound), and coefficients come four at a time
// from shared memory (rows of C padded to MMAX).
template <typename T, int MMAX>
__global__ void __launch_bounds__(256, 2) k_form_phi(const T* __restrict__ ring, int64_t N,
                                                     const int* __restrict__ win, int w,
                                                     const T* __restrict__ psi,
                                                     const T* __restrict__ C, int m,
                                                     const int* __restrict__ m_eff_dev,
                                                     T* __restrict__ phi, T* __restrict__ psi_next) {
  constexpr int U = 16;
  extern __shared__ unsigned char smraw[];
  T* Cs = reinterpret_cast<T*>(smraw);  // w x MMAX, zero padded
  __shared__ int ws[256];
  const int me = *m_eff_dev;
  for (int i = threadIdx.x; i < w * MMAX; i += blockDim.x) {
    const int r = i / MMAX, j = i % MMAX;
    Cs[i] = j < m && j < me ? C[r * m + j] : (T)0;
  }
  for (int i = threadIdx.x; i < w; i += blockDim.x) ws[i] = win[i];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    T acc[MMAX];
#pragma unroll
    for (int j = 0; j < MMAX; ++j) acc[j] = (T)0;
    const T pr = psi[r];
    T sum = (T)0, comp = (T)0;  // Kahan-compensated window sum
    for (int i0 = 0; i0 < w; i0 += U) {
      T g[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        g[u] = i0 + u < w ? __ldg(ring + (int64_t)ws[i0 + u] * N + r) : (T)0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (i0 + u < w) {
          const T yk = g[u] - comp, tk = sum + yk;
          comp = (tk - sum) - yk;
          sum = tk;
          const T x = g[u] - pr;
          const T* Ci = Cs + (i0 + u) * MMAX;
#pragma unroll
          for (int j = 0; j < MMAX; j += 4) {
            T cv[4];
            if (sizeof(T) == 4) {
              const float4 q = *reinterpret_cast<const float4*>(Ci + j);
              cv[0] = q.x; cv[1] = q.y; cv[2] = q.z; cv[3] = q.w;
            } else {
              cv[0] = Ci[j]; cv[1] = Ci[j + 1]; cv[2] = Ci[j + 2]; cv[3] = Ci[j + 3];
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[j + v] = fma(x, cv[v], acc[j + v]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < MMAX; ++j)
      if (j < me) phi[(int64_t)j * N + r] = acc[j];
    psi_next[r] = sum / (T)w;
  }
}

// FP32, m > 16: the same product as a register-tiled SGEMM.  A CTA takes
// 128-row tiles of the window: the raw values (w x 128, k-major) are staged
// in shared memory, one thread per row forms the Kahan window mean and
// centres the row in place, then each thread accumulates 8 rows x CT
// columns of Phi (CT = MM / 16), reading 8 centred values and CT
// coefficients from shared memory per window step (8 CT FMAs per 2 + CT/4
// shared loads).
template <int MM>
__global__ void __launch_bounds__(256, 2) k_form_phi_tiled(
    const float* __restrict__ ring, int64_t N, const int* __restrict__ win, int w,
    const float* __restrict__ psi, const float* __restrict__ C, int m,
    const int* __restrict__ m_eff_dev, float* __restrict__ phi, float* __restrict__ psi_next) {
  constexpr int TR = 128;
  constexpr int CT = MM / 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* Xs = reinterpret_cast<float*>(smraw);  // w x TR
  float* Cs = Xs + w * TR;                      // w x MM, zero padded
  __shared__ int ws[128];
  const int tid = threadIdx.x;
  const int me = *m_eff_dev;
  for (int i = tid; i < w * MM; i += blockDim.x) {
    const int r = i / MM, j = i % MM;
    Cs[i] = j < m && j < me ? C[r * m + j] : 0.f;
  }
  for (int i = tid; i < w; i += blockDim.x) ws[i] = win[i];
  const int rg = tid >> 4, cg = tid & 15;
  const bool vec = (N & 3) == 0;
  for (int64_t base = (int64_t)blockIdx.x * TR; base < N; base += (int64_t)gridDim.x * TR) {
    __syncthreads();  // Cs/ws ready; the previous tile's Xs fully consumed
    // stage the raw values: all (at most 16) loads of a thread in flight
    // before the first store
    {
      float4 buf[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = tid + u * 256;
        if (idx < w * (TR / 4)) {
          const int k = idx >> 5, q = idx & 31;
          const int64_t r0 = base + 4 * q;
          const float* src = ring + (int64_t)ws[k] * N + r0;
          if (vec && r0 + 3 < N) {
            buf[u] = __ldg(reinterpret_cast<const float4*>(src));
          } else {
            buf[u].x = r0 < N ? src[0] : 0.f;
            buf[u].y = r0 + 1 < N ? src[1] : 0.f;
            buf[u].z = r0 + 2 < N ? src[2] : 0.f;
            buf[u].w = r0 + 3 < N ? src[3] : 0.f;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = tid + u * 256;
        if (idx < w * (TR / 4))
          *reinterpret_cast<float4*>(Xs + (idx >> 5) * TR + 4 * (idx & 31)) = buf[u];
      }
    }
    __syncthreads();
    {
      // two threads per row, each over half of the window: Kahan partial
      // sums of the raw values, then the row is centred in place
      __shared__ float part_s[2][TR], part_c[2][TR];
      const int row = tid & (TR - 1), half = tid >> 7;
      const int64_t r = base + row;
      const float pr = r < N ? psi[r] : 0.f;
      const int k0 = half ? w / 2 : 0, k1 = half ? w : w / 2;
      float sum = 0.f, comp = 0.f;
      for (int k = k0; k < k1; ++k) {
        const float g = Xs[k * TR + row];
        const float yk = g - comp, tk = sum + yk;
        comp = (tk - sum) - yk;
        sum = tk;
        Xs[k * TR + row] = g - pr;
      }
      part_s[half][row] = sum;
      part_c[half][row] = comp;
      __syncthreads();
      if (half == 0 && r < N) {
        // (s0 - c0) + (s1 - c1) with the rounding of s0 + s1 recovered
        const float s0 = part_s[0][row], s1 = part_s[1][row];
        const float a = s0 + s1, bb = a - s0;
        const float e = (s0 - (a - bb)) + (s1 - bb);
        psi_next[r] = (a + (e - (part_c[0][row] + part_c[1][row]))) / (float)w;
      }
    }
    __syncthreads();
    float acc[8][CT];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < CT; ++j) acc[i][j] = 0.f;
#pragma unroll 4
    for (int k = 0; k < w; ++k) {
      const float4 xa = *reinterpret_cast<const float4*>(Xs + k * TR + rg * 8);
      const float4 xb = *reinterpret_cast<const float4*>(Xs + k * TR + rg * 8 + 4);
      const float x[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
      float cv[CT];
      if (CT == 4) {
        const float4 c4 = *reinterpret_cast<const float4*>(Cs + k * MM + cg * CT);
        cv[0] = c4.x;
        cv[1 % CT] = c4.y;
        cv[2 % CT] = c4.z;
        cv[3 % CT] = c4.w;
      } else {
        const float2 c2 = *reinterpret_cast<const float2*>(Cs + k * MM + cg * CT);
        cv[0] = c2.x;
        cv[1 % CT] = c2.y;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < CT; ++j) acc[i][j] = fmaf(x[i], cv[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < CT; ++j) {
      const int col = cg * CT + j;
      if (col >= me) continue;
      float* dst = phi + (int64_t)col * N + base + rg * 8;
      if (vec && base + rg * 8 + 7 < N) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (base + rg * 8 + i < N) dst[i] = acc[i][j];
      }
    }
  }
}

template <typename T>
void launch_form_phi(const T* ring, int64_t N, const int* win, int w, const T* psi, const T* C,
                     int m, const int* m_eff_dev, T* phi, T* psi_next, cudaStream_t s) {
  const int mm = m <= 8 ? 8 : (m <= 16 ? 16 : (m <= 32 ? 32 : 64));
  const size_t smem = sizeof(T) * (size_t)w * mm;
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
#define HY_FORM(MM)                                                                          \
  do {                                                                                       \
    smem_at_least((const void*)k_form_phi<T, MM>, smem);                                    \
    k_form_phi<T, MM><<<(int)blocks, 256, smem, HY_S(s)>>>(ring, N, win, w, psi, C, m, m_eff_dev,  \
                                                     phi, psi_next);                         \
  } while (0)
  if (sizeof(T) == 4 && m > 16) {
    const float* ringf = reinterpret_cast<const float*>(ring);
    const float* psif = reinterpret_cast<const float*>(psi);
    const float* Cf = reinterpret_cast<const float*>(C);
    float* phif = reinterpret_cast<float*>(phi);
    float* pnf = reinterpret_cast<float*>(psi_next);
    const int mt = m <= 32 ? 32 : 64;
    const size_t sm2 = sizeof(float) * (size_t)w * (128 + mt);
    int64_t tiles = (N + 127) / 128;
    if (tiles > 152 * 2) tiles = 152 * 2;
    if (mt == 32) {
      smem_at_least((const void*)k_form_phi_tiled<32>, sm2);
      k_form_phi_tiled<32><<<(int)tiles, 256, sm2, HY_S(s)>>>(ringf, N, win, w, psif, Cf, m,
                                                              m_eff_dev, phif, pnf);
    } else {
      smem_at_least((const void*)k_form_phi_tiled<64>, sm2);
      k_form_phi_tiled<64><<<(int)tiles, 256, sm2, HY_S(s)>>>(ringf, N, win, w, psif, Cf, m,
                                                              m_eff_dev, phif, pnf);
    }
    return;
  }
  if (m <= 8)
    HY_FORM(8);
  else if (m <= 16)
    HY_FORM(16);
  else if (m <= 32)
    HY_FORM(32);
  else
    HY_FORM(64);
#undef HY_FORM
}

// ---------------------------------------------------------------------------
// one-sided (Hestenes) Jacobi SVD of the centred window (FP64 path)
// ---------------------------------------------------------------------------

// X (N x wp, column-major, FP64) = ring[win[i]] - psi, zero columns beyond w.
template <typename T>
__global__ void k_center_window(const T* __restrict__ ring, int64_t N, const int* __restrict__ win,
                                int w, int wp, const T* __restrict__ psi, double* __restrict__ X,
                                double* __restrict__ raw_part) {
  double raw = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N * wp;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N);
    const int64_t r = idx % N;
    if (i < w) {
      const double g = (double)ring[(int64_t)win[i] * N + r];
      raw = fma(g, g, raw);
      X[idx] = g - (double)psi[r];
    } else {
      X[idx] = 0.0;
    }
  }
  raw = block_sum(raw);
  if (threadIdx.x == 0) raw_part[blockIdx.x] = raw;
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double* out) {
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  a = block_sum(a);
  if (threadIdx.x == 0) *out = a;
}

// One round of the one-sided Jacobi SVD of the window: the wp/2 disjoint
// column pairs (p, q) of round r are orthogonalised at once, spread over
// every SM in three launches:
//   k_hj_dots   - partial sums of |x_p|^2, |x_q|^2 and x_p . x_q, kHjBlocks
//                 row slices per pair;
//   k_hj_angles - one warp per pair sums its partials in a fixed order and
//                 forms the rotation (or none: g = 0 or |g| <= tol |x_p||x_q|),
//                 applies it to V;
//   k_hj_apply  - rotates the columns of X, row by row.
constexpr int kHjBlocks = 128;

__global__ void k_hj_dots(const double* __restrict__ X, int64_t N, int wp, int r,
                          double* __restrict__ part) {
  int p, q;
  rr_pair(wp, r, blockIdx.y, p, q);
  const double* xp = X + (int64_t)p * N;
  const double* xq = X + (int64_t)q * N;
  double a = 0.0, b = 0.0, g = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double u = xp[i], v = xq[i];
    a = fma(u, u, a);
    b = fma(v, v, b);
    g = fma(u, v, g);
  }
  a = block_sum(a);
  b = block_sum(b);
  g = block_sum(g);
  if (threadIdx.x == 0) {
    double* o = part + ((int64_t)blockIdx.y * kHjBlocks + blockIdx.x) * 3;
    o[0] = a;
    o[1] = b;
    o[2] = g;
  }
}

__global__ void k_hj_angles(const double* __restrict__ part, int wp, int r, double tol,
                            double* __restrict__ cs, double* __restrict__ V, int* rotated) {
  const int lane = threadIdx.x & 31;
  for (int pair = threadIdx.x >> 5; pair < wp / 2; pair += blockDim.x >> 5) {
  int p, q;
  rr_pair(wp, r, pair, p, q);
  double a = 0.0, b = 0.0, g = 0.0;
  for (int k = lane; k < kHjBlocks; k += 32) {
    const double* o = part + ((int64_t)pair * kHjBlocks + k) * 3;
    a += o[0];
    b += o[1];
    g += o[2];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  g = warp_sum(g);
  double c = 1.0, sn = 0.0;
  const bool rot = !(g == 0.0 || fabs(g) <= tol * sqrt(a * b));
  if (rot) {
    const double zeta = (b - a) / (2.0 * g);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    sn = c * t;
    for (int i = lane; i < wp; i += 32) {
      const double u = V[(int64_t)p * wp + i], v = V[(int64_t)q * wp + i];
      V[(int64_t)p * wp + i] = c * u - sn * v;
      V[(int64_t)q * wp + i] = sn * u + c * v;
    }
    if (lane == 0) *rotated = 1;
  }
  if (lane == 0) {
    cs[2 * pair] = c;
    cs[2 * pair + 1] = rot ? sn : 0.0;
  }
  }
}

__global__ void k_hj_apply(double* __restrict__ X, int64_t N, int wp, int r,
                           const double* __restrict__ cs) {
  const int np = wp / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int pair = 0; pair < np; ++pair) {
      const double sn = cs[2 * pair + 1];
      if (sn == 0.0) continue;
      const double c = cs[2 * pair];
      int p, q;
      rr_pair(wp, r, pair, p, q);
      double* xp = X + (int64_t)p * N;
      double* xq = X + (int64_t)q * N;
      const double u = xp[i], v = xq[i];
      xp[i] = c * u - sn * v;
      xq[i] = sn * u + c * v;
    }
  }
}

size_t hestenes_scratch_doubles(int wp) { return (size_t)(wp / 2) * (kHjBlocks * 3 + 2); }

void launch_hestenes_round(double* X, int64_t N, int wp, double* V, int r, double tol,
                           int* rotated, double* scratch, cudaStream_t s) {
  const int np = wp / 2;
  double* part = scratch;
  double* cs = scratch + (size_t)np * kHjBlocks * 3;
  k_hj_dots<<<dim3(kHjBlocks, np), 256, 0, HY_S(s)>>>(X, N, wp, r, part);
  k_hj_angles<<<1, 32 * (np < 32 ? np : 32), 0, HY_S(s)>>>(part, wp, r, tol, cs, V, rotated);
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_hj_apply<<<(int)blocks, 256, 0, HY_S(s)>>>(X, N, wp, r, cs);
}

__global__ void k_colnorm2(const double* __restrict__ X, int64_t N, double* __restrict__ out) {
  const double* x = X + (int64_t)blockIdx.x * N;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) a = fma(x[i], x[i], a);
  a = block_sum(a);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}




void launch_colnorm2(const double* X, int64_t N, int ncol, double* out, cudaStream_t s) {
  k_colnorm2<<<ncol, 256, 0, HY_S(s)>>>(X, N, out);
}

// Phi[:, j] = X[:, perm_j] / sigma_j for the kept modes; perm and the rank
// come from k_pod_coeffs run on the column norms (lam = squared norms, V = I).
template <typename T>
__global__ void k_phi_from_columns(const double* __restrict__ X, int64_t N, int wp,
                                   const double* __restrict__ C, const int* __restrict__ m_eff,
                                   int m, T* __restrict__ phi) {
  const int me = *m_eff;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N * me;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / N);
    const int64_t r = idx % N;
    // C is the identity-permutation coefficient block: column j has one
    // non-zero 1/sigma_j in row perm_j
    double acc = 0.0;
    for (int i = 0; i < wp; ++i) {
      const double cij = C[(int64_t)i * m + j];
      if (cij != 0.0) acc = X[(int64_t)i * N + r] * cij;
    }
    phi[idx] = (T)acc;
  }
}

template <typename T>
void launch_phi_from_columns(const double* X, int64_t N, int wp, const double* C,
                             const int* m_eff, int m, T* phi, cudaStream_t s) {
  k_phi_from_columns<T><<<152 * 8, 256, 0, HY_S(s)>>>(X, N, wp, C, m_eff, m, phi);
}

// psi_next = mean of the window slots (FP64 path)
template <typename T>
__global__ void k_window_mean(const T* __restrict__ ring, int64_t N, const int* __restrict__ win,
                              int w, T* __restrict__ out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    T acc = (T)0;
    for (int i = 0; i < w; ++i) acc += ring[(int64_t)win[i] * N + r];
    out[r] = acc / (T)w;
  }
}

template <typename T>
void launch_window_mean(const T* ring, int64_t N, const int* win, int w, T* out, cudaStream_t s) {
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_window_mean<T><<<(int)blocks, 256, 0, HY_S(s)>>>(ring, N, win, w, out);
}

// Sign convention: flip column j when its largest-magnitude entry (lowest
// row on ties) is negative.  One CTA per column.
template <typename T>
__global__ void k_sign_fix(T* __restrict__ phi, int64_t N, const int* __restrict__ m_eff) {
  const int j = blockIdx.x;
  if (j >= *m_eff) return;
  T* col = phi + (int64_t)j * N;
  __shared__ double bv[32];
  __shared__ long long bi[32];
  double best = -1.0;
  long long arg = -1;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    const double a = fabs((double)col[i]);
    if (a > best) {
      best = a;
      arg = i;
    }
  }
  // warp then block arg-max (ties -> lowest row)
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oi >= 0 && (arg < 0 || oi < arg))) {
      best = ob;
      arg = oi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    bv[wid] = best;
    bi[wid] = arg;
  }
  __syncthreads();
  __shared__ int flip;
  if (threadIdx.x == 0) {
    double b = -1.0;
    long long a = -1;
    for (int wdx = 0; wdx < (int)(blockDim.x >> 5); ++wdx)
      if (bv[wdx] > b || (bv[wdx] == b && bi[wdx] >= 0 && (a < 0 || bi[wdx] < a))) {
        b = bv[wdx];
        a = bi[wdx];
      }
    flip = (a >= 0 && col[a] < (T)0) ? 1 : 0;
  }
  __syncthreads();
  if (flip)
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) col[i] = -col[i];
}

template <typename T>
void launch_sign_fix(T* phi, int64_t N, int m, const int* m_eff, cudaStream_t s) {
  if (m > 0) k_sign_fix<T><<<m, 1024, 0, HY_S(s)>>>(phi, N, m_eff);
}

#define HY_INST(T)                                                                              \
  template void launch_gappy_pinv<T>(const T*, int64_t, int, const int*, int, double*, int*,    \
                                     cudaStream_t);                                             \
  template void launch_gappy_apply<T>(const double*, int, int, const int*, const T*, const T*,  \
                                      double*, const double*, double*, cudaStream_t,            \
                                      const int*);                                              \
  template void launch_reconstruct<T>(const T*, int64_t, int64_t, int, const double*, const T*, \
                                      const uint32_t*, int, T*, cudaStream_t);                  \
  template void launch_cell_error<T>(const T*, const T*, const T*, int64_t, int, int,           \
                                     const double*, T*, cudaStream_t);                          \
  template void launch_gram_row<T>(const T*, int64_t, int, int, double*, int, double*,          \
                                   cudaStream_t);                                               \
  template void launch_gram_rows2<T>(const T*, int64_t, int, int, int, double*, int, double*,   \
                                     cudaStream_t);                                             \
  template void launch_pod_coeffs<T>(const double*, const double*, int, int, int, double,       \
                                     double, const double*, double*, int*, T*, cudaStream_t);   \
  template void launch_form_phi<T>(const T*, int64_t, const int*, int, const T*, const T*, int, \
                                   const int*, T*, T*, cudaStream_t);                           \
  template void launch_phi_from_columns<T>(const double*, int64_t, int, const double*,          \
                                           const int*, int, T*, cudaStream_t);                  \
  template void launch_window_mean<T>(const T*, int64_t, const int*, int, T*, cudaStream_t);   \
  template void launch_sign_fix<T>(T*, int64_t, int, const int*, cudaStream_t);
HY_INST(float)
HY_INST(double)
#undef HY_INST

template <typename T>
void launch_center_window(const T* ring, int64_t N, const int* win, int w, int wp, const T* psi,
                          double* X, double* raw_part, double* raw_out, cudaStream_t s) {
  const int blocks = 152 * 4;
  k_center_window<T><<<blocks, 256, 0, HY_S(s)>>>(ring, N, win, w, wp, psi, X, raw_part);
  k_sum_parts<<<1, 256, 0, HY_S(s)>>>(raw_part, blocks, raw_out);
}
template void launch_center_window<float>(const float*, int64_t, const int*, int, int,
                                          const float*, double*, double*, double*, cudaStream_t);
template void launch_center_window<double>(const double*, int64_t, const int*, int, int,
                                           const double*, double*, double*, double*,
                                           cudaStream_t);

}  // namespace hy
