// Residual-gated explicit Shapiro filters: Sec. 2.3.4 of the paper.
//
// The order-2n Shapiro filter has the frequency response 1 - sin^{2n}(theta/2);
// its weights times 4^n are (1 2 1), (-1 4 10 4 -1), (1 -6 15 44 15 -6 1).
// It is applied along x, then along y; non-periodic sides use zeroth-order
// extrapolation (ghost = boundary value).  One gate pass keeps the filtered
// value on the cells whose residual measure rho = sum_v |R_v| (BDF1 residual)
// strictly decreases; passes stop when no cell is kept, when the kept
// cells' total decrease is below eps_f times their previous total, or after
// jmax_f passes.
//
// Device-side control: every pass kernel reads a `done` flag and returns at
// once when it is set, so the host enqueues jmax_f passes per order without
// reading anything back.
#include "common.cuh"
#include "internal.h"

namespace hy {

template <int N_>
struct Shapiro;
template <>
struct Shapiro<1> {
  static constexpr int W = 3;
  HY_DEV static double w(int t) { return t == 1 ? 2.0 : 1.0; }
};
template <>
struct Shapiro<2> {
  static constexpr int W = 5;
  HY_DEV static double w(int t) {
    return t == 0 || t == 4 ? -1.0 : (t == 2 ? 10.0 : 4.0);
  }
};
template <>
struct Shapiro<3> {
  static constexpr int W = 7;
  HY_DEV static double w(int t) {
    return t == 0 || t == 6 ? 1.0 : (t == 1 || t == 5 ? -6.0 : (t == 3 ? 44.0 : 15.0));
  }
};

// One direction (AX = 0: x, AX = 1: y) of the order-2n filter for every dof.
template <typename T, int N_, int AX>
__global__ void k_shapiro(DevCfg c, const T* __restrict__ in, T* __restrict__ out,
                          const int* __restrict__ done) {
  if (done && *done) return;
  const bool per = AX == 0 ? c.bc[0] == HYROM_BC_PERIODIC : c.bc[2] == HYROM_BC_PERIODIC;
  const int L = AX == 0 ? c.nx : c.ny;
  const T scale = (T)(N_ == 1 ? 0.25 : (N_ == 2 ? 0.0625 : 0.015625));
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < c.ndof;
       d += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = d / c.nc, cell = d % c.nc;
    const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
    const int pos = AX == 0 ? i : j;
    const T* base = in + v * c.nc;
    T acc = (T)0;
#pragma unroll
    for (int t = 0; t < Shapiro<N_>::W; ++t) {
      int p = pos + t - N_;
      if (per)
        p = imod(p, L);
      else
        p = p < 0 ? 0 : (p >= L ? L - 1 : p);
      const T x = AX == 0 ? base[(int64_t)j * c.nx + p] : base[(int64_t)p * c.nx + i];
      const double wt = Shapiro<N_>::w(t);
      const T term = wt == 1.0 ? x : (wt == -1.0 ? -x : (T)wt * x);
      acc = t == 0 ? term : acc + term;
    }
    out[d] = acc * scale;
  }
}

template <typename T>
void launch_shapiro(const DevCfg& c, int n, const T* in, T* tmp, T* out, const int* done,
                    cudaStream_t s) {
  int64_t blocks = (c.ndof + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const bool twoD = c.ny > 1;
  T* xdst = twoD ? tmp : out;
#define HY_SH(NN)                                                                  \
  do {                                                                             \
    k_shapiro<T, NN, 0><<<(int)blocks, 256, 0, HY_S(s)>>>(c, in, xdst, done);            \
    if (twoD) k_shapiro<T, NN, 1><<<(int)blocks, 256, 0, HY_S(s)>>>(c, tmp, out, done);  \
  } while (0)
  if (n == 1)
    HY_SH(1);
  else if (n == 2)
    HY_SH(2);
  else
    HY_SH(3);
#undef HY_SH
}

// Gate: keep the filtered value where rho_new < rho_old; per-block partial
// (kept count, sum of decreases, sum of old values) for a fixed-order
// reduction.
template <typename T>
__global__ void k_gate(int64_t nc, int nvar, T* __restrict__ q, const T* __restrict__ g,
                       const T* __restrict__ rho_old, const T* __restrict__ rho_new,
                       double* __restrict__ part, const int* __restrict__ done) {
  if (*done) return;
  double cnt = 0.0, dec = 0.0, tot = 0.0;
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < nc;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const T ro = rho_old[cell], rn = rho_new[cell];
    if (rn < ro) {
      for (int v = 0; v < nvar; ++v) q[v * nc + cell] = g[v * nc + cell];
      cnt += 1.0;
      dec += (double)(ro - rn);
      tot += (double)ro;
    }
  }
  cnt = block_sum(cnt);
  dec = block_sum(dec);
  tot = block_sum(tot);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = cnt;
    part[3 * blockIdx.x + 1] = dec;
    part[3 * blockIdx.x + 2] = tot;
  }
}

// ctl[0] = done, ctl[1] = passes run, ctl[2] = cells kept (running total)
__global__ void k_gate_finalize(const double* __restrict__ part, int nblk, double eps_f,
                                int* ctl) {
  if (ctl[0]) return;
  double cnt = 0.0, dec = 0.0, tot = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    cnt += part[3 * i];
    dec += part[3 * i + 1];
    tot += part[3 * i + 2];
  }
  cnt = block_sum(cnt);
  dec = block_sum(dec);
  tot = block_sum(tot);
  if (threadIdx.x == 0) {
    ctl[1] += 1;
    ctl[2] += (int)cnt;
    if (cnt == 0.0 || dec < eps_f * tot) ctl[0] = 1;
  }
}

__global__ void k_set_int(int* p, int v) { *p = v; }

template <typename T>
void launch_filter(const DevCfg& c, const int* orders, int norders, int jmax_f, double eps_f,
                   T* q, const T* qp, int64_t k, T* g, T* tmp, T* rho_old, T* rho_new,
                   double* part, int* ctl, cudaStream_t s) {
  const int nblk = 152 * 4;
  cudaMemsetAsync(ctl, 0, 3 * sizeof(int), s);
  for (int o = 0; o < norders; ++o) {
    k_set_int<<<1, 1, 0, HY_S(s)>>>(ctl, 0);
    launch_cell_residual_skip<T>(c, q, qp, k, rho_old, ctl, s);
    for (int pass = 0; pass < jmax_f; ++pass) {
      launch_shapiro<T>(c, orders[o], q, tmp, g, ctl, s);
      launch_cell_residual_skip<T>(c, g, qp, k, rho_new, ctl, s);
      k_gate<T><<<nblk, 256, 0, HY_S(s)>>>(c.nc, c.nvar, q, g, rho_old, rho_new, part, ctl);
      k_gate_finalize<<<1, 256, 0, HY_S(s)>>>(part, nblk, eps_f, ctl);
      if (pass + 1 < jmax_f) launch_cell_residual_skip<T>(c, q, qp, k, rho_old, ctl, s);
    }
  }
}

template void launch_filter<float>(const DevCfg&, const int*, int, int, double, float*,
                                   const float*, int64_t, float*, float*, float*, float*, double*,
                                   int*, cudaStream_t);
template void launch_filter<double>(const DevCfg&, const int*, int, int, double, double*,
                                    const double*, int64_t, double*, double*, double*, double*,
                                    double*, int*, cudaStream_t);

}  // namespace hy
