// The paper's HDM (Sec. 3.1) on the GPU: second-order MUSCL reconstruction
// of the primitive variables with the minmod limiter, the Roe flux (no
// entropy fix), and the BDF2 scheme of Eq. bdf (a0 = 1/3, a1 = -4/3,
// a2 = 1, beta = 2/3; BDF1 for the first step), each step R_k(q) = 0
// (Eq. hdm) solved by Newton's method with restarted GMRES driven by exact
// Jacobian-vector products (the cost model of the method's speedup, Sec.
// 2.4.2).  The partial HDM of Eq. partial_hdm2 solves the rows of the
// sampled cells with every other cell frozen; its unknowns are compact
// (4 values per sampled cell), so its work is proportional to n_s.
//
// Residual and face states follow one fixed order of operations (the file is
// compiled with -fmad=false): the FP64 residual is the same bits as any
// evaluation of the same expressions in the same order.  The JVP kernels
// evaluate the same expressions on dual numbers (value, derivative), so the
// directional derivative is exact up to rounding; minmod, |.| and the
// comparisons take their branch from the values (at a kink the derivative
// of the branch taken).
//
// Ghost cells (two layers) as in the HDM's other paths: periodic sides wrap,
// outflow sides repeat the boundary cell, shock sides take the exact planar
// shock state at the ghost cell's centre.
#include <math.h>

#include <vector>

#include "common.cuh"
#include "internal.h"

namespace hy {
namespace {

// ---- dual numbers: value and directional derivative -----------------------
struct Dual {
  double v, d;
};
HY_DEV Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
HY_DEV Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
HY_DEV Dual operator-(Dual a) { return {-a.v, -a.d}; }
HY_DEV Dual operator*(Dual a, Dual b) { return {a.v * b.v, fma(a.d, b.v, a.v * b.d)}; }
HY_DEV Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
HY_DEV Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
HY_DEV Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
HY_DEV Dual dsqrt(Dual a) {
  const double s = sqrt(a.v);
  return {s, a.d / (2.0 * s)};
}
HY_DEV Dual dabs(Dual a) { return a.v < 0.0 ? -a : a; }
HY_DEV double val(Dual a) { return a.v; }

HY_DEV double dsqrt(double a) { return sqrt(a); }
HY_DEV double dabs(double a) { return fabs(a); }
HY_DEV double val(double a) { return a; }
template <typename N>
HY_DEV N cst(double c);
template <>
HY_DEV double cst<double>(double c) { return c; }
template <>
HY_DEV Dual cst<Dual>(double c) { return Dual{c, 0.0}; }

template <typename N>
HY_DEV N minmod(N a, N b) {
  if (!(val(a) * val(b) > 0.0)) return cst<N>(0.0);
  return fabs(val(a)) < fabs(val(b)) ? a : b;
}

template <typename N>
HY_DEV void to_prim(const N* q, double g, N* w) {
  const N u = q[1] / q[0], v = q[2] / q[0];
  w[0] = q[0];
  w[1] = u;
  w[2] = v;
  w[3] = (g - 1.0) * (q[3] - (0.5 * q[0]) * (u * u + v * v));
}

template <typename N>
HY_DEV void to_cons(const N* w, double g, N* q) {
  q[0] = w[0];
  q[1] = w[0] * w[1];
  q[2] = w[0] * w[2];
  q[3] = w[3] / (g - 1.0) + (0.5 * w[0]) * (w[1] * w[1] + w[2] * w[2]);
}

template <typename N, int AX>
HY_DEV void phys_flux(const N* q, double g, N* f) {
  const N u = q[1] / q[0], v = q[2] / q[0];
  const N p = (g - 1.0) * (q[3] - (0.5 * q[0]) * (u * u + v * v));
  if (AX == 0) {
    f[0] = q[1];
    f[1] = q[1] * u + p;
    f[2] = q[2] * u;
    f[3] = (q[3] + p) * u;
  } else {
    f[0] = q[2];
    f[1] = q[1] * v;
    f[2] = q[2] * v + p;
    f[3] = (q[3] + p) * v;
  }
}

// Roe flux across a face normal to x (AX = 0) or y (AX = 1)
template <typename N, int AX>
HY_DEV void roe(const N* qL, const N* qR, double g, N* F) {
  const N rL = qL[0], rR = qR[0];
  const N uL = qL[1] / rL, uR = qR[1] / rR;
  const N vL = qL[2] / rL, vR = qR[2] / rR;
  const N pL = (g - 1.0) * (qL[3] - (0.5 * rL) * (uL * uL + vL * vL));
  const N pR = (g - 1.0) * (qR[3] - (0.5 * rR) * (uR * uR + vR * vR));
  const N HL = (qL[3] + pL) / rL, HR = (qR[3] + pR) / rR;
  const N sL = dsqrt(rL), sR = dsqrt(rR);
  const N w = sL + sR;
  const N u = (sL * uL + sR * uR) / w;
  const N v = (sL * vL + sR * vR) / w;
  const N H = (sL * HL + sR * HR) / w;
  const N c = dsqrt((g - 1.0) * (H - 0.5 * (u * u + v * v)));
  const N rho = sL * sR;
  const N un = AX == 0 ? u : v;
  const N dr = rR - rL;
  const N dp = pR - pL;
  const N dun = AX == 0 ? (uR - uL) : (vR - vL);
  const N dut = AX == 0 ? (vR - vL) : (uR - uL);
  const N c2 = (2.0 * c) * c;
  const N a1 = (dp - (rho * c) * dun) / c2;
  const N a3 = (dp + (rho * c) * dun) / c2;
  const N a2 = dr - dp / (c * c);
  const N a4 = rho * dut;
  const N l1 = dabs(un - c), l2 = dabs(un), l3 = dabs(un + c);
  const N one = cst<N>(1.0), zero = cst<N>(0.0) * one;
  N r1[4], r2[4], r3[4], r4[4];
  const N ke = 0.5 * (u * u + v * v);
  if (AX == 0) {
    r1[0] = one; r1[1] = u - c; r1[2] = v; r1[3] = H - u * c;
    r3[0] = one; r3[1] = u + c; r3[2] = v; r3[3] = H + u * c;
    r4[0] = zero; r4[1] = zero; r4[2] = one; r4[3] = v;
  } else {
    r1[0] = one; r1[1] = u; r1[2] = v - c; r1[3] = H - v * c;
    r3[0] = one; r3[1] = u; r3[2] = v + c; r3[3] = H + v * c;
    r4[0] = zero; r4[1] = one; r4[2] = zero; r4[3] = u;
  }
  r2[0] = one; r2[1] = u; r2[2] = v; r2[3] = ke;
  const N b1 = l1 * a1, b2 = l2 * a2, b3 = l3 * a3, b4 = l2 * a4;
  N fL[4], fR[4];
  phys_flux<N, AX>(qL, g, fL);
  phys_flux<N, AX>(qR, g, fR);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const N diss = ((b1 * r1[k] + b2 * r2[k]) + b3 * r3[k]) + b4 * r4[k];
    F[k] = 0.5 * (fL[k] + fR[k]) - 0.5 * diss;
  }
}

// exact planar-shock state at cell (gi, gj) and time t
HY_DEV void shock_cell(const DevCfg& c, int gi, int gj, double t, double* out) {
  const double x = ((double)gi + 0.5) * c.dx;
  const double y = ((double)gj + 0.5) * c.dy;
  const bool post = c.sn0 * x + c.sn1 * y < c.sd0 + c.sspeed * t;
  for (int v = 0; v < 4; ++v) out[v] = post ? c.post[v] : c.pre[v];
}

// State (and direction, for duals) at grid position (gi, gj), which may lie
// up to two layers outside the domain along one axis.
template <typename N>
struct Src;
template <>
struct Src<double> {
  const double* q;
  HY_DEV void at(const DevCfg& c, int gi, int gj, double t, double* out) const {
    int side = -1;
    if (gi < 0 || gi >= c.nx) {
      if (c.bc[0] == HYROM_BC_PERIODIC) gi = imod(gi, c.nx);
      else side = gi < 0 ? 0 : 1;
    } else if (c.ny > 1 && (gj < 0 || gj >= c.ny)) {
      if (c.bc[2] == HYROM_BC_PERIODIC) gj = imod(gj, c.ny);
      else side = gj < 0 ? 2 : 3;
    }
    if (side >= 0 && c.bc[side] == HYROM_BC_SHOCK) {
      shock_cell(c, gi, gj, t, out);
      return;
    }
    gi = gi < 0 ? 0 : (gi >= c.nx ? c.nx - 1 : gi);
    gj = gj < 0 ? 0 : (gj >= c.ny ? c.ny - 1 : gj);
    const int64_t cell = (int64_t)gj * c.nx + gi;
    for (int v = 0; v < 4; ++v) out[v] = q[v * c.nc + cell];
  }
};
template <>
struct Src<Dual> {
  const double* q;
  const double* dq;  // direction on every cell (zero where it does not act)
  HY_DEV void at(const DevCfg& c, int gi, int gj, double t, Dual* out) const {
    int side = -1;
    if (gi < 0 || gi >= c.nx) {
      if (c.bc[0] == HYROM_BC_PERIODIC) gi = imod(gi, c.nx);
      else side = gi < 0 ? 0 : 1;
    } else if (c.ny > 1 && (gj < 0 || gj >= c.ny)) {
      if (c.bc[2] == HYROM_BC_PERIODIC) gj = imod(gj, c.ny);
      else side = gj < 0 ? 2 : 3;
    }
    if (side >= 0 && c.bc[side] == HYROM_BC_SHOCK) {
      double s[4];
      shock_cell(c, gi, gj, t, s);
      for (int v = 0; v < 4; ++v) out[v] = Dual{s[v], 0.0};
      return;
    }
    gi = gi < 0 ? 0 : (gi >= c.nx ? c.nx - 1 : gi);
    gj = gj < 0 ? 0 : (gj >= c.ny ? c.ny - 1 : gj);
    const int64_t cell = (int64_t)gj * c.nx + gi;
    for (int v = 0; v < 4; ++v) out[v] = Dual{q[v * c.nc + cell], dq[v * c.nc + cell]};
  }
};

// MUSCL flux across the face between cells `a` and `a + 1` along axis AX
// (a is the x index for AX = 0, the y index for AX = 1; `o` the other one)
template <typename N, int AX>
HY_DEV void muscl_face(const DevCfg& c, const Src<N>& src, int a, int o, double t, N* F) {
  N w[4][4];  // primitives of cells a-1 .. a+2
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    N qv[4];
    if (AX == 0) src.at(c, a - 1 + s, o, t, qv);
    else src.at(c, o, a - 1 + s, t, qv);
    to_prim(qv, c.gamma, w[s]);
  }
  N wl[4], wr[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const N d0 = w[1][k] - w[0][k], d1 = w[2][k] - w[1][k], d2 = w[3][k] - w[2][k];
    const N sa = minmod(d0, d1), sb = minmod(d1, d2);
    wl[k] = w[1][k] + 0.5 * sa;
    wr[k] = w[2][k] - 0.5 * sb;
  }
  N qL[4], qR[4];
  to_cons(wl, c.gamma, qL);
  to_cons(wr, c.gamma, qR);
  roe<N, AX>(qL, qR, c.gamma, F);
}

// f*(q) at cell (i, j)
template <typename N>
HY_DEV void muscl_rhs_cell(const DevCfg& c, const Src<N>& src, int i, int j, double t, N* out) {
  N Fl[4], Fr[4];
  muscl_face<N, 0>(c, src, i - 1, j, t, Fl);
  muscl_face<N, 0>(c, src, i, j, t, Fr);
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = -(Fr[v] - Fl[v]) / c.dx;
  if (c.ny > 1) {
    N Gb[4], Gt[4];
    muscl_face<N, 1>(c, src, j - 1, i, t, Gb);
    muscl_face<N, 1>(c, src, j, i, t, Gt);
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = out[v] - (Gt[v] - Gb[v]) / c.dy;
  }
}

// cell of compact index idx: cells[idx], or idx itself when cells is null
HY_DEV int64_t cell_of(const int* __restrict__ cells, int64_t idx) {
  return cells ? (int64_t)cells[idx] : idx;
}

// R_k rows of the listed cells (compact SoA: out[v * n + idx]):
//   BDF2: a2 q + a1 q_prev + a0 q_prev2 - (dt beta) f*(q),  BDF1: (q - q_prev) - dt f*(q)
__global__ void k_muscl_residual(DevCfg c, const double* __restrict__ q,
                                 const double* __restrict__ qp, const double* __restrict__ qp2,
                                 double t, const int* __restrict__ cells, int64_t n,
                                 double* __restrict__ out) {
  const Src<double> src{q};
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = cell_of(cells, idx);
    const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
    double f[4];
    muscl_rhs_cell<double>(c, src, i, j, t, f);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double qc = q[v * c.nc + cell], p1 = qp[v * c.nc + cell];
      double R;
      if (qp2) {
        const double p2 = qp2[v * c.nc + cell];
        R = ((1.0 * qc + (-4.0 / 3.0) * p1) + (1.0 / 3.0) * p2) - (c.dt * (2.0 / 3.0)) * f[v];
      } else {
        R = (qc - p1) - c.dt * f[v];
      }
      out[v * n + idx] = R;
    }
  }
}

// J v on the listed rows: a2 v - (dt beta) (d f*/d q) v, with v given on
// every cell (dv, zero where it does not act)
__global__ void k_muscl_jvp(DevCfg c, const double* __restrict__ q, const double* __restrict__ dv,
                            double t, double a2, double dtb, const int* __restrict__ cells,
                            int64_t n, const int* __restrict__ done, double* __restrict__ out) {
  if (done && *done) return;
  const Src<Dual> src{q, dv};
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = cell_of(cells, idx);
    const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
    Dual f[4];
    muscl_rhs_cell<Dual>(c, src, i, j, t, f);
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v * n + idx] = fma(a2, dv[v * c.nc + cell], -dtb * f[v].d);
  }
}

// the filter's residual measure rho_i = sum_v |R_v| on every cell
__global__ void k_muscl_rho(DevCfg c, const double* __restrict__ q, const double* __restrict__ qp,
                            const double* __restrict__ qp2, double t, double* __restrict__ rho) {
  const Src<double> src{q};
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < c.nc;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
    double f[4];
    muscl_rhs_cell<double>(c, src, i, j, t, f);
    double acc = 0.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double qc = q[v * c.nc + cell], p1 = qp[v * c.nc + cell];
      double R;
      if (qp2) {
        const double p2 = qp2[v * c.nc + cell];
        R = ((1.0 * qc + (-4.0 / 3.0) * p1) + (1.0 / 3.0) * p2) - (c.dt * (2.0 / 3.0)) * f[v];
      } else {
        R = (qc - p1) - c.dt * f[v];
      }
      acc = v == 0 ? fabs(R) : acc + fabs(R);
    }
    rho[cell] = acc;
  }
}

// ---- GMRES building blocks on compact vectors of length L -----------------
constexpr int kRestart = 30;
constexpr int kRedBlocks = 304;  // partial sums per reduction (2 per SM)

// part[i * kRedBlocks + b] = sum over block b's slice of V_i . w, i = 0..j
__global__ void k_multidot(const double* __restrict__ V, int64_t L, int j,
                           const double* __restrict__ w, const int* __restrict__ done,
                           double* __restrict__ part) {
  if (*done) return;
  const int i = blockIdx.y;
  if (i > j) return;
  const double* vi = V + (int64_t)i * L;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
       e += (int64_t)gridDim.x * blockDim.x)
    acc = fma(vi[e], w[e], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[i * kRedBlocks + blockIdx.x] = acc;
}

// h[i] (+)= sum_b part[i][b] for i = 0..j (fixed order); into column j of H
__global__ void k_multidot_reduce(const double* __restrict__ part, int j, int accumulate,
                                  const int* __restrict__ done, double* __restrict__ Hcol,
                                  double* __restrict__ hbuf) {
  if (*done) return;
  for (int i = threadIdx.x >> 5; i <= j; i += blockDim.x >> 5) {
    double acc = 0.0;
    for (int b = threadIdx.x & 31; b < kRedBlocks; b += 32) acc += part[i * kRedBlocks + b];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) {
      hbuf[i] = acc;
      Hcol[i] = accumulate ? Hcol[i] + acc : acc;
    }
  }
}

// w -= sum_i h_i V_i, i = 0..j
__global__ void k_sub_combination(const double* __restrict__ V, int64_t L, int j,
                                  const double* __restrict__ h, const int* __restrict__ done,
                                  double* __restrict__ w) {
  if (*done) return;
  __shared__ double hs[kRestart + 1];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
       e += (int64_t)gridDim.x * blockDim.x) {
    double x = w[e];
    for (int i = 0; i <= j; ++i) x = fma(-hs[i], V[(int64_t)i * L + e], x);
    w[e] = x;
  }
}

// part[b] = partial sum of x.x (and of max |x| in part[kRedBlocks + b])
__global__ void k_norm_part(const double* __restrict__ x, int64_t L, const int* __restrict__ done,
                            double* __restrict__ part) {
  if (done && *done) return;
  double acc = 0.0, mx = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
       e += (int64_t)gridDim.x * blockDim.x) {
    acc = fma(x[e], x[e], acc);
    mx = fmax(mx, fabs(x[e]));
  }
  acc = block_sum(acc);
  mx = block_max(mx);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = acc;
    part[kRedBlocks + blockIdx.x] = mx;
  }
}

// out[0] = sqrt(sum part), out[1] = max part (fixed order)
__global__ void k_norm_reduce(const double* __restrict__ part, const int* __restrict__ done,
                              double* __restrict__ out) {
  if (done && *done) return;
  double acc = 0.0, mx = 0.0;
  for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) {
    acc += part[b];
    mx = fmax(mx, part[kRedBlocks + b]);
  }
  acc = block_sum(acc);
  mx = block_max(mx);
  if (threadIdx.x == 0) {
    out[0] = sqrt(acc);
    out[1] = mx;
  }
}

// y = s * x (s = 1 / nrm[0], or -1 / nrm[0] with neg)
__global__ void k_scale(const double* __restrict__ x, int64_t L, const double* __restrict__ nrm,
                        int neg, const int* __restrict__ done, double* __restrict__ y) {
  if (done && *done) return;
  const double nv = nrm[0];
  const double s = nv > 0.0 ? (neg ? -1.0 : 1.0) / nv : 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = s * x[e];
}

// GMRES state: H column-major (kRestart + 1) x kRestart, Givens cosines /
// sines, the rotated right-hand side g, the column count kept, the stop flag
struct GmresState {
  double H[(kRestart + 1) * kRestart];
  double cs[kRestart], sn[kRestart], g[kRestart + 1];
  double beta, eta;
  int kept;
  int done;
};

// start: g = (beta, 0, ...), beta = ||r0|| (nrm[0]); done when beta == 0
__global__ void k_gmres_start(GmresState* st, const double* __restrict__ nrm, double eta) {
  st->beta = nrm[0];
  st->eta = eta;
  for (int i = 0; i <= kRestart; ++i) st->g[i] = 0.0;
  st->g[0] = nrm[0];
  st->kept = 0;
  st->done = !(nrm[0] > 0.0);
}

// column j of H complete (h_{j+1,j} = nrm[0]): apply the previous rotations,
// form rotation j, update g; stop when |g_{j+1}| <= eta beta or the column
// count reaches kRestart (or a breakdown h_{j+1,j} = 0)
__global__ void k_gmres_givens(GmresState* st, int j, const double* __restrict__ nrm) {
  if (st->done) return;
  double* h = st->H + j * (kRestart + 1);
  h[j + 1] = nrm[0];
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = st->cs[i] * a + st->sn[i] * b;
    h[i + 1] = -st->sn[i] * a + st->cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  const double r = hypot(a, b);
  const double cj = r > 0.0 ? a / r : 1.0, sj = r > 0.0 ? b / r : 0.0;
  st->cs[j] = cj;
  st->sn[j] = sj;
  h[j] = r;
  h[j + 1] = 0.0;
  st->g[j + 1] = -sj * st->g[j];
  st->g[j] = cj * st->g[j];
  st->kept = j + 1;
  if (fabs(st->g[j + 1]) <= st->eta * st->beta || j + 1 == kRestart || !(b != 0.0)) st->done = 1;
}

// y = H^{-1} g (upper triangular, kept columns), into st->g's slots
__global__ void k_gmres_solve(GmresState* st, double* __restrict__ y) {
  const int kk = st->kept;
  for (int i = kk - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int c = i + 1; c < kk; ++c) s -= st->H[c * (kRestart + 1) + i] * y[c];
    const double d = st->H[i * (kRestart + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
  for (int i = kk; i < kRestart; ++i) y[i] = 0.0;
}

// q[cells] += sum_i y_i V_i (compact -> state)
__global__ void k_update_state(DevCfg c, const double* __restrict__ V, int64_t n,
                               const double* __restrict__ y, const GmresState* __restrict__ st,
                               const int* __restrict__ cells, double* __restrict__ q) {
  __shared__ double ys[kRestart];
  __shared__ int kk;
  if (threadIdx.x == 0) kk = st->kept;
  for (int i = threadIdx.x; i < kRestart; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  const int64_t L = 4 * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
       e += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int i = 0; i < kk; ++i) d = fma(ys[i], V[(int64_t)i * L + e], d);
    const int64_t v = e / n, idx = e % n;
    q[v * c.nc + cell_of(cells, idx)] += d;
  }
}

// dv[cells] = V_j (compact -> every cell; the other cells stay zero)
__global__ void k_scatter(DevCfg c, const double* __restrict__ x, int64_t n,
                          const int* __restrict__ cells, const int* __restrict__ done,
                          double* __restrict__ dv) {
  if (done && *done) return;
  const int64_t L = 4 * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / n, idx = e % n;
    dv[v * c.nc + cells[idx]] = x[e];
  }
}

// Shapiro filter of order 2n along x (AX = 0) or y (AX = 1), every variable:
// weights (times 4^n) (1 2 1), (-1 4 10 4 -1), (1 -6 15 44 15 -6 1) summed left
// to right, then scaled by 4^-n; zeroth-order extrapolation on non-periodic
// sides, wrap on periodic ones
template <int AX>
__global__ void k_shapiro(DevCfg c, int n, const double* __restrict__ in, double* __restrict__ out) {
  const double W1[3] = {1.0, 2.0, 1.0};
  const double W2[5] = {-1.0, 4.0, 10.0, 4.0, -1.0};
  const double W3[7] = {1.0, -6.0, 15.0, 44.0, 15.0, -6.0, 1.0};
  const double* wt = n == 1 ? W1 : (n == 2 ? W2 : W3);
  const double scale = n == 1 ? 0.25 : (n == 2 ? 0.0625 : 0.015625);
  const bool per = AX == 0 ? c.bc[0] == HYROM_BC_PERIODIC : c.bc[2] == HYROM_BC_PERIODIC;
  const int len = AX == 0 ? c.nx : c.ny;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 4 * c.nc;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / c.nc, cell = e % c.nc;
    const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
    const int a = AX == 0 ? i : j;
    double acc = 0.0;
    for (int tt = 0; tt <= 2 * n; ++tt) {
      int b = a + tt - n;
      b = per ? imod(b, len) : (b < 0 ? 0 : (b >= len ? len - 1 : b));
      const int64_t src = AX == 0 ? (int64_t)j * c.nx + b : (int64_t)b * c.nx + i;
      const double x = in[v * c.nc + src];
      const double term = wt[tt] == 1.0 ? x : (wt[tt] == -1.0 ? -x : wt[tt] * x);
      acc = tt == 0 ? term : acc + term;
    }
    out[e] = acc * scale;
  }
}

// gate: keep the filtered value where rho_new < rho_old; per-block partial
// counts, decrease and previous total of the kept cells
__global__ void k_gate(DevCfg c, const double* __restrict__ rho_old,
                       const double* __restrict__ rho_new, const double* __restrict__ g,
                       double* __restrict__ q, double* __restrict__ part) {
  double cnt = 0.0, dec = 0.0, tot = 0.0;
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < c.nc;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const double ro = rho_old[cell], rn = rho_new[cell];
    if (rn < ro) {
      cnt += 1.0;
      dec += ro - rn;
      tot += ro;
      for (int v = 0; v < 4; ++v) q[v * c.nc + cell] = g[v * c.nc + cell];
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

__global__ void k_gate_sum(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double cnt = 0.0, dec = 0.0, tot = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    cnt += part[3 * b];
    dec += part[3 * b + 1];
    tot += part[3 * b + 2];
  }
  cnt = block_sum(cnt);
  dec = block_sum(dec);
  tot = block_sum(tot);
  if (threadIdx.x == 0) {
    out[0] = cnt;
    out[1] = dec;
    out[2] = tot;
  }
}

// ---- sparse filter passes ---------------------------------------------------
// dst = src dilated by r cells along one axis (square dilation = x then y)
template <int AX>
__global__ void k_dilate_axis(DevCfg c, const uint32_t* __restrict__ src, int r,
                              uint32_t* __restrict__ dst) {
  const bool per = AX == 0 ? c.bc[0] == HYROM_BC_PERIODIC : c.bc[2] == HYROM_BC_PERIODIC;
  const int len = AX == 0 ? c.nx : c.ny;
  const int64_t nwords = (c.nc + 31) / 32;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll;
       base < nwords * 32; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = base + (threadIdx.x & 31);
    bool on = false;
    if (cell < c.nc) {
      const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
      const int a = AX == 0 ? i : j;
      for (int d = -r; d <= r && !on; ++d) {
        int b = a + d;
        if (per) b = imod(b, len);
        else if (b < 0 || b >= len) continue;
        on = bit_get(src, AX == 0 ? (int64_t)j * c.nx + b : (int64_t)b * c.nx + i);
      }
    }
    const unsigned word = __ballot_sync(0xffffffffu, on);
    if ((threadIdx.x & 31) == 0 && base < c.nc) dst[base >> 5] = word;
  }
}

// g on the listed cells: the separable filter x then y, each sum left to
// right and scaled, as the dense kernels (and the oracle) form it
__global__ void k_filter_cells(DevCfg c, int n, const double* __restrict__ q,
                               const int* __restrict__ cells, const long long* __restrict__ count,
                               double* __restrict__ g) {
  const double W1[3] = {1.0, 2.0, 1.0};
  const double W2[5] = {-1.0, 4.0, 10.0, 4.0, -1.0};
  const double W3[7] = {1.0, -6.0, 15.0, 44.0, 15.0, -6.0, 1.0};
  const double* wt = n == 1 ? W1 : (n == 2 ? W2 : W3);
  const double scale = n == 1 ? 0.25 : (n == 2 ? 0.0625 : 0.015625);
  const bool px = c.bc[0] == HYROM_BC_PERIODIC, py = c.bc[2] == HYROM_BC_PERIODIC;
  const bool two = c.ny > 1;
  const int64_t cnt = *count;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 4 * cnt;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / cnt, cell = cells[e % cnt];
    const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
    double acc_y = 0.0;
    const int ty = two ? 2 * n : 0;
    for (int tt = 0; tt <= ty; ++tt) {
      int jj = two ? j + tt - n : j;
      jj = py ? imod(jj, c.ny) : (jj < 0 ? 0 : (jj >= c.ny ? c.ny - 1 : jj));
      double acc = 0.0;
      for (int ss = 0; ss <= 2 * n; ++ss) {
        int ii = i + ss - n;
        ii = px ? imod(ii, c.nx) : (ii < 0 ? 0 : (ii >= c.nx ? c.nx - 1 : ii));
        const double x = q[v * c.nc + (int64_t)jj * c.nx + ii];
        const double term = wt[ss] == 1.0 ? x : (wt[ss] == -1.0 ? -x : wt[ss] * x);
        acc = ss == 0 ? term : acc + term;
      }
      const double fx = acc * scale;
      if (!two) {
        acc_y = fx;
        break;
      }
      const double term = wt[tt] == 1.0 ? fx : (wt[tt] == -1.0 ? -fx : wt[tt] * fx);
      acc_y = tt == 0 ? term : acc_y + term;
    }
    g[v * c.nc + cell] = two ? acc_y * scale : acc_y;
  }
}

// rho on the listed cells
__global__ void k_muscl_rho_cells(DevCfg c, const double* __restrict__ q,
                                  const double* __restrict__ qp, const double* __restrict__ qp2,
                                  double t, const int* __restrict__ cells,
                                  const long long* __restrict__ count, double* __restrict__ rho) {
  const Src<double> src{q};
  const int64_t cnt = *count;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < cnt;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = cells[idx];
    const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
    double f[4];
    muscl_rhs_cell<double>(c, src, i, j, t, f);
    double acc = 0.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double qc = q[v * c.nc + cell], p1 = qp[v * c.nc + cell];
      double R;
      if (qp2) {
        const double p2 = qp2[v * c.nc + cell];
        R = ((1.0 * qc + (-4.0 / 3.0) * p1) + (1.0 / 3.0) * p2) - (c.dt * (2.0 / 3.0)) * f[v];
      } else {
        R = (qc - p1) - c.dt * f[v];
      }
      acc = v == 0 ? fabs(R) : acc + fabs(R);
    }
    rho[cell] = acc;
  }
}

// gate on the listed cells (all cells when cells is null): keep where
// rho_new < rho_old, set the cell's bit in kbits, per-block partial sums
__global__ void k_gate_cells(DevCfg c, const int* __restrict__ cells,
                             const long long* __restrict__ count,
                             const double* __restrict__ rho_old,
                             const double* __restrict__ rho_new, const double* __restrict__ g,
                             double* __restrict__ q, uint32_t* __restrict__ kbits,
                             double* __restrict__ part) {
  double cnt = 0.0, dec = 0.0, tot = 0.0;
  const int64_t n = cells ? *count : c.nc;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = cells ? cells[idx] : idx;
    const double ro = rho_old[cell], rn = rho_new[cell];
    if (rn < ro) {
      cnt += 1.0;
      dec += ro - rn;
      tot += ro;
      for (int v = 0; v < 4; ++v) q[v * c.nc + cell] = g[v * c.nc + cell];
      atomicOr(kbits + (cell >> 5), 1u << (cell & 31));
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

int grid_for(int64_t n, int per = 256) {
  int64_t b = (n + per - 1) / per;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct MusclSolver {
  int64_t nc = 0, maxn = 0;
  double* V = nullptr;     // (kRestart + 1) compact vectors of 4 maxn
  double* w = nullptr;     // compact
  double* R = nullptr;     // compact residual
  double* dv = nullptr;    // direction on every cell (4 nc)
  double* part = nullptr;  // reduction partials
  double* hbuf = nullptr;
  double* nrm = nullptr;   // [0] 2-norm, [1] max
  double* y = nullptr;
  GmresState* st = nullptr;
  double* host = nullptr;  // pinned: [0] max |R|, [1] scale
  // sparse filter passes: kept cells, the two dilations and their lists
  uint32_t *kbits = nullptr, *bm_a = nullptr, *bm_b = nullptr, *bm_t = nullptr;
  int *list_r = nullptr, *list_g = nullptr;
  long long *cnt = nullptr, *scan = nullptr;
  size_t bytes = 0;
};

MusclSolver* muscl_create(int64_t nc, int64_t max_cells) {
  MusclSolver* m = new MusclSolver;
  m->nc = nc;
  m->maxn = max_cells;
  const int64_t L = 4 * max_cells;
  bool ok = true;
  auto al = [&](void** p, size_t b) {
    if (!ok) return;
    if (cudaMalloc(p, b) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
      return;
    }
    m->bytes += b;
  };
  al((void**)&m->V, sizeof(double) * (kRestart + 1) * L);
  al((void**)&m->w, sizeof(double) * L);
  al((void**)&m->R, sizeof(double) * L);
  al((void**)&m->dv, sizeof(double) * 4 * nc);
  al((void**)&m->part, sizeof(double) * (kRestart + 1) * kRedBlocks * 2);
  al((void**)&m->hbuf, sizeof(double) * (kRestart + 1));
  al((void**)&m->nrm, sizeof(double) * 4);
  al((void**)&m->y, sizeof(double) * kRestart);
  al((void**)&m->st, sizeof(GmresState));
  const int64_t nw = (nc + 31) / 32;
  al((void**)&m->kbits, sizeof(uint32_t) * nw);
  al((void**)&m->bm_a, sizeof(uint32_t) * nw);
  al((void**)&m->bm_b, sizeof(uint32_t) * nw);
  al((void**)&m->bm_t, sizeof(uint32_t) * nw);
  al((void**)&m->list_r, sizeof(int) * nc);
  al((void**)&m->list_g, sizeof(int) * nc);
  al((void**)&m->cnt, sizeof(long long) * 4);
  al((void**)&m->scan, sizeof(long long) * 1024);
  if (ok && cudaMallocHost((void**)&m->host, 64) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
  }
  if (!ok) {
    muscl_destroy(m);
    return nullptr;
  }
  return m;
}

void muscl_destroy(MusclSolver* m) {
  if (!m) return;
  cudaFree(m->V);
  cudaFree(m->w);
  cudaFree(m->R);
  cudaFree(m->dv);
  cudaFree(m->part);
  cudaFree(m->hbuf);
  cudaFree(m->nrm);
  cudaFree(m->y);
  cudaFree(m->st);
  cudaFree(m->kbits);
  cudaFree(m->bm_a);
  cudaFree(m->bm_b);
  cudaFree(m->bm_t);
  cudaFree(m->list_r);
  cudaFree(m->list_g);
  cudaFree(m->cnt);
  cudaFree(m->scan);
  if (m->host) cudaFreeHost(m->host);
  delete m;
}

size_t muscl_bytes(const MusclSolver* m) { return m ? m->bytes : 0; }

void launch_muscl_residual(const DevCfg& c, const double* q, const double* qp, const double* qp2,
                           double t, const int* cells, int64_t n, double* out, cudaStream_t s) {
  k_muscl_residual<<<grid_for(n, 128), 128, 0, HY_S(s)>>>(c, q, qp, qp2, t, cells, n, out);
}

void launch_muscl_jvp(const DevCfg& c, const double* q, const double* dv, double t, double a2,
                      double dtb, const int* cells, int64_t n, double* out, cudaStream_t s) {
  k_muscl_jvp<<<grid_for(n, 128), 128, 0, HY_S(s)>>>(c, q, dv, t, a2, dtb, cells, n, nullptr,
                                                      out);
}

void launch_muscl_rho(const DevCfg& c, const double* q, const double* qp, const double* qp2,
                      double t, double* rho, cudaStream_t s) {
  k_muscl_rho<<<grid_for(c.nc, 128), 128, 0, HY_S(s)>>>(c, q, qp, qp2, t, rho);
}

// Newton's method on R_k(q) = 0 over the listed cells (all when cells is
// null), the other cells frozen; each Newton step solves J d = -R by one
// GMRES cycle of at most kRestart Arnoldi steps to relative residual eta
// (classical Gram-Schmidt, applied twice), then q += d.  Stops when
// max |R| <= tol_abs (checked on the host: one read-back per Newton step).
// Returns 0 (converged), 1 (newton_max reached), -1 (CUDA error).
int muscl_newton(MusclSolver* m, const DevCfg& c, double* q, const double* qp,
                 const double* qp2, int64_t k, const int* cells, int64_t n, double tol_abs,
                 int newton_max, double eta, cudaStream_t s, int* iters_out, int* arnoldi_out) {
  const double t = (double)k * c.dt;
  const double a2 = 1.0, dtb = qp2 ? c.dt * (2.0 / 3.0) : c.dt;
  const int64_t L = 4 * n;
  const int gL = grid_for(L), gn = grid_for(n, 128);
  int* done = &m->st->done;
  int arnoldi = 0;
  if (cudaMemsetAsync(m->dv, 0, sizeof(double) * 4 * c.nc, s) != cudaSuccess) return -1;
  for (int it = 0; it <= newton_max; ++it) {
    k_muscl_residual<<<gn, 128, 0, HY_S(s)>>>(c, q, qp, qp2, t, cells, n, m->R);
    k_norm_part<<<kRedBlocks, 256, 0, HY_S(s)>>>(m->R, L, nullptr, m->part);
    k_norm_reduce<<<1, 256, 0, HY_S(s)>>>(m->part, nullptr, m->nrm);
    if (cudaMemcpyAsync(m->host, m->nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return -1;
    if (iters_out) *iters_out = it;
    if (arnoldi_out) *arnoldi_out = arnoldi;
    if (m->host[0] <= tol_abs) return 0;
    if (it == newton_max) break;
    // GMRES on J d = -R: V_0 = -R / ||R||
    k_gmres_start<<<1, 1, 0, HY_S(s)>>>(m->st, m->nrm, eta);
    k_scale<<<gL, 256, 0, HY_S(s)>>>(m->R, L, m->nrm, 1, nullptr, m->V);
    for (int j = 0; j < kRestart; ++j) {
      const double* vj = m->V + (int64_t)j * L;
      const double* dir = vj;
      if (cells) {
        k_scatter<<<gL, 256, 0, HY_S(s)>>>(c, vj, n, cells, done, m->dv);
        dir = m->dv;
      }
      k_muscl_jvp<<<gn, 128, 0, HY_S(s)>>>(c, q, dir, t, a2, dtb, cells, n, done, m->w);
      double* Hcol = m->st->H + j * (kRestart + 1);
      for (int pass = 0; pass < 2; ++pass) {
        k_multidot<<<dim3(kRedBlocks, j + 1), 256, 0, HY_S(s)>>>(m->V, L, j, m->w, done, m->part);
        k_multidot_reduce<<<1, 1024, 0, HY_S(s)>>>(m->part, j, pass, done, Hcol, m->hbuf);
        k_sub_combination<<<gL, 256, 0, HY_S(s)>>>(m->V, L, j, m->hbuf, done, m->w);
      }
      k_norm_part<<<kRedBlocks, 256, 0, HY_S(s)>>>(m->w, L, done, m->part);
      k_norm_reduce<<<1, 256, 0, HY_S(s)>>>(m->part, done, m->nrm);
      k_scale<<<gL, 256, 0, HY_S(s)>>>(m->w, L, m->nrm, 0, done, m->V + (int64_t)(j + 1) * L);
      k_gmres_givens<<<1, 1, 0, HY_S(s)>>>(m->st, j, m->nrm);
      // every fourth step: stop enqueueing once the cycle has converged
      if ((j & 3) == 3 && j + 1 < kRestart) {
        if (cudaMemcpyAsync(m->host + 2, &m->st->done, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          return -1;
        if (*reinterpret_cast<int*>(m->host + 2)) break;
      }
    }
    k_gmres_solve<<<1, 1, 0, HY_S(s)>>>(m->st, m->y);
    k_update_state<<<gL, 256, 0, HY_S(s)>>>(c, m->V, n, m->y, m->st, cells, q);
    if (cells)  // the next direction scatter must start from zero elsewhere
      if (cudaMemsetAsync(m->dv, 0, sizeof(double) * 4 * c.nc, s) != cudaSuccess) return -1;
    arnoldi += kRestart;  // upper bound; the exact count is not read back
  }
  return 1;
}

// SpatialFilter of Algorithm 1 (Sec. 2.3.4) gated on this HDM's residual
// R_k of Eq. hdm (BDF2; BDF1 when qp2 is null): for each order, the
// residual measure of q, then passes of filter / measure / gate until no
// cell is kept, the kept cells' decrease falls below eps_f times their
// previous total, or jmax_f passes ran.  The first pass of an order covers
// the grid.  A later pass can change g only within a square of n cells of
// the cells K the previous pass kept, and the residual measure only within
// two more (the MUSCL stencil): it visits the square of radius n + 2 around
// K for the measures and the gate and that of radius n + 4 for g; every
// other cell keeps its "not kept" decision, as the dense pass would give.
// The decisions are read back once per pass.  g, tmp: 4 nc doubles;
// rho_old, rho_new: nc; part: 3 * 1216 doubles; out3: 3 device doubles.
// Returns the passes run, or -1 on a CUDA error.
int muscl_filter(MusclSolver* m, const DevCfg& c, double* q, const double* qp, const double* qp2,
                 int64_t k, const int* orders, int n_filt, int jmax_f, double eps_f, double* g,
                 double* tmp, double* rho_old, double* rho_new, double* part, double* out3,
                 double* host3, cudaStream_t s) {
  const double t = (double)k * c.dt;
  const int gq = grid_for(4 * c.nc), gc = grid_for(c.nc);
  const int64_t nw = (c.nc + 31) / 32;
  const int gw = grid_for(nw * 32);
  int passes = 0;
  auto dilate = [&](int r, uint32_t* out) {
    k_dilate_axis<0><<<gw, 256, 0, HY_S(s)>>>(c, m->kbits, r, c.ny > 1 ? m->bm_t : out);
    if (c.ny > 1) k_dilate_axis<1><<<gw, 256, 0, HY_S(s)>>>(c, m->bm_t, r, out);
  };
  auto listify = [&](const uint32_t* bm, int* list, long long* cnt) {
    launch_popcount(bm, nw, cnt, s);
    launch_bits_to_list(bm, c.nc, m->scan, list, c.nc, s);
  };
  for (int o = 0; o < n_filt; ++o) {
    const int n = orders[o];
    for (int p = 0; p < jmax_f; ++p) {
      if (cudaMemsetAsync(m->kbits, 0, sizeof(uint32_t) * nw, s) != cudaSuccess) return -1;
      if (p == 0) {
        k_muscl_rho<<<grid_for(c.nc, 128), 128, 0, HY_S(s)>>>(c, q, qp, qp2, t, rho_old);
        if (c.ny > 1) {
          k_shapiro<0><<<gq, 256, 0, HY_S(s)>>>(c, n, q, tmp);
          k_shapiro<1><<<gq, 256, 0, HY_S(s)>>>(c, n, tmp, g);
        } else {
          k_shapiro<0><<<gq, 256, 0, HY_S(s)>>>(c, n, q, g);
        }
        k_muscl_rho<<<grid_for(c.nc, 128), 128, 0, HY_S(s)>>>(c, g, qp, qp2, t, rho_new);
        k_gate_cells<<<gc, 256, 0, HY_S(s)>>>(c, nullptr, nullptr, rho_old, rho_new, g, q,
                                              m->kbits, part);
      } else {
        // the cells kept by the previous pass are in bm_a (saved below)
        const int gr = grid_for(c.nc, 128);
        k_muscl_rho_cells<<<gr, 128, 0, HY_S(s)>>>(c, q, qp, qp2, t, m->list_r, m->cnt,
                                                    rho_old);
        k_filter_cells<<<gq, 256, 0, HY_S(s)>>>(c, n, q, m->list_g, m->cnt + 1, g);
        k_muscl_rho_cells<<<gr, 128, 0, HY_S(s)>>>(c, g, qp, qp2, t, m->list_r, m->cnt,
                                                    rho_new);
        k_gate_cells<<<gc, 256, 0, HY_S(s)>>>(c, m->list_r, m->cnt, rho_old, rho_new, g, q,
                                              m->kbits, part);
      }
      k_gate_sum<<<1, 256, 0, HY_S(s)>>>(part, gc, out3);
      if (cudaMemcpyAsync(host3, out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
      ++passes;
      if (host3[0] == 0.0) break;
      if (host3[1] < eps_f * host3[2]) break;
      if (p + 1 < jmax_f) {  // the next pass's cells, from the cells just kept
        dilate(n + 2, m->bm_a);
        listify(m->bm_a, m->list_r, m->cnt);
        dilate(n + 4, m->bm_b);
        listify(m->bm_b, m->list_g, m->cnt + 1);
      }
    }
  }
  return passes;
}

}  // namespace hy
