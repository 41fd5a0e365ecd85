// Adjoint (vector-Jacobian product) of the SSP-RK2 Euler HDM step, full or
// restricted to the sampled cells: the first piece of the differentiation
// form.  For the step
//   q1 = q + dt L(q, t_{k-1}),   q_k = q/2 + (q1 + dt L(q1, t_k))/2
// (Sec. 2.2, the explicit scheme of the run configurations), a cotangent
// lambda of q_k pulls back to
//   lambda_1 = lambda/2 + (dt/2) L'(q1)^T lambda,
//   lambda_q = lambda/2 + lambda_1 + dt L'(q)^T lambda_1.
// The partial step of Algorithm 1 replaces only the cells of S-hat, so
// there lambda is first restricted to S-hat and the other cells pass their
// lambda through unchanged.
//
// L'(q)^T mu is a gather per cell over its faces.  L_i = -(F_{i+1/2} -
// F_{i-1/2})/dx - (G_{j+1/2} - G_{j-1/2})/dy, so a face carries the
// cotangent Fbar_{i+1/2} = (mu_{i+1} - mu_i)/dx (mu = 0 at a ghost cell) and
// passes dF/dq_side^T Fbar to each side's cell; an outflow ghost is a copy
// of its boundary cell and passes its share to that cell too; a shock
// ghost is a fixed state and passes nothing; periodic sides wrap.  The face
// Jacobians come from the Rusanov flux's tangent (primitives, flux, wave
// speed; at a tie of the two wave speeds the left one is differentiated)
// applied to the unit vectors.  FP64 throughout.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"
#include "phys.cuh"

namespace hy {

namespace {

// tangent of the primitives (u, v, p, c) along dq
HY_DEV void prims_tan(const double* q, const double* dq, double g, double* w, double* dw) {
  const double u = q[1] / q[0], v = q[2] / q[0];
  const double du = (dq[1] - u * dq[0]) / q[0];
  const double dv = (dq[2] - v * dq[0]) / q[0];
  const double k2 = u * u + v * v;
  const double p = (g - 1.0) * (q[3] - 0.5 * q[0] * k2);
  const double dp = (g - 1.0) * (dq[3] - 0.5 * dq[0] * k2 - q[0] * (u * du + v * dv));
  const double a2 = g * p / q[0];
  const double da2 = g * (dp - p * dq[0] / q[0]) / q[0];
  const double c = sqrt(a2 > 0.0 ? a2 : 0.0);
  w[0] = u;
  w[1] = v;
  w[2] = p;
  w[3] = c;
  dw[0] = du;
  dw[1] = dv;
  dw[2] = dp;
  dw[3] = (a2 > 0.0 && c > 0.0) ? 0.5 * da2 / c : 0.0;
}

HY_DEV double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// tangent of the Rusanov flux across an AX face along (dqL, dqR)
template <int AX>
HY_DEV void rusanov_tan(const double* qL, const double* dqL, const double* qR, const double* dqR,
                        double g, double* dF) {
  double wL[4], dwL[4], wR[4], dwR[4];
  prims_tan(qL, dqL, g, wL, dwL);
  prims_tan(qR, dqR, g, wR, dwR);
  double dfL[4], dfR[4];
  const double* W[2] = {wL, wR};
  const double* DW[2] = {dwL, dwR};
  const double* Q[2] = {qL, qR};
  const double* DQ[2] = {dqL, dqR};
  double* DF[2] = {dfL, dfR};
  for (int s = 0; s < 2; ++s) {
    const double *q = Q[s], *dq = DQ[s], *w = W[s], *dw = DW[s];
    double* df = DF[s];
    if (AX == 0) {
      df[0] = dq[1];
      df[1] = dq[1] * w[0] + q[1] * dw[0] + dw[2];
      df[2] = dq[2] * w[0] + q[2] * dw[0];
      df[3] = (dq[3] + dw[2]) * w[0] + (q[3] + w[2]) * dw[0];
    } else {
      df[0] = dq[2];
      df[1] = dq[1] * w[1] + q[1] * dw[1];
      df[2] = dq[2] * w[1] + q[2] * dw[1] + dw[2];
      df[3] = (dq[3] + dw[2]) * w[1] + (q[3] + w[2]) * dw[1];
    }
  }
  const double nL = AX == 0 ? wL[0] : wL[1], nR = AX == 0 ? wR[0] : wR[1];
  const double dnL = AX == 0 ? dwL[0] : dwL[1], dnR = AX == 0 ? dwR[0] : dwR[1];
  const double sL = fabs(nL) + wL[3], sR = fabs(nR) + wR[3];
  const double a = sL > sR ? sL : sR;
  const double da = sL >= sR ? sgn(nL) * dnL + dwL[3] : sgn(nR) * dnR + dwR[3];
  for (int r = 0; r < 4; ++r)
    dF[r] = 0.5 * (dfL[r] + dfR[r]) - 0.5 * (da * (qR[r] - qL[r]) + a * (dqR[r] - dqL[r]));
}

// acc += (dF/dq_side)^T fbar for the face (qL, qR); side 0 = left, 1 = right
template <int AX>
HY_DEV void face_pullback(const double* qL, const double* qR, double g, int side,
                          const double* fbar, double* acc) {
  const double zero[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = 0; c < 4; ++c) {
    double e[4] = {0.0, 0.0, 0.0, 0.0};
    e[c] = 1.0;
    double dF[4];
    if (side == 0)
      rusanov_tan<AX>(qL, e, qR, zero, g, dF);
    else
      rusanov_tan<AX>(qL, zero, qR, e, g, dF);
    acc[c] += dF[0] * fbar[0] + dF[1] * fbar[1] + dF[2] * fbar[2] + dF[3] * fbar[3];
  }
}

// mu at grid position (gi, gj): a domain cell (wrapped on periodic sides) or
// 0 at a ghost
HY_DEV void mu_at(const DevCfg& c, const double* mu, int gi, int gj, double* out) {
  bool ghost = false;
  if (gi < 0 || gi >= c.nx) {
    if (c.bc[0] == HYROM_BC_PERIODIC)
      gi = imod(gi, c.nx);
    else
      ghost = true;
  }
  if (c.ny > 1 && (gj < 0 || gj >= c.ny)) {
    if (c.bc[2] == HYROM_BC_PERIODIC)
      gj = imod(gj, c.ny);
    else
      ghost = true;
  }
  for (int v = 0; v < 4; ++v) out[v] = ghost ? 0.0 : mu[v * c.nc + (int64_t)gj * c.nx + gi];
}

// out = c1 b1 + c2 b2 + c3 b3 + coef L'(q, t)^T mu   (b2, b3 may be null)
__global__ void k_rhs_vjp(DevCfg c, const double* __restrict__ q, const double* __restrict__ mu,
                          double t, double coef, const double* __restrict__ b1, double c1,
                          const double* __restrict__ b2, double c2,
                          const double* __restrict__ b3, double c3, double* __restrict__ out) {
  const bool twoD = c.ny > 1;
  const double g = c.gamma;
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < c.nc;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const int gi = (int)(cell % c.nx), gj = (int)(cell / c.nx);
    double qC[4], m0[4], acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int v = 0; v < 4; ++v) {
      qC[v] = q[v * c.nc + cell];
      m0[v] = mu[v * c.nc + cell];
    }
    for (int ax = 0; ax < (twoD ? 2 : 1); ++ax) {
      const double inv = ax == 0 ? 1.0 / c.dx : 1.0 / c.dy;
      for (int s = 0; s < 2; ++s) {  // s = 0: the face below (left), 1: above (right)
        const int ni = ax == 0 ? gi + (s ? 1 : -1) : gi;
        const int nj = ax == 1 ? gj + (s ? 1 : -1) : gj;
        double qN[4], mN[4], fbar[4];
        fetch<double, 4>(c, q, ni, nj, t, qN);
        mu_at(c, mu, ni, nj, mN);
        // Fbar of the face: (mu_right - mu_left) / h
        for (int v = 0; v < 4; ++v) fbar[v] = s ? (mN[v] - m0[v]) * inv : (m0[v] - mN[v]) * inv;
        const double* qL = s ? qC : qN;
        const double* qR = s ? qN : qC;
        // this cell is the right state of the face below, the left of the one above
        if (ax == 0)
          face_pullback<0>(qL, qR, g, s ? 0 : 1, fbar, acc);
        else
          face_pullback<1>(qL, qR, g, s ? 0 : 1, fbar, acc);
        // an outflow ghost is a copy of this cell: its side of the face too
        const bool outside = ax == 0 ? (ni < 0 || ni >= c.nx) : (nj < 0 || nj >= c.ny);
        const int side = ax == 0 ? (ni < 0 ? 0 : 1) : (nj < 0 ? 2 : 3);
        if (outside && c.bc[side] == HYROM_BC_OUTFLOW) {
          if (ax == 0)
            face_pullback<0>(qL, qR, g, s ? 1 : 0, fbar, acc);
          else
            face_pullback<1>(qL, qR, g, s ? 1 : 0, fbar, acc);
        }
      }
    }
    for (int v = 0; v < 4; ++v) {
      const int64_t i = v * c.nc + cell;
      double o = c1 * b1[i];
      if (b2) o += c2 * b2[i];
      if (b3) o += c3 * b3[i];
      out[i] = o + coef * acc[v];
    }
  }
}

// q1 = q + dt L(q, t) (stage 1 of the step, the expressions of rhs_cell)
__global__ void k_stage1(DevCfg c, const double* __restrict__ q, double t,
                         double* __restrict__ q1) {
  const bool twoD = c.ny > 1;
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < c.nc;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const int gi = (int)(cell % c.nx), gj = (int)(cell / c.nx);
    double qC[4], qW[4], qE[4], qS[4], qN[4], r[4];
    for (int v = 0; v < 4; ++v) qC[v] = q[v * c.nc + cell];
    fetch<double, 4>(c, q, gi - 1, gj, t, qW);
    fetch<double, 4>(c, q, gi + 1, gj, t, qE);
    if (twoD) {
      fetch<double, 4>(c, q, gi, gj - 1, t, qS);
      fetch<double, 4>(c, q, gi, gj + 1, t, qN);
    } else {
      for (int v = 0; v < 4; ++v) qS[v] = qN[v] = qC[v];
    }
    rhs_cell<double, 4>(c, qC, qW, qE, qS, qN, r);
    for (int v = 0; v < 4; ++v) q1[v * c.nc + cell] = qC[v] + c.dt * r[v];
  }
}

// lam_m = lambda on the cells of the mask (all cells without one), else 0
__global__ void k_restrict(DevCfg c, const double* __restrict__ lam, const uint32_t* mask,
                           double* __restrict__ lam_m) {
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < c.nc;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const bool in = !mask || bit_get(mask, cell);
    for (int v = 0; v < 4; ++v) lam_m[v * c.nc + cell] = in ? lam[v * c.nc + cell] : 0.0;
  }
}

// ---------------------------------------------------------------------------
// adjoint of the reduced step: v_final = v on the dofs of S-hat and
// psi + Phi y on the others, y = argmin |Phi[rows] y - (v - psi)[rows]|
// (Eq. red_coord).  Phi column-major N x m.
// ---------------------------------------------------------------------------

constexpr int kRedBlocks = 152 * 8;

// split lam into the S-hat part (lam_v) and the reconstructed part lam_rec:
// lam_psi = lam_rec, lam_phi = lam_rec y^T, and per-block partial sums of
// Phi^T lam_rec (part[block * m + j])
__global__ void __launch_bounds__(256) k_red_split(int64_t N, int64_t nc, int m,
                                                   const double* __restrict__ lam,
                                                   const uint32_t* __restrict__ s_hat,
                                                   const double* __restrict__ phi,
                                                   const double* __restrict__ y,
                                                   double* __restrict__ lam_v,
                                                   double* __restrict__ lam_psi,
                                                   double* __restrict__ lam_phi,
                                                   double* __restrict__ part) {
  __shared__ double red[8][64];
  double acc[64];
  for (int j = 0; j < 64; ++j) acc[j] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool in = bit_get(s_hat, i % nc);
    const double l = lam[i];
    const double lr = in ? 0.0 : l;
    lam_v[i] = in ? l : 0.0;
    lam_psi[i] = lr;
    for (int j = 0; j < m; ++j) {
      lam_phi[(int64_t)j * N + i] = lr * y[j];
      acc[j] = fma(phi[(int64_t)j * N + i], lr, acc[j]);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < m; ++j) {
    double v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][j] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][j];
    part[(int64_t)blockIdx.x * m + j] = s;
  }
}

// one CTA: lam_y = sum of the partials, A = Phi[rows], r = b - A y,
// z = (A^T A)^{-1} lam_y by Cholesky; writes z (m), Az and r (n_r)
__global__ void __launch_bounds__(256) k_red_small(int64_t N, int m, const int* __restrict__ rows,
                                                   int nr, const double* __restrict__ phi,
                                                   const double* __restrict__ v,
                                                   const double* __restrict__ psi,
                                                   const double* __restrict__ y,
                                                   const double* __restrict__ part, int nblk,
                                                   double* __restrict__ z,
                                                   double* __restrict__ Az,
                                                   double* __restrict__ rvec) {
  __shared__ double M[64][65];
  __shared__ double ly[64];
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * m + j];
    ly[j] = s;
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    double s = 0.0;
    for (int r = 0; r < nr; ++r)
      s = fma(phi[(int64_t)i * N + rows[r]], phi[(int64_t)j * N + rows[r]], s);
    M[i][j] = s;
  }
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    double s = v[rows[r]] - psi[rows[r]];
    for (int j = 0; j < m; ++j) s -= phi[(int64_t)j * N + rows[r]] * y[j];
    rvec[r] = s;
  }
  __syncthreads();
  // Cholesky M = L L^T in the lower triangle
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) M[k][k] = sqrt(M[k][k]);
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) M[i][k] /= M[k][k];
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e % m;
      if (j > k && i >= j) M[i][j] -= M[i][k] * M[j][k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // L w = lam_y, L^T z = w
    for (int i = 0; i < m; ++i) {
      double s = ly[i];
      for (int j = 0; j < i; ++j) s -= M[i][j] * ly[j];
      ly[i] = s / M[i][i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double s = ly[i];
      for (int j = i + 1; j < m; ++j) s -= M[j][i] * ly[j];
      ly[i] = s / M[i][i];
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) z[j] = ly[j];
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s = fma(phi[(int64_t)j * N + rows[r]], ly[j], s);
    Az[r] = s;
  }
}

// the regression rows: lam_phi[rows] += r z^T - (A z) y^T, lam_v[rows] += A z,
// lam_psi[rows] -= A z (rows distinct)
__global__ void k_red_rows(int64_t N, int m, const int* __restrict__ rows, int nr,
                           const double* __restrict__ y, const double* __restrict__ z,
                           const double* __restrict__ Az, const double* __restrict__ rvec,
                           double* __restrict__ lam_v, double* __restrict__ lam_psi,
                           double* __restrict__ lam_phi) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nr * m; e += gridDim.x * blockDim.x) {
    const int r = e / m, j = e % m;
    const int64_t row = rows[r];
    lam_phi[(int64_t)j * N + row] += rvec[r] * z[j] - Az[r] * y[j];
    if (j == 0) {
      lam_v[row] += Az[r];
      lam_psi[row] -= Az[r];
    }
  }
}

}  // namespace

void launch_reduced_vjp(int64_t N, int64_t nc, int m, const double* phi, const int* rows, int nr,
                        const double* v, const double* psi, const double* y,
                        const uint32_t* s_hat, const double* lam, double* lam_v, double* lam_psi,
                        double* lam_phi, double* work, cudaStream_t s) {
  double* part = work;
  double* z = part + (size_t)kRedBlocks * m;
  double* Az = z + 64;
  double* rvec = Az + nr;
  k_red_split<<<kRedBlocks, 256, 0, HY_S(s)>>>(N, nc, m, lam, s_hat, phi, y, lam_v, lam_psi,
                                               lam_phi, part);
  k_red_small<<<1, 256, 0, HY_S(s)>>>(N, m, rows, nr, phi, v, psi, y, part, kRedBlocks, z, Az,
                                      rvec);
  const int blocks = (nr * m + 255) / 256;
  k_red_rows<<<blocks < 1 ? 1 : blocks, 256, 0, HY_S(s)>>>(N, m, rows, nr, y, z, Az, rvec, lam_v,
                                                           lam_psi, lam_phi);
}

size_t reduced_vjp_work_doubles(int m, int nr) { return (size_t)kRedBlocks * m + 64 + 2 * nr; }

void launch_rk2_vjp(const DevCfg& c, const double* q, const double* lam_out, double* lam_in,
                    const uint32_t* mask, int64_t k, double* work, cudaStream_t s) {
  const int64_t N = c.ndof;
  double* q1 = work;
  double* lam_m = work + N;
  double* lam1 = work + 2 * N;
  int64_t blocks = (c.nc + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const double t0 = (double)(k - 1) * c.dt, t1 = (double)k * c.dt;
  k_stage1<<<(int)blocks, 256, 0, HY_S(s)>>>(c, q, t0, q1);
  k_restrict<<<(int)blocks, 256, 0, HY_S(s)>>>(c, lam_out, mask, lam_m);
  // lambda_1 = lam_m/2 + (dt/2) L'(q1)^T lam_m
  k_rhs_vjp<<<(int)blocks, 256, 0, HY_S(s)>>>(c, q1, lam_m, t1, 0.5 * c.dt, lam_m, 0.5, nullptr,
                                              0.0, nullptr, 0.0, lam1);
  // lambda_q = lam_m/2 + lambda_1 + dt L'(q)^T lambda_1 + (lambda - lam_m)
  k_rhs_vjp<<<(int)blocks, 256, 0, HY_S(s)>>>(c, q, lam1, t0, c.dt, lam_m, -0.5, lam1, 1.0,
                                              lam_out, 1.0, lam_in);
}

// ---------------------------------------------------------------------------
// reverse sweep pieces (hyrom_adjoint)
// ---------------------------------------------------------------------------

// lam += w (dp/dq)^T on the cells of the box [i0, i1) x [j0, j1), p the ideal
// gas pressure (gamma - 1)(E - |m|^2 / (2 rho)): the output term of a step
__global__ void k_pressure_vjp(DevCfg c, const double* __restrict__ q, int i0, int i1, int j0,
                               int j1, double w, double* __restrict__ lam) {
  const int bw = i1 - i0;
  const int64_t nb = (int64_t)bw * (j1 - j0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nb;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = (int64_t)(j0 + e / bw) * c.nx + (i0 + e % bw);
    const double rho = q[cell], mx = q[c.nc + cell], my = q[2 * c.nc + cell];
    const double kin = (mx * mx + my * my) / rho;
    const double g1 = (c.gamma - 1.0) * w;
    lam[cell] += g1 * (0.5 * kin / rho);
    lam[c.nc + cell] += g1 * (-mx / rho);
    lam[2 * c.nc + cell] += g1 * (-my / rho);
    lam[3 * c.nc + cell] += g1;
  }
}

// sum over the box of w p(q), one partial per block, added into *acc by the
// last step of the reduction
__global__ void k_box_pressure(DevCfg c, const double* __restrict__ q, int i0, int i1, int j0,
                               int j1, double w, double* __restrict__ acc) {
  const int bw = i1 - i0;
  const int64_t nb = (int64_t)bw * (j1 - j0);
  double sum = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nb;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = (int64_t)(j0 + e / bw) * c.nx + (i0 + e % bw);
    const double rho = q[cell], mx = q[c.nc + cell], my = q[2 * c.nc + cell],
                 en = q[3 * c.nc + cell];
    sum += (c.gamma - 1.0) * (en - 0.5 * (mx * mx + my * my) / rho);
  }
  sum = block_sum(sum);
  if (threadIdx.x == 0) acc[blockIdx.x] = w * sum;
}

__global__ void k_sum_into(const double* __restrict__ part, int n, double* __restrict__ total) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *total += s;
}

// kept = lam on the cells of `keep` (zero elsewhere); lam zeroed there
__global__ void k_keep_split(DevCfg c, const uint32_t* __restrict__ keep, double* __restrict__ lam,
                             double* __restrict__ kept) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < c.ndof;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = e % c.nc;
    const bool k = bit_get(keep, cell);
    kept[e] = k ? lam[e] : 0.0;
    if (k) lam[e] = 0.0;
  }
}

// Transpose of the order-2n Shapiro filter along x (AX = 0) or y (AX = 1):
// out_a = 4^-n sum over the (b, t) whose tap b + t - n lands on a (after the
// wrap of a periodic side or the clamp of another) of w_t in_b
template <int AX>
__global__ void k_shapiro_T(DevCfg c, int n, const double* __restrict__ in,
                            double* __restrict__ out, int accumulate) {
  const double W1[3] = {1.0, 2.0, 1.0};
  const double W2[5] = {-1.0, 4.0, 10.0, 4.0, -1.0};
  const double W3[7] = {1.0, -6.0, 15.0, 44.0, 15.0, -6.0, 1.0};
  const double* wt = n == 1 ? W1 : (n == 2 ? W2 : W3);
  const double scale = n == 1 ? 0.25 : (n == 2 ? 0.0625 : 0.015625);
  const bool per = AX == 0 ? c.bc[0] == HYROM_BC_PERIODIC : c.bc[2] == HYROM_BC_PERIODIC;
  const int len = AX == 0 ? c.nx : c.ny;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < c.ndof;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / c.nc, cell = e % c.nc;
    const int i = (int)(cell % c.nx), j = (int)(cell / c.nx);
    const int a = AX == 0 ? i : j;
    double acc = 0.0;
    if (per) {
      // tap t of source b lands on a exactly when b = a - t + n (mod len)
      for (int t = 0; t <= 2 * n; ++t) {
        const int bb = imod(a - t + n, len);
        const int64_t src = AX == 0 ? (int64_t)j * c.nx + bb : (int64_t)bb * c.nx + i;
        acc += wt[t] * in[v * c.nc + src];
      }
    } else {
      // sources b within n of a, and on an end cell also the sources whose
      // taps run past it and are clamped onto it
      const int lo = a - n - (a == 0 ? n : 0), hi = a + n + (a == len - 1 ? n : 0);
      for (int b = lo < 0 ? 0 : lo; b <= hi && b < len; ++b) {
        for (int t = 0; t <= 2 * n; ++t) {
          int tap = b + t - n;
          tap = tap < 0 ? 0 : (tap >= len ? len - 1 : tap);
          if (tap != a) continue;
          const int64_t src = AX == 0 ? (int64_t)j * c.nx + b : (int64_t)b * c.nx + i;
          acc += wt[t] * in[v * c.nc + src];
        }
      }
    }
    const double r = acc * scale;
    out[e] = accumulate ? out[e] + r : r;
  }
}

// X[:, c] = state_{win_c} - psi (column-major N x wp; columns w..wp-1 zero)
__global__ void k_center_states(const double* __restrict__ states, int64_t N,
                                const int* __restrict__ win, int w, int wp,
                                const double* __restrict__ psi, double* __restrict__ X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * wp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(e / N);
    const int64_t r = e % N;
    X[e] = col < w ? states[(int64_t)win[col] * N + r] - psi[r] : 0.0;
  }
}

// part[(a * nb + b)] = partial sums of A[:, a] . B[:, b] over row slices
// (grid.x slices, grid.y = na * nb pairs)
__global__ void k_tsdots(const double* __restrict__ A, int na, const double* __restrict__ B,
                         int nb, int64_t N, double* __restrict__ part) {
  const int pair = blockIdx.y, a = pair / nb, b = pair % nb;
  double acc = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x)
    acc = fma(A[(int64_t)a * N + r], B[(int64_t)b * N + r], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[(int64_t)pair * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_tsdots_reduce(const double* __restrict__ part, int npairs, int nslice,
                                double* __restrict__ out) {
  for (int p = threadIdx.x >> 5; p < npairs; p += blockDim.x >> 5) {
    double acc = 0.0;
    for (int k = threadIdx.x & 31; k < nslice; k += 32) acc += part[(int64_t)p * nslice + k];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) out[p] = acc;
  }
}

// The thin-SVD adjoint applied to the window: for each window column c,
//   lx = sum_j L[:, j] B1[j, c] + sum_i X[:, i] B2[i, c],
// lam_{win_c} += lx + lpsi_new / w, and lpsi_cur -= sum_c lx.
// L: N x m, X: N x wp, B1: m x w, B2: wp x w (row-major small matrices).
__global__ void k_pod_vjp_apply(int64_t N, int m, int wp, int w, const double* __restrict__ L,
                                const double* __restrict__ X, const double* __restrict__ B1,
                                const double* __restrict__ B2, const int* __restrict__ win,
                                const double* __restrict__ lpsi_new, double* __restrict__ lam,
                                double* __restrict__ lpsi_cur) {
  extern __shared__ double sb[];
  double* b1 = sb;
  double* b2 = sb + m * w;
  for (int i = threadIdx.x; i < m * w; i += blockDim.x) b1[i] = B1[i];
  for (int i = threadIdx.x; i < wp * w; i += blockDim.x) b2[i] = B2[i];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double pn = lpsi_new ? lpsi_new[r] / (double)w : 0.0;
    double tot = 0.0;
    for (int col = 0; col < w; ++col) {
      double lx = 0.0;
      for (int j = 0; j < m; ++j) lx = fma(L[(int64_t)j * N + r], b1[j * w + col], lx);
      for (int i = 0; i < wp; ++i) lx = fma(X[(int64_t)i * N + r], b2[i * w + col], lx);
      lam[(int64_t)win[col] * N + r] += lx + pn;
      tot += lx;
    }
    lpsi_cur[r] -= tot;
  }
}

// lam_{j} += lpsi / w for the w window snapshots j = win[c]
__global__ void k_mean_vjp(int64_t N, const int* __restrict__ win, int w,
                           const double* __restrict__ lpsi, double* __restrict__ lam) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double v = lpsi[r] / (double)w;
    for (int c = 0; c < w; ++c) lam[(int64_t)win[c] * N + r] += v;
  }
}

namespace {
int agrid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}
}  // namespace

void launch_pressure_vjp(const DevCfg& c, const double* q, const int* box, double w, double* lam,
                         cudaStream_t s) {
  const int64_t nb = (int64_t)(box[1] - box[0]) * (box[3] - box[2]);
  k_pressure_vjp<<<agrid(nb), 256, 0, HY_S(s)>>>(c, q, box[0], box[1], box[2], box[3], w, lam);
}

void launch_box_pressure(const DevCfg& c, const double* q, const int* box, double w,
                         double* part, double* total, cudaStream_t s) {
  const int64_t nb = (int64_t)(box[1] - box[0]) * (box[3] - box[2]);
  const int g = agrid(nb);
  k_box_pressure<<<g, 256, 0, HY_S(s)>>>(c, q, box[0], box[1], box[2], box[3], w, part);
  k_sum_into<<<1, 256, 0, HY_S(s)>>>(part, g, total);
}

// lam <- lam off the kept cells + F^T (lam on them), the passes in reverse
void launch_filter_vjp(const DevCfg& c, const uint32_t* keeps, const int* orders, int npass,
                       double* lam, double* tmp1, double* tmp2, cudaStream_t s) {
  const int64_t nw = (c.nc + 31) / 32;
  const int g = agrid(c.ndof);
  for (int p = npass - 1; p >= 0; --p) {
    const int n = orders[p];
    k_keep_split<<<g, 256, 0, HY_S(s)>>>(c, keeps + (int64_t)p * nw, lam, tmp1);
    if (c.ny > 1) {
      k_shapiro_T<1><<<g, 256, 0, HY_S(s)>>>(c, n, tmp1, tmp2, 0);
      k_shapiro_T<0><<<g, 256, 0, HY_S(s)>>>(c, n, tmp2, lam, 1);
    } else {
      k_shapiro_T<0><<<g, 256, 0, HY_S(s)>>>(c, n, tmp1, lam, 1);
    }
  }
}

void launch_center_states(const double* states, int64_t N, const int* win, int w, int wp,
                          const double* psi, double* X, cudaStream_t s) {
  k_center_states<<<agrid(N * wp), 256, 0, HY_S(s)>>>(states, N, win, w, wp, psi, X);
}

// out (na x nb, row-major a, b) = A^T B for column-major N x na and N x nb
void launch_tsdots(const double* A, int na, const double* B, int nb, int64_t N, double* part,
                   double* out, cudaStream_t s) {
  const int ns = 64;
  k_tsdots<<<dim3(ns, na * nb), 256, 0, HY_S(s)>>>(A, na, B, nb, N, part);
  k_tsdots_reduce<<<1, 1024, 0, HY_S(s)>>>(part, na * nb, ns, out);
}

size_t tsdots_part_doubles(int na, int nb) { return (size_t)64 * na * nb; }

void launch_pod_vjp_apply(int64_t N, int m, int wp, int w, const double* L, const double* X,
                          const double* B1, const double* B2, const int* win,
                          const double* lpsi_new, double* lam, double* lpsi_cur,
                          cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)m * w + (size_t)wp * w);
  smem_at_least((const void*)k_pod_vjp_apply, smem);
  k_pod_vjp_apply<<<agrid(N), 256, smem, HY_S(s)>>>(N, m, wp, w, L, X, B1, B2, win, lpsi_new, lam,
                                                    lpsi_cur);
}

void launch_mean_vjp(int64_t N, const int* win, int w, const double* lpsi, double* lam,
                     cudaStream_t s) {
  k_mean_vjp<<<agrid(N), 256, 0, HY_S(s)>>>(N, win, w, lpsi, lam);
}

}  // namespace hy
