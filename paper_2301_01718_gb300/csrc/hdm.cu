// High-dimensional model on the GPU: Sec. 2.1-2.2 of the paper (conservation
// law, semi-discrete FV operator f*, BDF residual R_k = q - F_k(q)),
// Sec. 2.3 (the partial residual restricted to the sampled cells, Eq.
// partial_hdm2) and Sec. 3.1 (Euler equations, ideal gas).
//
// Fluxes: Burgers f(u) = u^2/2 with the Godunov flux; Euler with the
// Rusanov flux.  Time stepping: SSP-RK2 (explicit; the partial step on
// S-hat needs gamma_{k-1} two cells away) and BDF1 solved by Newton with the
// exact tridiagonal Jacobian (Burgers; per contiguous segment of S-hat, or
// one cyclic system for the full periodic step).
//
// Memory layout: SoA q[v*Nc + j*nx + i].  The RK2 kernel stages a tile of
// 32 x 8 cells (256 x 1 in 1D) plus a two-cell halo in shared memory, runs
// stage 1 on the tile plus a one-cell ring in shared memory and stage 2 on
// the tile, so each launch reads gamma_{k-1} once and writes gamma_k once.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "phys.cuh"

namespace hy {

// ---------------------------------------------------------------------------
// fused SSP-RK2 step over tiles (full grid, or the active tiles of S-hat)
// ---------------------------------------------------------------------------

template <typename T, int NV, int TX, int TY>
__global__ void __launch_bounds__(256) k_rk2_tile(DevCfg c, const T* __restrict__ q,
                                                  T* __restrict__ out, int64_t k,
                                                  const uint32_t* __restrict__ mask,
                                                  const int* __restrict__ tiles,
                                                  const int* __restrict__ ntiles_dev, int ntiles_all) {
  constexpr int HX = TX + 4, HY = TY + 4, H1X = TX + 2, H1Y = TY + 2;
  __shared__ T qs[NV][HY][HX];
  __shared__ T q1s[NV][H1Y][H1X];
  const bool twoD = c.ny > 1;
  const int tiles_x = (c.nx + TX - 1) / TX;
  const int ntiles = tiles ? *ntiles_dev : ntiles_all;
  const double t0 = (double)(k - 1) * c.dt, t1 = (double)k * c.dt;
  const T dt = (T)c.dt;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int tile = tiles ? tiles[it] : it;
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    __syncthreads();
    for (int idx = threadIdx.x; idx < HY * HX; idx += blockDim.x) {
      const int ly = idx / HX, lx = idx % HX;
      if (!twoD && ly != 2) continue;
      T v[NV];
      fetch<T, NV>(c, q, x0 + lx - 2, y0 + ly - 2, t0, v);
      for (int a = 0; a < NV; ++a) qs[a][ly][lx] = v[a];
    }
    __syncthreads();
    // stage 1 on the tile and its one-cell ring (positions inside the
    // domain after periodic wrap)
    for (int idx = threadIdx.x; idx < H1Y * H1X; idx += blockDim.x) {
      const int ly = idx / H1X, lx = idx % H1X;
      if (!twoD && ly != 1) continue;
      const int gi = x0 + lx - 1, gj = twoD ? y0 + ly - 1 : 0;
      const bool inx = (gi >= 0 && gi < c.nx) || c.bc[0] == HYROM_BC_PERIODIC;
      const bool iny = !twoD || (gj >= 0 && gj < c.ny) || c.bc[2] == HYROM_BC_PERIODIC;
      if (!(inx && iny)) continue;
      T qC[NV], qW[NV], qE[NV], qS[NV], qN[NV], r[NV];
      const int sy = ly + 1, sx = lx + 1;
      for (int a = 0; a < NV; ++a) {
        qC[a] = qs[a][sy][sx];
        qW[a] = qs[a][sy][sx - 1];
        qE[a] = qs[a][sy][sx + 1];
        qS[a] = twoD ? qs[a][sy - 1][sx] : qC[a];
        qN[a] = twoD ? qs[a][sy + 1][sx] : qC[a];
      }
      rhs_cell<T, NV>(c, qC, qW, qE, qS, qN, r);
      for (int a = 0; a < NV; ++a) q1s[a][ly][lx] = qC[a] + dt * r[a];
    }
    __syncthreads();
    // boundary values of the stage-1 state at t_k on non-periodic sides
    for (int idx = threadIdx.x; idx < H1Y * H1X; idx += blockDim.x) {
      const int ly = idx / H1X, lx = idx % H1X;
      if (!twoD && ly != 1) continue;
      const int gi = x0 + lx - 1, gj = twoD ? y0 + ly - 1 : 0;
      const bool outx = !((gi >= 0 && gi < c.nx) || c.bc[0] == HYROM_BC_PERIODIC);
      const bool outy = twoD && !((gj >= 0 && gj < c.ny) || c.bc[2] == HYROM_BC_PERIODIC);
      if (outx == outy) continue;  // inside, or an unused corner
      const int side = outx ? (gi < 0 ? 0 : 1) : (gj < 0 ? 2 : 3);
      if (c.bc[side] == HYROM_BC_SHOCK) {
        T s[4];
        shock_state<T>(c, gi, gj, t1, s);
        for (int a = 0; a < NV; ++a) q1s[a][ly][lx] = s[a];
      } else {
        const int cx = outx ? (gi < 0 ? lx + 1 : lx - 1) : lx;
        const int cy = outy ? (gj < 0 ? ly + 1 : ly - 1) : ly;
        for (int a = 0; a < NV; ++a) q1s[a][ly][lx] = q1s[a][cy][cx];
      }
    }
    __syncthreads();
    // stage 2 on the tile
    for (int idx = threadIdx.x; idx < TY * TX; idx += blockDim.x) {
      const int ly = idx / TX, lx = idx % TX;
      const int gi = x0 + lx, gj = y0 + ly;
      if (gi >= c.nx || gj >= c.ny) continue;
      const int64_t cell = (int64_t)gj * c.nx + gi;
      if (mask && !bit_get(mask, cell)) continue;
      T qC[NV], qW[NV], qE[NV], qS[NV], qN[NV], r[NV];
      const int sy = ly + 1, sx = lx + 1;
      for (int a = 0; a < NV; ++a) {
        qC[a] = q1s[a][sy][sx];
        qW[a] = q1s[a][sy][sx - 1];
        qE[a] = q1s[a][sy][sx + 1];
        qS[a] = twoD ? q1s[a][sy - 1][sx] : qC[a];
        qN[a] = twoD ? q1s[a][sy + 1][sx] : qC[a];
      }
      rhs_cell<T, NV>(c, qC, qW, qE, qS, qN, r);
      for (int a = 0; a < NV; ++a) {
        const T q0 = qs[a][ly + 2][lx + 2];
        out[a * c.nc + cell] = (T)0.5 * q0 + (T)0.5 * (qC[a] + dt * r[a]);
      }
    }
  }
}

// The same fused SSP-RK2 step for the Euler equations, with the work per
// cell cut to what the stencil needs: the primitives (u, v, p, c) of every
// staged cell are formed once, and every face flux once (a cell's residual
// is the difference of its face fluxes).  Each face is evaluated by
// rusanov_p on the same two states as rhs_cell evaluates it, so the step
// gives the same bits as k_rk2_tile.
template <typename T, int TX, int TY>
constexpr size_t rk2_euler_smem() {
  constexpr bool TWO = TY > 1;
  constexpr int HX = TX + 4, HY = TWO ? TY + 4 : 1, H1X = TX + 2, H1Y = TWO ? TY + 2 : 1;
  constexpr int NX1 = (TWO ? TY + 2 : 1) * (TX + 3), NY1 = TWO ? (TY + 3) * (TX + 2) : 0;
  // q on the tile + 2 ring, q1 on the tile + 1 ring, primitives (of q, then
  // of q1), x and y face fluxes (of stage 1, then of stage 2)
  return sizeof(T) * 4 * ((size_t)2 * HY * HX + H1Y * H1X + NX1 + NY1);
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256) k_rk2_euler(DevCfg c, const T* __restrict__ q,
                                                   T* __restrict__ out, int64_t k,
                                                   const uint32_t* __restrict__ mask,
                                                   const int* __restrict__ tiles,
                                                   const int* __restrict__ ntiles_dev,
                                                   int ntiles_all) {
  constexpr bool TWO = TY > 1;
  constexpr int HX = TX + 4, HY = TWO ? TY + 4 : 1, H1X = TX + 2, H1Y = TWO ? TY + 2 : 1;
  constexpr int NX1 = (TWO ? TY + 2 : 1) * (TX + 3), NY1 = TWO ? (TY + 3) * (TX + 2) : 0;
  constexpr int NX2 = TY * (TX + 1), NY2 = TWO ? (TY + 1) * TX : 0;
  constexpr int PQ = HY * HX, P1 = H1Y * H1X;  // per-variable strides
  extern __shared__ unsigned char rk_sm[];
  T* qs = reinterpret_cast<T*>(rk_sm);  // [4][HY][HX]
  T* q1s = qs + 4 * PQ;                  // [4][H1Y][H1X]
  T* ws = q1s + 4 * P1;                  // [4][HY][HX] (stage 2: [4][H1Y][H1X])
  T* fx = ws + 4 * PQ;                   // [4][NX1] (stage 2: [4][NX2])
  T* fy = fx + 4 * NX1;                  // [4][NY1] (stage 2: [4][NY2])
  const int tiles_x = (c.nx + TX - 1) / TX;
  const int ntiles = tiles ? *ntiles_dev : ntiles_all;
  const double t0 = (double)(k - 1) * c.dt, t1 = (double)k * c.dt;
  const T dt = (T)c.dt, dxT = (T)c.dx, dyT = (T)c.dy, g = (T)c.gamma;
  const bool perx = c.bc[0] == HYROM_BC_PERIODIC, pery = c.bc[2] == HYROM_BC_PERIODIC;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int tile = tiles ? tiles[it] : it;
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    // every staged cell inside the domain: plain loads, no ghost values
    const bool interior = x0 >= 2 && x0 + TX + 2 <= c.nx &&
                          (!TWO || (y0 >= 2 && y0 + TY + 2 <= c.ny));
    __syncthreads();
    // q on the tile and its two-cell ring (ghost values at t_{k-1}), and
    // the primitives of each staged cell
    for (int idx = threadIdx.x; idx < PQ; idx += blockDim.x) {
      const int sy = idx / HX, sx = idx % HX;
      T v[4], w[4];
      if (interior) {
        const int64_t cell = (int64_t)(TWO ? y0 + sy - 2 : 0) * c.nx + (x0 + sx - 2);
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = q[a * c.nc + cell];
      } else {
        fetch<T, 4>(c, q, x0 + sx - 2, TWO ? y0 + sy - 2 : 0, t0, v);
      }
      prims(v, g, w[0], w[1], w[2], w[3]);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        qs[a * PQ + idx] = v[a];
        ws[a * PQ + idx] = w[a];
      }
    }
    __syncthreads();
    // stage-1 face fluxes: x faces on the rows of the tile + 1 ring (face f
    // between staged columns f and f + 1), y faces on its columns
    for (int e = threadIdx.x; e < NX1 + NY1; e += blockDim.x) {
      int oL, oR;
      if (e < NX1) {
        const int r = e / (TX + 3), f = e % (TX + 3);
        oL = (TWO ? r + 1 : 0) * HX + f;
        oR = oL + 1;
      } else {
        const int f = (e - NX1) / (TX + 2), cx = (e - NX1) % (TX + 2);
        oL = f * HX + cx + 1;
        oR = oL + HX;
      }
      T qL[4], wL[4], qR[4], wR[4], F[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        qL[a] = qs[a * PQ + oL];
        wL[a] = ws[a * PQ + oL];
        qR[a] = qs[a * PQ + oR];
        wR[a] = ws[a * PQ + oR];
      }
      if (e < NX1) {
        rusanov_p<T, 0>(qL, wL, qR, wR, F);
#pragma unroll
        for (int a = 0; a < 4; ++a) fx[a * NX1 + e] = F[a];
      } else {
        rusanov_p<T, 1>(qL, wL, qR, wR, F);
#pragma unroll
        for (int a = 0; a < 4; ++a) fy[a * NY1 + (e - NX1)] = F[a];
      }
    }
    __syncthreads();
    // stage 1 on the tile and its one-cell ring (positions inside the
    // domain after periodic wrap)
    for (int idx = threadIdx.x; idx < P1; idx += blockDim.x) {
      const int ly = idx / H1X, lx = idx % H1X;
      const int gi = x0 + lx - 1, gj = TWO ? y0 + ly - 1 : 0;
      const bool inx = (gi >= 0 && gi < c.nx) || perx;
      const bool iny = !TWO || (gj >= 0 && gj < c.ny) || pery;
      if (!(inx && iny)) continue;
      const int sc = (TWO ? ly + 1 : 0) * HX + lx + 1;
      const int eL = ly * (TX + 3) + lx, eB = ly * (TX + 2) + lx;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T r = -(fx[a * NX1 + eL + 1] - fx[a * NX1 + eL]) / dxT;
        if (TWO) r = r - (fy[a * NY1 + eB + TX + 2] - fy[a * NY1 + eB]) / dyT;
        q1s[a * P1 + idx] = qs[a * PQ + sc] + dt * r;
      }
    }
    __syncthreads();
    // boundary values of the stage-1 state at t_k on non-periodic sides
    // (none on an interior tile)
    for (int idx = interior ? P1 : threadIdx.x; idx < P1; idx += blockDim.x) {
      const int ly = idx / H1X, lx = idx % H1X;
      const int gi = x0 + lx - 1, gj = TWO ? y0 + ly - 1 : 0;
      const bool outx = !((gi >= 0 && gi < c.nx) || perx);
      const bool outy = TWO && !((gj >= 0 && gj < c.ny) || pery);
      if (outx == outy) continue;  // inside, or an unused corner
      const int side = outx ? (gi < 0 ? 0 : 1) : (gj < 0 ? 2 : 3);
      if (c.bc[side] == HYROM_BC_SHOCK) {
        T s4[4];
        shock_state<T>(c, gi, gj, t1, s4);
#pragma unroll
        for (int a = 0; a < 4; ++a) q1s[a * P1 + idx] = s4[a];
      } else {
        const int cx = outx ? (gi < 0 ? lx + 1 : lx - 1) : lx;
        const int cy = outy ? (gj < 0 ? ly + 1 : ly - 1) : ly;
#pragma unroll
        for (int a = 0; a < 4; ++a) q1s[a * P1 + idx] = q1s[a * P1 + cy * H1X + cx];
      }
    }
    __syncthreads();
    // primitives of the stage-1 state (the unused corners of the ring
    // excepted)
    for (int idx = threadIdx.x; idx < P1; idx += blockDim.x) {
      const int ly = idx / H1X, lx = idx % H1X;
      if (TWO && (lx == 0 || lx == H1X - 1) && (ly == 0 || ly == H1Y - 1)) continue;
      T v[4], w[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) v[a] = q1s[a * P1 + idx];
      prims(v, g, w[0], w[1], w[2], w[3]);
#pragma unroll
      for (int a = 0; a < 4; ++a) ws[a * P1 + idx] = w[a];
    }
    __syncthreads();
    // stage-2 face fluxes on the tile
    for (int e = threadIdx.x; e < NX2 + NY2; e += blockDim.x) {
      int oL, oR;
      if (e < NX2) {
        const int r = e / (TX + 1), f = e % (TX + 1);
        oL = (TWO ? r + 1 : 0) * H1X + f;
        oR = oL + 1;
      } else {
        const int f = (e - NX2) / TX, cx = (e - NX2) % TX;
        oL = f * H1X + cx + 1;
        oR = oL + H1X;
      }
      T qL[4], wL[4], qR[4], wR[4], F[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        qL[a] = q1s[a * P1 + oL];
        wL[a] = ws[a * P1 + oL];
        qR[a] = q1s[a * P1 + oR];
        wR[a] = ws[a * P1 + oR];
      }
      if (e < NX2) {
        rusanov_p<T, 0>(qL, wL, qR, wR, F);
#pragma unroll
        for (int a = 0; a < 4; ++a) fx[a * NX2 + e] = F[a];
      } else {
        rusanov_p<T, 1>(qL, wL, qR, wR, F);
#pragma unroll
        for (int a = 0; a < 4; ++a) fy[a * NY2 + (e - NX2)] = F[a];
      }
    }
    __syncthreads();
    // stage 2 on the tile
    for (int idx = threadIdx.x; idx < TY * TX; idx += blockDim.x) {
      const int ly = idx / TX, lx = idx % TX;
      const int gi = x0 + lx, gj = y0 + ly;
      if (gi >= c.nx || gj >= c.ny) continue;
      const int64_t cell = (int64_t)gj * c.nx + gi;
      if (mask && !bit_get(mask, cell)) continue;
      const int s1 = (TWO ? ly + 1 : 0) * H1X + lx + 1;
      const int s0 = (TWO ? ly + 2 : 0) * HX + lx + 2;
      const int eL = ly * (TX + 1) + lx, eB = ly * TX + lx;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T r = -(fx[a * NX2 + eL + 1] - fx[a * NX2 + eL]) / dxT;
        if (TWO) r = r - (fy[a * NY2 + eB + TX] - fy[a * NY2 + eB]) / dyT;
        out[a * c.nc + cell] = (T)0.5 * qs[a * PQ + s0] + (T)0.5 * (q1s[a * P1 + s1] + dt * r);
      }
    }
  }
}

template <typename T>
void launch_rk2(const DevCfg& c, const T* q, T* out, int64_t k, const uint32_t* mask,
                const int* tiles, const int* ntiles_dev, cudaStream_t s) {
  const bool twoD = c.ny > 1;
  const int TX = twoD ? 32 : 256, TY = twoD ? 8 : 1;
  const int ntx = (c.nx + TX - 1) / TX, nty = (c.ny + TY - 1) / TY;
  const int nt = ntx * nty;
  int grid = tiles ? (nt < 152 * 8 ? nt : 152 * 8) : nt;
  if (grid < 1) grid = 1;
  if constexpr (sizeof(T) == 4) {
    // FP32 full step: the register-sweep kernel of hdm_f32.cu
    if (!mask && !tiles && rk2_euler_sweep_ok(c)) {
      launch_rk2_euler_sweep(c, (const float*)q, (float*)out, k, s);
      return;
    }
  }
  if (c.nvar == 4) {
    if (twoD) {
      constexpr size_t sm = rk2_euler_smem<T, 32, 8>();
      smem_at_least((const void*)k_rk2_euler<T, 32, 8>, sm);
      k_rk2_euler<T, 32, 8><<<grid, 256, sm, HY_S(s)>>>(c, q, out, k, mask, tiles, ntiles_dev, nt);
    } else {
      constexpr size_t sm = rk2_euler_smem<T, 256, 1>();
      smem_at_least((const void*)k_rk2_euler<T, 256, 1>, sm);
      k_rk2_euler<T, 256, 1><<<grid, 256, sm, HY_S(s)>>>(c, q, out, k, mask, tiles, ntiles_dev,
                                                          nt);
    }
  } else {
    if (twoD)
      k_rk2_tile<T, 1, 32, 8><<<grid, 256, 0, HY_S(s)>>>(c, q, out, k, mask, tiles, ntiles_dev, nt);
    else
      k_rk2_tile<T, 1, 256, 1><<<grid, 256, 0, HY_S(s)>>>(c, q, out, k, mask, tiles, ntiles_dev, nt);
  }
}

int rk2_tile_width(const DevCfg& c) { return c.ny > 1 ? 32 : 256; }
int rk2_tile_height(const DevCfg& c) { return c.ny > 1 ? 8 : 1; }

// ---------------------------------------------------------------------------
// per-cell BDF1 residual measure rho_i = sum_v |R_v|,
// R = (q - q_prev) - dt f*(q, t)   (the filter's error indicator)
// ---------------------------------------------------------------------------

template <typename T, int NV>
__global__ void k_cell_residual(DevCfg c, const T* __restrict__ q, const T* __restrict__ qp,
                                double t, T* __restrict__ rho, const uint32_t* __restrict__ only,
                                const int* __restrict__ skip) {
  if (skip && *skip) return;
  const bool twoD = c.ny > 1;
  const T dt = (T)c.dt;
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < c.nc;
       cell += (int64_t)gridDim.x * blockDim.x) {
    if (only && !bit_get(only, cell)) continue;
    const int gi = (int)(cell % c.nx), gj = (int)(cell / c.nx);
    T qC[NV], qW[NV], qE[NV], qS[NV], qN[NV], r[NV];
    for (int a = 0; a < NV; ++a) qC[a] = q[a * c.nc + cell];
    fetch<T, NV>(c, q, gi - 1, gj, t, qW);
    fetch<T, NV>(c, q, gi + 1, gj, t, qE);
    if (twoD) {
      fetch<T, NV>(c, q, gi, gj - 1, t, qS);
      fetch<T, NV>(c, q, gi, gj + 1, t, qN);
    } else {
      for (int a = 0; a < NV; ++a) qS[a] = qN[a] = qC[a];
    }
    rhs_cell<T, NV>(c, qC, qW, qE, qS, qN, r);
    T acc = (T)0;
    for (int a = 0; a < NV; ++a) {
      const T R = (qC[a] - qp[a * c.nc + cell]) - dt * r[a];
      acc = a == 0 ? fabs(R) : acc + fabs(R);
    }
    rho[cell] = acc;
  }
}

template <typename T>
void launch_cell_residual(const DevCfg& c, const T* q, const T* qp, int64_t k, T* rho,
                          const uint32_t* only, cudaStream_t s) {
  const double t = (double)k * c.dt;
  int64_t blocks = (c.nc + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (c.nvar == 4)
    k_cell_residual<T, 4><<<(int)blocks, 256, 0, HY_S(s)>>>(c, q, qp, t, rho, only, nullptr);
  else
    k_cell_residual<T, 1><<<(int)blocks, 256, 0, HY_S(s)>>>(c, q, qp, t, rho, only, nullptr);
}

template <typename T>
void launch_cell_residual_skip(const DevCfg& c, const T* q, const T* qp, int64_t k, T* rho,
                               const int* skip, cudaStream_t s) {
  const double t = (double)k * c.dt;
  int64_t blocks = (c.nc + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (c.nvar == 4)
    k_cell_residual<T, 4><<<(int)blocks, 256, 0, HY_S(s)>>>(c, q, qp, t, rho, nullptr, skip);
  else
    k_cell_residual<T, 1><<<(int)blocks, 256, 0, HY_S(s)>>>(c, q, qp, t, rho, nullptr, skip);
}

// ---------------------------------------------------------------------------
// Burgers BDF1 solved by Newton (FP64)
// ---------------------------------------------------------------------------

HY_DEV void godunov_d(double uL, double uR, double& dL, double& dR) {
  const double a = uL > 0.0 ? uL : 0.0;
  const double b = uR < 0.0 ? uR : 0.0;
  const bool left = 0.5 * a * a >= 0.5 * b * b;
  dL = left ? a : 0.0;
  dR = left ? 0.0 : b;
}

HY_DEV double burgers_R(const DevCfg& c, const double* u, const double* up, int i) {
  const int n = c.nx;
  const double uW = u[imod(i - 1, n)], uC = u[i], uE = u[imod(i + 1, n)];
  const double Fl = godunov<double>(uW, uC), Fr = godunov<double>(uC, uE);
  const double r = -(Fr - Fl) / c.dx;
  return (uC - up[i]) - c.dt * r;
}

HY_DEV void burgers_J(const DevCfg& c, const double* u, int i, double& sub, double& dia,
                      double& sup) {
  const int n = c.nx;
  const double lam = c.dt / c.dx;
  double dLm, dRm, dLp, dRp;
  godunov_d(u[imod(i - 1, n)], u[i], dLm, dRm);
  godunov_d(u[i], u[imod(i + 1, n)], dLp, dRp);
  sub = -lam * dLm;
  dia = 1.0 + lam * (dLp - dRm);
  sup = lam * dRp;
}

// Newton on all cells of the periodic grid: residual and Jacobian in
// parallel, the cyclic tridiagonal solve (Sherman-Morrison with two Thomas
// sweeps) by one thread.  ws: 6*n doubles.
__global__ void k_burgers_newton_full(DevCfg c, const double* __restrict__ up, double* u,
                                      const double* __restrict__ tol_dev, int newton_max,
                                      double* ws, int* fail) {
  const int n = c.nx;
  double *A = ws, *B = ws + n, *C = ws + 2 * n, *R = ws + 3 * n, *X = ws + 4 * n, *Z = ws + 5 * n;
  const double tol = *tol_dev;
  for (int it = 0;; ++it) {
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double r = burgers_R(c, u, up, i);
      R[i] = r;
      mx = fmax(mx, fabs(r));
      burgers_J(c, u, i, A[i], B[i], C[i]);
    }
    mx = block_max(mx);
    if (mx <= tol) return;
    if (it >= newton_max) {
      if (threadIdx.x == 0) atomicAdd(fail, 1);
      return;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // cyclic system: A[0] multiplies x[n-1], C[n-1] multiplies x[0]
      const double g = -B[0];
      const double b0 = B[0] - g, bl = B[n - 1] - A[0] * C[n - 1] / g;
      // Thomas on the modified tridiagonal for rhs R -> X and rhs u -> Z
      double cp_prev = 0.0, xp = 0.0, zp = 0.0;
      for (int i = 0; i < n; ++i) {
        const double bi = i == 0 ? b0 : (i == n - 1 ? bl : B[i]);
        const double ai = i == 0 ? 0.0 : A[i];
        const double den = bi - ai * cp_prev;
        const double ci = i == n - 1 ? 0.0 : C[i];
        const double ri = R[i];
        const double ui = i == 0 ? g : (i == n - 1 ? C[n - 1] : 0.0);
        const double cpi = ci / den;
        xp = (ri - ai * xp) / den;
        zp = (ui - ai * zp) / den;
        X[i] = xp;
        Z[i] = zp;
        R[i] = cpi;  // reuse R as c'
        cp_prev = cpi;
      }
      for (int i = n - 2; i >= 0; --i) {
        X[i] = X[i] - R[i] * X[i + 1];
        Z[i] = Z[i] - R[i] * Z[i + 1];
      }
      const double fact = (X[0] + A[0] * X[n - 1] / g) / (1.0 + Z[0] + A[0] * Z[n - 1] / g);
      for (int i = 0; i < n; ++i) X[i] = X[i] - fact * Z[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) u[i] = u[i] - X[i];
    __syncthreads();
  }
}

// Segment starts of S-hat (cells in S-hat whose left neighbour is not).
__global__ void k_segment_starts(DevCfg c, const uint32_t* __restrict__ s_hat, int* starts,
                                 int* nstart) {
  const int n = c.nx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (bit_get(s_hat, i) && !bit_get(s_hat, imod(i - 1, n))) starts[atomicAdd(nstart, 1)] = i;
  }
}

// Newton on one contiguous segment of S-hat per thread; the neighbours
// outside the segment are frozen (S-tilde values of u).  ws: 4*n doubles
// indexed by cell (segments are disjoint).
__global__ void k_burgers_newton_seg(DevCfg c, const double* __restrict__ up, double* u,
                                     const uint32_t* __restrict__ s_hat,
                                     const int* __restrict__ starts,
                                     const int* __restrict__ nstart,
                                     const double* __restrict__ tol_dev, int newton_max,
                                     double* ws, int* fail) {
  const int n = c.nx;
  const int ns = *nstart;
  const double tol = *tol_dev;
  double *A = ws, *B = ws + n, *C = ws + 2 * n, *R = ws + 3 * n;
  for (int sgi = blockIdx.x * blockDim.x + threadIdx.x; sgi < ns; sgi += gridDim.x * blockDim.x) {
    const int s = starts[sgi];
    int len = 0;
    while (len < n && bit_get(s_hat, (s + len) % n)) ++len;
    for (int it = 0;; ++it) {
      double mx = 0.0;
      for (int l = 0; l < len; ++l) {
        const int i = (s + l) % n;
        const double r = burgers_R(c, u, up, i);
        R[i] = r;
        mx = fmax(mx, fabs(r));
        burgers_J(c, u, i, A[i], B[i], C[i]);
      }
      if (mx <= tol) break;
      if (it >= newton_max) {
        atomicAdd(fail, 1);
        break;
      }
      // Thomas (sub-diagonal of the first and super-diagonal of the last
      // unknown multiply frozen values and drop out)
      double cp = 0.0, xp = 0.0;
      for (int l = 0; l < len; ++l) {
        const int i = (s + l) % n;
        const double ai = l == 0 ? 0.0 : A[i];
        const double den = B[i] - ai * cp;
        const double ci = l == len - 1 ? 0.0 : C[i];
        cp = ci / den;
        xp = (R[i] - ai * xp) / den;
        A[i] = cp;  // store c'
        R[i] = xp;  // store x'
      }
      double xn = 0.0;
      for (int l = len - 1; l >= 0; --l) {
        const int i = (s + l) % n;
        const double x = l == len - 1 ? R[i] : R[i] - A[i] * xn;
        xn = x;
        u[i] = u[i] - x;
      }
    }
  }
}

__global__ void k_absmax(const double* __restrict__ x, int64_t n, double scale, double* out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  m = block_max(m);
  if (threadIdx.x == 0) *out = scale * fmax(1.0, m);
}

void launch_newton_tol(const DevCfg& c, const double* qp, double newton_tol, double* tol_dev,
                       cudaStream_t s) {
  k_absmax<<<1, 1024, 0, HY_S(s)>>>(qp, c.ndof, newton_tol, tol_dev);
}

void launch_burgers_newton_full(const DevCfg& c, const double* up, double* u,
                                const double* tol_dev, int newton_max, double* ws, int* fail,
                                cudaStream_t s) {
  k_burgers_newton_full<<<1, 1024, 0, HY_S(s)>>>(c, up, u, tol_dev, newton_max, ws, fail);
}

void launch_burgers_newton_partial(const DevCfg& c, const double* up, double* u,
                                   const uint32_t* s_hat, int* starts, int* nstart,
                                   const double* tol_dev, int newton_max, double* ws, int* fail,
                                   cudaStream_t s) {
  cudaMemsetAsync(nstart, 0, sizeof(int), s);
  k_segment_starts<<<(c.nx + 255) / 256, 256, 0, HY_S(s)>>>(c, s_hat, starts, nstart);
  k_burgers_newton_seg<<<(c.nx + 127) / 128, 128, 0, HY_S(s)>>>(c, up, u, s_hat, starts, nstart,
                                                          tol_dev, newton_max, ws, fail);
}

// Cells of an Euler state that are not physical: rho <= 0, p <= 0 (ideal
// gas, Sec. 3.1), or either not finite.  One count per call into *count
// (which the caller clears).
template <typename T>
__global__ void k_count_nonphys(DevCfg c, const T* __restrict__ q, int* __restrict__ count) {
  int bad = 0;
  const T g1 = (T)(c.gamma - 1.0);
  const T inf = (T)INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.nc;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T r = q[i], mx = q[c.nc + i], my = q[2 * c.nc + i], en = q[3 * c.nc + i];
    const T p = g1 * (en - (T)0.5 * (mx * mx + my * my) / r);
    bad += !(r > (T)0 && r < inf && p > (T)0 && p < inf);
  }
  bad = __reduce_add_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, bad);
}

template <typename T>
void launch_count_nonphys(const DevCfg& c, const T* q, int* count, cudaStream_t s) {
  int64_t blocks = (c.nc + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_count_nonphys<T><<<(int)blocks, 256, 0, HY_S(s)>>>(c, q, count);
}

template void launch_count_nonphys<float>(const DevCfg&, const float*, int*, cudaStream_t);
template void launch_count_nonphys<double>(const DevCfg&, const double*, int*, cudaStream_t);
template void launch_rk2<float>(const DevCfg&, const float*, float*, int64_t, const uint32_t*,
                                 const int*, const int*, cudaStream_t);
template void launch_rk2<double>(const DevCfg&, const double*, double*, int64_t, const uint32_t*,
                                  const int*, const int*, cudaStream_t);
template void launch_cell_residual<float>(const DevCfg&, const float*, const float*, int64_t,
                                          float*, const uint32_t*, cudaStream_t);
template void launch_cell_residual<double>(const DevCfg&, const double*, const double*, int64_t,
                                           double*, const uint32_t*, cudaStream_t);
template void launch_cell_residual_skip<float>(const DevCfg&, const float*, const float*,
                                               int64_t, float*, const int*, cudaStream_t);
template void launch_cell_residual_skip<double>(const DevCfg&, const double*, const double*,
                                                int64_t, double*, const int*, cudaStream_t);

}  // namespace hy
