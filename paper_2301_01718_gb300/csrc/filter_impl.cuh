// The body of the residual-gated filter (templates), compiled twice: in
// filter.cu for FP64 states with the library's IEEE arithmetic (the
// oracle's operation order, bit for bit), and in filter_f32.cu for FP32
// states with contraction and approximate division and square root (the
// FP32 path's tolerance is 1e-5; its gate decisions near a tie may differ).
#pragma once
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
#include "phys.cuh"

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

// ctl[0] = done, ctl[1] = passes run, ctl[2] = cells kept (running total),
// ctl[3] = CTAs of the current pass finished, ctl[4] = pass stamp.  The
// pass's totals over its CTAs' partials (fixed order) and the stop test:
// no cell kept, or the kept cells' decrease below eps_f of their total.
HY_DEV void gate_close(const double* __restrict__ part, int nblk, double eps_f, int* ctl) {
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
    ctl[3] = 0;
    ctl[4] += 1;
  }
}

static __global__ void k_set_int(int* p, int v) { *p = v; }


// ---------------------------------------------------------------------------
// fused, sparse filter pass
//
// One kernel per pass computes, for every cell of a tile, rho_old = rho(q),
// the filtered state g = F_y(F_x(q)) and rho_new = rho(g) in shared memory
// and takes the gate decision; kept cells get g in gbuf and a bit in kbits.
// The filter is the two one-dimensional sweeps (x, then y) with the weights
// above, evaluated in that order.  After the first pass of an order,
// q has changed only on the kept cells K, so g can change only within
// distance n of K and rho_old / rho_new only within distance n + 1: every
// other cell keeps its previous decision ("not kept").  The next pass
// therefore visits only the tiles within n + 1 cells of K.
// ---------------------------------------------------------------------------

template <typename T, int NV>
HY_DEV void nb_value(const DevCfg& c, const T* sm, int stride_v, int pos, int gi, int gj, double t,
                     T* out) {
  // neighbour value for the residual: smem value (in-domain, wrapped or
  // clamped), or the exact shock state on a shock side
  const bool outx = (gi < 0 || gi >= c.nx) && c.bc[0] != HYROM_BC_PERIODIC;
  const bool outy = c.ny > 1 && (gj < 0 || gj >= c.ny) && c.bc[2] != HYROM_BC_PERIODIC;
  if (outx || outy) {
    const int side = outx ? (gi < 0 ? 0 : 1) : (gj < 0 ? 2 : 3);
    if (c.bc[side] == HYROM_BC_SHOCK) {
      T s4[4];
      shock_state<T>(c, gi, gj, t, s4);
      for (int a = 0; a < NV; ++a) out[a] = s4[a];
      return;
    }
  }
  for (int a = 0; a < NV; ++a) out[a] = sm[a * stride_v + pos];
}

// The per-call arguments of the passes (the state filtered in place, the
// previous state, the time), read from device memory so that one captured
// graph of the whole filter serves every call.
template <typename T>
struct FiltArgs {
  T* q;
  const T* qp;
  double t;
  // optional record of the passes run (the adjoint's forward tape): pass p's
  // keep bitmap at keeps + p * nwords, its Shapiro n at orders[p], the
  // number recorded in *count (null keeps: nothing is recorded)
  uint32_t* keeps;
  int* orders;
  int* count;
};

template <typename T>
__global__ void k_set_filt_args(FiltArgs<T>* fa, T* q, const T* qp, double t, uint32_t* keeps,
                                int* orders, int* count) {
  fa->q = q;
  fa->qp = qp;
  fa->t = t;
  fa->keeps = keeps;
  fa->orders = orders;
  fa->count = count;
  if (count) *count = 0;
}

// Record this pass's keep bitmap and order when it ran (ctl[1], the passes
// run, moved past the count recorded so far) and a record is asked for.
template <typename T>
__global__ void k_tape_pass(const FiltArgs<T>* __restrict__ fa, const uint32_t* __restrict__ kbits,
                            int64_t nwords, int n, const int* __restrict__ ctl) {
  if (!fa->keeps) return;
  const int ran = ctl[1];
  const int have = *fa->count;
  if (ran <= have) return;
  uint32_t* dst = fa->keeps + (int64_t)have * nwords;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = kbits[i];
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) fa->orders[have] = n;
}

template <typename T>
__global__ void k_tape_commit(const FiltArgs<T>* __restrict__ fa, const int* __restrict__ ctl) {
  if (fa->keeps && ctl[1] > *fa->count) *fa->count = ctl[1];
}

// shared memory of k_filter_pass: q on the tile and an NF+1 halo, F_x q,
// g on the tile and a one-cell ring; for the Euler equations also the
// resolved q and g on that ring, their primitives and the face fluxes
template <typename T, int NV, int NF, int TX, int TY>
constexpr size_t filter_pass_smem() {
  constexpr bool TWO = TY > 1;
  constexpr int H = NF + 1, SX = TX + 2 * H, SY = TWO ? TY + 2 * H : 1;
  constexpr int GX = TX + 2, GY = TWO ? TY + 2 : 1;
  size_t n = (size_t)NV * (SY * SX + SY * GX + GY * GX);
  if (NV == 4)
    n += (size_t)2 * NV * GY * GX + 2 * 4 * GY * GX + 2 * NV * TY * (TX + 1) +
         (TWO ? 2 * NV * (TY + 1) * TX : 0);
  return sizeof(T) * n;
}

template <typename T, int NV, int NF, int TX, int TY>
__global__ void __launch_bounds__(256, 3) k_filter_pass(DevCfg c, const FiltArgs<T>* __restrict__ fa,
                                                     T* __restrict__ gbuf, uint32_t* __restrict__ kbits,
                                                     const int* __restrict__ tiles,
                                                     const int* __restrict__ ntiles_dev,
                                                     int ntiles_all, double* __restrict__ part,
                                                     int* __restrict__ ctl, double eps_f) {
  constexpr bool TWO = TY > 1;
  constexpr int H = NF + 1;
  constexpr int SX = TX + 2 * H, SY = TWO ? TY + 2 * H : 1;
  constexpr int FX = TX + 2, FY = SY;  // F_x rows aligned with the q rows
  constexpr int GX = TX + 2, GY = TWO ? TY + 2 : 1;
  extern __shared__ unsigned char fsm[];
  T* qs = reinterpret_cast<T*>(fsm);
  T* fx = qs + NV * SY * SX;
  T* gs = fx + NV * FY * FX;
  if (*(volatile int*)ctl) return;
  const T* __restrict__ q = fa->q;
  const T* __restrict__ qp = fa->qp;
  const double t = fa->t;
  const int tiles_x = (c.nx + TX - 1) / TX;
  const int ntiles = tiles ? *ntiles_dev : ntiles_all;
  const bool perx = c.bc[0] == HYROM_BC_PERIODIC, pery = c.bc[2] == HYROM_BC_PERIODIC;
  const T scale = (T)(NF == 1 ? 0.25 : (NF == 2 ? 0.0625 : 0.015625));
  // the constants in the state's precision, converted once (a conversion
  // from FP64 runs on the narrow FP64 pipe)
  const T dt = (T)c.dt;
  const T gam = (T)c.gamma, dxT = (T)c.dx, dyT = (T)c.dy;
  // the gate's totals: a thread's sums in the state's precision (one kept
  // cell per thread and tile), the CTA's too, combined over CTAs in FP64
  int cnt_i = 0;
  T dec_t = (T)0, tot_t = (T)0;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int tile = tiles ? tiles[it] : it;
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    __syncthreads();
    // q on the tile and an H-cell halo (periodic sides wrap, others clamp)
    // (all of a thread's loads are issued before its stores)
    constexpr int kPer = (SY * SX + 255) / 256;
    T stage[kPer][NV];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int idx = threadIdx.x + u * 256;
      if (idx < SY * SX) {
        const int sy = idx / SX, sx = idx % SX;
        int gi = x0 - H + sx, gj = TWO ? y0 - H + sy : 0;
        gi = perx ? imod(gi, c.nx) : (gi < 0 ? 0 : (gi >= c.nx ? c.nx - 1 : gi));
        if (TWO) gj = pery ? imod(gj, c.ny) : (gj < 0 ? 0 : (gj >= c.ny ? c.ny - 1 : gj));
        const int64_t cell = (int64_t)gj * c.nx + gi;
#pragma unroll
        for (int a = 0; a < NV; ++a) stage[u][a] = q[a * c.nc + cell];
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int idx = threadIdx.x + u * 256;
      if (idx < SY * SX) {
        const int sy = idx / SX, sx = idx % SX;
#pragma unroll
        for (int a = 0; a < NV; ++a) qs[(a * SY + sy) * SX + sx] = stage[u][a];
      }
    }
    __syncthreads();
    // F_x on columns tile +- 1, every staged row (rows hold clamped/wrapped
    // data; row fy is global row y0 - H + fy, like the q rows)
    for (int idx = threadIdx.x; idx < FY * FX; idx += blockDim.x) {
      const int fy = idx / FX, fxc = idx % FX;
      const int sy = fy, sx = fxc + NF;
      for (int a = 0; a < NV; ++a) {
        const T* row = qs + (a * SY + sy) * SX;
        T acc = (T)0;
#pragma unroll
        for (int tt = 0; tt < 2 * NF + 1; ++tt) {
          const double wt = Shapiro<NF>::w(tt);
          const T x = row[sx + tt - NF];
          const T term = wt == 1.0 ? x : (wt == -1.0 ? -x : (T)wt * x);
          acc = tt == 0 ? term : acc + term;
        }
        fx[(a * FY + fy) * FX + fxc] = acc * scale;
      }
    }
    __syncthreads();
    // g = F_y(F_x q) on tile +- 1: g row gy is global row y0 - 1 + gy, whose
    // taps are F_x rows gy + tt (tt = 0..2 NF) since H - 1 = NF
    for (int idx = threadIdx.x; idx < GY * GX; idx += blockDim.x) {
      const int gy = idx / GX, gx = idx % GX;
      for (int a = 0; a < NV; ++a) {
        T val;
        if (TWO) {
          T acc = (T)0;
#pragma unroll
          for (int tt = 0; tt < 2 * NF + 1; ++tt) {
            const double wt = Shapiro<NF>::w(tt);
            const T x = fx[(a * FY + gy + tt) * FX + gx];
            const T term = wt == 1.0 ? x : (wt == -1.0 ? -x : (T)wt * x);
            acc = tt == 0 ? term : acc + term;
          }
          val = acc * scale;
        } else {
          val = fx[a * FX + gx];
        }
        gs[(a * GY + gy) * GX + gx] = val;
      }
    }
    __syncthreads();
    if constexpr (NV == 4) {
      // Euler: the states the residuals read (q and g on the tile and its
      // one-cell ring, ghost values resolved), their primitives once per
      // cell, and each face flux once per face
      T* qe = gs + NV * GY * GX;
      T* ge = qe + NV * GY * GX;
      T* wq = ge + NV * GY * GX;  // u, v, p, c of qe
      T* wg = wq + 4 * GY * GX;
      T* fxq = wg + 4 * GY * GX;  // x faces: row ly, face lx between ring columns lx, lx + 1
      T* fxg = fxq + NV * TY * (TX + 1);
      T* fyq = fxg + NV * TY * (TX + 1);  // y faces: row ly between ring rows ly, ly + 1
      T* fyg = fyq + (TWO ? NV * (TY + 1) * TX : 0);
      const T g = gam;
      for (int idx = threadIdx.x; idx < GY * GX; idx += blockDim.x) {
        const int gy = idx / GX, gx = idx % GX;
        if (TWO && (gx == 0 || gx == GX - 1) && (gy == 0 || gy == GY - 1)) continue;  // unused
        const int gi = x0 - 1 + gx, gj = TWO ? y0 - 1 + gy : 0;
        T qv[NV], gv[NV];
        // q: the staged (wrapped or clamped) value, or the shock state
        nb_value<T, NV>(c, qs, SY * SX, (TWO ? gy + H - 1 : 0) * SX + gx + H - 1, gi, gj, t, qv);
        // g: outside a non-periodic side, the boundary cell's g (or the
        // shock state)
        int gxe = gx, gye = gy;
        if (!perx) gxe = gi < 0 ? gx + 1 : (gi >= c.nx ? gx - 1 : gx);
        if (TWO && !pery) gye = gj < 0 ? gy + 1 : (gj >= c.ny ? gy - 1 : gy);
        nb_value<T, NV>(c, gs, GY * GX, gye * GX + gxe, gi, gj, t, gv);
        T wv[4], ww[4];
        prims(qv, g, wv[0], wv[1], wv[2], wv[3]);
        prims(gv, g, ww[0], ww[1], ww[2], ww[3]);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          qe[(a * GY + gy) * GX + gx] = qv[a];
          ge[(a * GY + gy) * GX + gx] = gv[a];
          wq[(a * GY + gy) * GX + gx] = wv[a];
          wg[(a * GY + gy) * GX + gx] = ww[a];
        }
      }
      __syncthreads();
      constexpr int NFX = TY * (TX + 1), NFY = TWO ? (TY + 1) * TX : 0;
      for (int f = threadIdx.x; f < 2 * (NFX + NFY); f += blockDim.x) {
        const bool isg = f >= NFX + NFY;
        const int e = isg ? f - (NFX + NFY) : f;
        const T* S = isg ? ge : qe;
        const T* Wp = isg ? wg : wq;
        T qL[4], wL[4], qR[4], wR[4], F[4];
        int oL, oR;
        if (e < NFX) {
          const int ly = e / (TX + 1), lx = e % (TX + 1), gy = TWO ? ly + 1 : 0;
          oL = gy * GX + lx;
          oR = oL + 1;
        } else {
          const int ly = (e - NFX) / TX, lx = (e - NFX) % TX;
          oL = ly * GX + lx + 1;
          oR = oL + GX;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          qL[a] = S[a * GY * GX + oL];
          qR[a] = S[a * GY * GX + oR];
          wL[a] = Wp[a * GY * GX + oL];
          wR[a] = Wp[a * GY * GX + oR];
        }
        if (e < NFX) {
          rusanov_p<T, 0>(qL, wL, qR, wR, F);
          T* dst = isg ? fxg : fxq;
#pragma unroll
          for (int a = 0; a < 4; ++a) dst[a * NFX + e] = F[a];
        } else {
          rusanov_p<T, 1>(qL, wL, qR, wR, F);
          T* dst = isg ? fyg : fyq;
#pragma unroll
          for (int a = 0; a < 4; ++a) dst[a * NFY + (e - NFX)] = F[a];
        }
      }
      __syncthreads();
      // residual measures and the gate on the tile (the operator's
      // expressions of rhs_cell, from the shared face fluxes)
      for (int idx = threadIdx.x; idx < TY * TX; idx += blockDim.x) {
        const int ly = idx / TX, lx = idx % TX;
        const int gi = x0 + lx, gj = y0 + ly;
        if (gi >= c.nx || gj >= c.ny) continue;
        const int64_t cell = (int64_t)gj * c.nx + gi;
        const int oc = (TWO ? ly + 1 : 0) * GX + lx + 1;
        const int fx0 = ly * (TX + 1) + lx, fy0 = ly * TX + lx;
        T ro = (T)0, rn = (T)0;
        T gC[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T r = -(fxq[a * NFX + fx0 + 1] - fxq[a * NFX + fx0]) / dxT;
          T rg = -(fxg[a * NFX + fx0 + 1] - fxg[a * NFX + fx0]) / dxT;
          if (TWO) {
            r = r - (fyq[a * NFY + fy0 + TX] - fyq[a * NFY + fy0]) / dyT;
            rg = rg - (fyg[a * NFY + fy0 + TX] - fyg[a * NFY + fy0]) / dyT;
          }
          const T qC = qe[a * GY * GX + oc];
          gC[a] = ge[a * GY * GX + oc];
          const T p = qp[a * c.nc + cell];
          const T Ro = (qC - p) - dt * r;
          const T Rn = (gC[a] - p) - dt * rg;
          ro = a == 0 ? fabs(Ro) : ro + fabs(Ro);
          rn = a == 0 ? fabs(Rn) : rn + fabs(Rn);
        }
        if (rn < ro) {
#pragma unroll
          for (int a = 0; a < 4; ++a) gbuf[a * c.nc + cell] = gC[a];
          atomicOr(&kbits[cell >> 5], 1u << (cell & 31));
          ++cnt_i;
          dec_t += ro - rn;
          tot_t += ro;
        }
      }
    } else {
    // Burgers: residual measures and the gate on the tile
    for (int idx = threadIdx.x; idx < TY * TX; idx += blockDim.x) {
      const int ly = idx / TX, lx = idx % TX;
      const int gi = x0 + lx, gj = y0 + ly;
      if (gi >= c.nx || gj >= c.ny) continue;
      const int64_t cell = (int64_t)gj * c.nx + gi;
      T qC[NV], qW[NV], qE[NV], qS[NV], qN[NV], r[NV];
      T gC[NV], gW[NV], gE[NV], gS[NV], gN[NV], rg[NV];
      // q neighbours (clamped smem == outflow ghost; shock sides exact)
      const int qsy = TWO ? ly + H : 0, qsx = lx + H;
      const int qv = SY * SX;
      nb_value<T, NV>(c, qs, qv, qsy * SX + qsx, gi, gj, t, qC);
      nb_value<T, NV>(c, qs, qv, qsy * SX + qsx - 1, gi - 1, gj, t, qW);
      nb_value<T, NV>(c, qs, qv, qsy * SX + qsx + 1, gi + 1, gj, t, qE);
      if (TWO) {
        nb_value<T, NV>(c, qs, qv, (qsy - 1) * SX + qsx, gi, gj - 1, t, qS);
        nb_value<T, NV>(c, qs, qv, (qsy + 1) * SX + qsx, gi, gj + 1, t, qN);
      } else {
        for (int a = 0; a < NV; ++a) qS[a] = qN[a] = qC[a];
      }
      // g neighbours: out-of-domain non-periodic positions take the
      // boundary cell's g (outflow) or the shock state
      const int gy = TWO ? ly + 1 : 0, gx = lx + 1, gv = GY * GX;
      const int wxm = (gi - 1 < 0 && !perx) ? gx : gx - 1;
      const int wxp = (gi + 1 >= c.nx && !perx) ? gx : gx + 1;
      nb_value<T, NV>(c, gs, gv, gy * GX + gx, gi, gj, t, gC);
      nb_value<T, NV>(c, gs, gv, gy * GX + wxm, gi - 1, gj, t, gW);
      nb_value<T, NV>(c, gs, gv, gy * GX + wxp, gi + 1, gj, t, gE);
      if (TWO) {
        const int wym = (gj - 1 < 0 && !pery) ? gy : gy - 1;
        const int wyp = (gj + 1 >= c.ny && !pery) ? gy : gy + 1;
        nb_value<T, NV>(c, gs, gv, wym * GX + gx, gi, gj - 1, t, gS);
        nb_value<T, NV>(c, gs, gv, wyp * GX + gx, gi, gj + 1, t, gN);
      } else {
        for (int a = 0; a < NV; ++a) gS[a] = gN[a] = gC[a];
      }
      rhs_cell<T, NV>(c, qC, qW, qE, qS, qN, r);
      rhs_cell<T, NV>(c, gC, gW, gE, gS, gN, rg);
      T ro = (T)0, rn = (T)0;
      for (int a = 0; a < NV; ++a) {
        const T p = qp[a * c.nc + cell];
        const T Ro = (qC[a] - p) - dt * r[a];
        const T Rn = (gC[a] - p) - dt * rg[a];
        ro = a == 0 ? fabs(Ro) : ro + fabs(Ro);
        rn = a == 0 ? fabs(Rn) : rn + fabs(Rn);
      }
      if (rn < ro) {
        for (int a = 0; a < NV; ++a) gbuf[a * c.nc + cell] = gC[a];
        atomicOr(&kbits[cell >> 5], 1u << (cell & 31));
        ++cnt_i;
        dec_t += ro - rn;
        tot_t += ro;
      }
    }
    }
  }
  // over the CTA in the state's precision (the count exactly), then FP64
  double cnt = 0.0, dec = 0.0, tot = 0.0;
  if ((int)blockIdx.x < ntiles) {  // (a CTA without a tile adds nothing)
    cnt = (double)block_sum(cnt_i);
    dec = (double)block_sum(dec_t);
    tot = (double)block_sum(tot_t);
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = cnt;
    part[3 * blockIdx.x + 1] = dec;
    part[3 * blockIdx.x + 2] = tot;
  }
  // the CTA that finishes last closes the pass: the kept count, the stop
  // test, and the stamp of the next tile search (ctl[3]: CTAs finished,
  // ctl[4]: pass stamp)
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&ctl[3], 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  gate_close(part, gridDim.x, eps_f, ctl);
}

// any bit set in [b, b + len) of the bitmap (len <= 64: at most 3 words)
HY_DEV bool bits_any(const uint32_t* __restrict__ bm, int64_t b, int len) {
  const int64_t w0 = b >> 5;
  const int off = (int)(b & 31);
  const int64_t e = b + len;  // exclusive end
  const int64_t w_last = (e - 1) >> 5;
  uint32_t acc = 0u;
  for (int64_t wd = w0; wd <= w_last; ++wd) {
    uint32_t v = bm[wd];
    if (wd == w0) v &= 0xffffffffu << off;
    if (wd == w_last) {
      const int hi = (int)((e - 1) & 31);
      v &= hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u);
    }
    acc |= v;
  }
  return acc != 0u;
}

// Whether tile t has a kept cell within R cells (x and y), by one warp.
// Interior tiles: lane r reads neighbourhood row r (TY + 2R rows) as at most
// three masked words of the bitmap, and a ballot combines the rows.  Tiles
// whose neighbourhood crosses the domain edge (and 1D tiles, wider than 64
// cells) take the per-cell path with the periodic wrap or the clip, their
// cells spread over the lanes 32 at a time.
HY_DEV bool tile_near_kept(const DevCfg& c, const uint32_t* __restrict__ kbits, int TX, int TY,
                           int R, int t) {
  const int lane = threadIdx.x & 31;
  const int tx = (c.nx + TX - 1) / TX;
  const bool twoD = c.ny > 1;
  const bool perx = c.bc[0] == HYROM_BC_PERIODIC, pery = c.bc[2] == HYROM_BC_PERIODIC;
  const int Ry = twoD ? R : 0;
  const int nrows = TY + 2 * Ry, ncols = TX + 2 * R;
  const int x0 = (t % tx) * TX, y0 = (t / tx) * TY;
  const bool inx = x0 - R >= 0 && x0 + TX + R <= c.nx;
  const bool iny = !twoD || (y0 - Ry >= 0 && y0 + TY + Ry <= c.ny);
  bool any = false;
  if (inx && iny && ncols <= 64 && nrows <= 32) {
    bool mine = false;
    if (lane < nrows)
      mine = bits_any(kbits, (int64_t)(twoD ? y0 - Ry + lane : 0) * c.nx + (x0 - R), ncols);
    any = __any_sync(0xffffffffu, mine);
  } else {
    const int cells = nrows * ncols;
    for (int e0 = 0; e0 < cells && !any; e0 += 32) {
      bool mine = false;
      const int e = e0 + lane;
      if (e < cells) {
        const int j = y0 - Ry + e / ncols, i = x0 - R + e % ncols;
        int jj = 0, ii = i;
        bool ok = true;
        if (twoD) {
          jj = j;
          if (pery)
            jj = imod(j, c.ny);
          else if (j < 0 || j >= c.ny)
            ok = false;
        }
        if (perx)
          ii = imod(i, c.nx);
        else if (i < 0 || i >= c.nx)
          ok = false;
        mine = ok && bit_get(kbits, (int64_t)jj * c.nx + ii);
      }
      any = __any_sync(0xffffffffu, mine);
    }
  }
  return any;
}

// After a pass: q = g on its kept cells (the pass's tiles), and, when another
// pass follows and the gate has not stopped, the tiles for it: those within
// R = n + 1 cells of a kept cell.  After the first pass of an order every
// tile is a candidate; after a sparse pass only the pass's tiles and their
// eight neighbours can be (R is below the tile size and kept cells lie in
// the pass's tiles), each claimed once through a per-tile stamp (the pass
// stamp ctl[4]).
template <typename T>
__global__ void k_filter_apply_next(DevCfg c, const FiltArgs<T>* __restrict__ fa,
                                    const T* __restrict__ gbuf, const uint32_t* __restrict__ kbits,
                                    int TX, int TY, const int* __restrict__ tiles,
                                    const int* __restrict__ ntiles_dev, int ntiles_all, int R,
                                    int* __restrict__ nxt, int* __restrict__ nxt_n,
                                    int* __restrict__ tstamp, const int* __restrict__ ctl,
                                    int next) {
  const int tiles_x = (c.nx + TX - 1) / TX, tiles_y = (c.ny + TY - 1) / TY;
  const int ntiles = tiles ? *ntiles_dev : ntiles_all;
  T* __restrict__ q = fa->q;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int tile = tiles ? tiles[it] : it;
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    for (int idx = threadIdx.x; idx < TX * TY; idx += blockDim.x) {
      const int gi = x0 + idx % TX, gj = y0 + idx / TX;
      if (gi >= c.nx || gj >= c.ny) continue;
      const int64_t cell = (int64_t)gj * c.nx + gi;
      if (!bit_get(kbits, cell)) continue;
      for (int v = 0; v < c.nvar; ++v) q[v * c.nc + cell] = gbuf[v * c.nc + cell];
    }
  }
  if (!next || ctl[0]) return;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (!tiles) {
    for (int t = w0; t < ntiles_all; t += warps)
      if (tile_near_kept(c, kbits, TX, TY, R, t) && lane == 0) nxt[atomicAdd(nxt_n, 1)] = t;
    return;
  }
  const int stamp = ctl[4];
  const bool twoD = c.ny > 1;
  const bool perx = c.bc[0] == HYROM_BC_PERIODIC, pery = c.bc[2] == HYROM_BC_PERIODIC;
  const int nb = twoD ? 9 : 3;
  for (int k = w0; k < ntiles * nb; k += warps) {
    const int tile = tiles[k / nb], d = k % nb;
    const int dx = twoD ? d % 3 - 1 : d - 1, dy = twoD ? d / 3 - 1 : 0;
    int txi = tile % tiles_x + dx, tyi = tile / tiles_x + dy;
    if (txi < 0 || txi >= tiles_x) {
      if (!perx) continue;
      txi = imod(txi, tiles_x);
    }
    if (tyi < 0 || tyi >= tiles_y) {
      if (!pery) continue;
      tyi = imod(tyi, tiles_y);
    }
    const int t = tyi * tiles_x + txi;
    int first = 0;
    if (lane == 0) first = atomicExch(&tstamp[t], stamp) != stamp;
    if (!__shfl_sync(0xffffffffu, first, 0)) continue;  // claimed by another warp
    if (tile_near_kept(c, kbits, TX, TY, R, t) && lane == 0) nxt[atomicAdd(nxt_n, 1)] = t;
  }
}

template <typename T>
void launch_filter_sparse(const DevCfg& c, const int* orders, int norders, int jmax_f,
                          double eps_f, T* q, const T* qp, int64_t k, T* gbuf, uint32_t* kbits,
                          int* tiles_a, int* tiles_b, int* counts, double* part, int* ctl,
                          void* fargs, GraphSlot* graph, cudaStream_t s, uint32_t* tape_keeps,
                          int* tape_orders, int* tape_count) {
  const bool twoD = c.ny > 1;
  const int TX = twoD ? 32 : 256, TY = twoD ? 8 : 1;
  const int nt = ((c.nx + TX - 1) / TX) * ((c.ny + TY - 1) / TY);
  const int64_t nwords = (c.nc + 31) / 32;
  FiltArgs<T>* fa = reinterpret_cast<FiltArgs<T>*>(fargs);
  int* tstamp = tiles_b + nt;  // per-tile claim stamps (the buffer holds 2 nt)
  // shared-memory limits of the pass kernels, set outside any capture
  for (int o = 0; o < norders; ++o) {
    const int n = orders[o];
#define HY_FA(NV, NN, TXX, TYY)                                                              \
  do {                                                                                       \
    constexpr size_t sm_ = filter_pass_smem<T, NV, NN, TXX, TYY>();                          \
    smem_at_least((const void*)k_filter_pass<T, NV, NN, TXX, TYY>, sm_);                    \
  } while (0)
#define HY_FA_N(NV, TXX, TYY) \
  do {                        \
    if (n == 1)               \
      HY_FA(NV, 1, TXX, TYY); \
    else if (n == 2)          \
      HY_FA(NV, 2, TXX, TYY); \
    else                      \
      HY_FA(NV, 3, TXX, TYY); \
  } while (0)
    if (c.nvar == 4) {
      if (twoD) HY_FA_N(4, 32, 8); else HY_FA_N(4, 256, 1);
    } else {
      if (twoD) HY_FA_N(1, 32, 8); else HY_FA_N(1, 256, 1);
    }
#undef HY_FA_N
#undef HY_FA
  }
  k_set_filt_args<T><<<1, 1, 0, HY_S(s)>>>(fa, q, qp, (double)k * c.dt, tape_keeps, tape_orders,
                                          tape_count);
  auto body = [&]() {
  cudaMemsetAsync(ctl, 0, 3 * sizeof(int), s);
  for (int o = 0; o < norders; ++o) {
    const int n = orders[o];
    k_set_int<<<1, 1, 0, HY_S(s)>>>(ctl, 0);
    int* cur = nullptr;  // first pass: all tiles
    int* nxt = tiles_a;
    int* cur_n = counts;
    int* nxt_n = counts + 1;
    for (int pass = 0; pass < jmax_f; ++pass) {
      cudaMemsetAsync(kbits, 0, nwords * sizeof(uint32_t), s);
      // one wave: three CTAs per SM (the kernel's register and shared
      // memory bounds), tiles taken grid-stride
      const int grid = cur ? 152 * 3 : (nt < 152 * 3 ? nt : 152 * 3);
#define HY_FP(NV, NN, TXX, TYY)                                                              \
  do {                                                                                       \
    constexpr size_t sm_ = filter_pass_smem<T, NV, NN, TXX, TYY>();                          \
    k_filter_pass<T, NV, NN, TXX, TYY><<<grid, 256, sm_, HY_S(s)>>>(                         \
        c, fa, gbuf, kbits, cur, cur_n, nt, part, ctl, eps_f);                               \
  } while (0)
#define HY_FP_N(NV, TXX, TYY) \
  do {                        \
    if (n == 1)               \
      HY_FP(NV, 1, TXX, TYY); \
    else if (n == 2)          \
      HY_FP(NV, 2, TXX, TYY); \
    else                      \
      HY_FP(NV, 3, TXX, TYY); \
  } while (0)
      if (c.nvar == 4) {
        if (twoD) HY_FP_N(4, 32, 8); else HY_FP_N(4, 256, 1);
      } else {
        if (twoD) HY_FP_N(1, 32, 8); else HY_FP_N(1, 256, 1);
      }
#undef HY_FP_N
#undef HY_FP
      const bool more = pass + 1 < jmax_f;
      if (more) cudaMemsetAsync(nxt_n, 0, sizeof(int), s);
      if (tape_keeps) {  // recording (direct launches only: not in the captured graph)
        k_tape_pass<T><<<1, 256, 0, HY_S(s)>>>(fa, kbits, nwords, n, ctl);
        k_tape_commit<T><<<1, 1, 0, HY_S(s)>>>(fa, ctl);
      }
      k_filter_apply_next<T><<<152 * 8, 256, 0, HY_S(s)>>>(c, fa, gbuf, kbits, TX, TY, cur, cur_n,
                                                           nt, n + 1, nxt, nxt_n, tstamp, ctl,
                                                           more ? 1 : 0);
      if (more) {
        cur = nxt;
        nxt = (nxt == tiles_a) ? tiles_b : tiles_a;
        int* tn = cur_n;
        cur_n = nxt_n;
        nxt_n = tn;
      }
    }
  }
  };
  if (graph && !tape_keeps)
    run_graphed(graph, s, body);
  else
    body();
}

}  // namespace hy
