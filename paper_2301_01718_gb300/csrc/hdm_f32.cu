// The full SSP-RK2 step of the 2D Euler equations (Sec. 2.2, the explicit
// scheme; Sec. 3.1, ideal gas with the Rusanov flux) for FP32 states, built
// to stream the state once from HBM: read gamma_{k-1} once, write gamma_k
// once, everything else in registers.
//
// Work layout: one warp owns a strip of 64 columns x H rows of the grid and
// sweeps it upwards one row per iteration.  Lane l holds the column pair
// (x0 - 2 + 2l, x0 - 1 + 2l) as the two halves of packed FP32 pairs, so
// every arithmetic instruction works on two cells (Blackwell's packed f32x2
// add, mul and fma).  Lanes 0 and 31 are the two-cell halo in x, so a strip
// writes 60 columns; the sweep starts two rows below and ends two rows above
// its H output rows.  At the iteration that loads row r, the warp
//   * forms the primitives, the physical fluxes and wave speeds of row r,
//   * takes the Rusanov fluxes of the two x faces left of and between its
//     columns (the left neighbour's second column comes by a warp shuffle)
//     and the y-face flux between rows r-1 and r from the registers that
//     hold row r-1,
//   * finishes stage 1 (q* = q + dt f*(q)) on row r-1,
//   * does the same for the stage-1 state and finishes stage 2
//     (q = q/2 + (q* + dt f*(q*))/2) on row r-2, which it stores.
// Only two rows of each stage live in registers, so the kernel holds no
// shared memory and no tile halo is re-read from HBM (the halo columns come
// from L2 for the neighbouring strip).  Rows are loaded two iterations ahead.
//
// Arithmetic: FP32 with fused multiply-adds (this file is compiled with
// contraction on), 1/rho from the approximate reciprocal and one Newton step,
// the sound speed from the approximate square root; the difference of two
// face fluxes (each formed without its factor 1/2) is multiplied by
// dt/(2 dx) (dt/(2 dy)) once.  Results differ from the
// correctly rounded FP64-order expressions of hdm.cu by a few FP32 ulps,
// within the FP32 path's 1e-5 tolerance; FP64 states keep the bit-exact
// kernel.
//
// Boundaries follow fetch() in phys.cuh: periodic sides wrap, outflow sides
// repeat the boundary cell, shock sides take the exact planar-shock state,
// the stage-1 state at t_k.  The shock's side of a ghost cell is decided in
// FP32 where the cell is clearly on one side and in FP64 near the front, so
// the decision is the FP64 one of the other paths.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace hy {
namespace {

constexpr int kStripW = 60;  // output columns per warp
constexpr int kWarps = 4;    // warps per block
// launch shape: blocks per SM the register budget is cut for, row-loop
// unrolling, strips per resident warp slot (waves) and the least strip height
#ifndef HY_SWEEP_MINB
#define HY_SWEEP_MINB 4
#endif
#ifndef HY_SWEEP_UNROLL
#define HY_SWEEP_UNROLL 2
#endif
#ifndef HY_SWEEP_WAVES
#define HY_SWEEP_WAVES 2
#endif
#ifndef HY_SWEEP_MINH
#define HY_SWEEP_MINH 16
#endif
constexpr int kUnroll = HY_SWEEP_UNROLL;

// ---- packed FP32 pairs (f32x2 instructions, one issue slot per pair; the
// PTX forms kept the FP64 pipe idle where the float2 intrinsics did not)
HY_DEV unsigned long long pk(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
HY_DEV float2 upk(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
HY_DEV float2 add2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
HY_DEV float2 sub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
HY_DEV float2 mul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
HY_DEV float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
  return upk(d);
}
HY_DEV float2 splat(float a) { return make_float2(a, a); }

HY_DEV float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
HY_DEV float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// physical fluxes f_x, f_y and wave speeds |u| + c, |v| + c of two states
struct Flux2 {
  float2 fx[4], fy[4], sx, sy;
};

HY_DEV void cell_flux2(const float2* q, float g, Flux2& o) {
  float2 r = make_float2(rcp_approx(q[0].x), rcp_approx(q[0].y));
  const float2 e = fma2(make_float2(-q[0].x, -q[0].y), r, splat(1.0f));  // one Newton step
  r = fma2(r, e, r);
  const float2 u = mul2(q[1], r), v = mul2(q[2], r);
  const float2 ke = fma2(q[2], v, mul2(q[1], u));                       // rho |u|^2
  const float2 p = mul2(splat(g - 1.0f), fma2(splat(-0.5f), ke, q[3]));
  const float2 a2 = mul2(mul2(splat(g), p), r);
  const float2 c = make_float2(sqrt_approx(fmaxf(a2.x, 0.0f)), sqrt_approx(fmaxf(a2.y, 0.0f)));
  const float2 ep = add2(q[3], p);
  o.fx[0] = q[1];
  o.fx[1] = fma2(q[1], u, p);
  o.fx[2] = mul2(q[2], u);
  o.fx[3] = mul2(ep, u);
  o.fy[0] = q[2];
  o.fy[1] = mul2(q[1], v);
  o.fy[2] = fma2(q[2], v, p);
  o.fy[3] = mul2(ep, v);
  o.sx = make_float2(fabsf(u.x) + c.x, fabsf(u.y) + c.y);
  o.sy = make_float2(fabsf(v.x) + c.x, fabsf(v.y) + c.y);
}

// Twice the Rusanov flux of two faces at once: 2F = fL + fR - max(sL, sR)
// (qR - qL); the factor 1/2 is applied with dt/dx (dt/dy) by the callers.
HY_DEV void rusanov2(const float2* qL, const float2* fL, float2 sL, const float2* qR,
                     const float2* fR, float2 sR, float2* F) {
  const float2 na = make_float2(-fmaxf(sL.x, sR.x), -fmaxf(sL.y, sR.y));
#pragma unroll
  for (int v = 0; v < 4; ++v) F[v] = fma2(na, sub2(qR[v], qL[v]), add2(fL[v], fR[v]));
}

HY_DEV float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
HY_DEV float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// x divergence 2F(right face) - 2F(left face) of both columns of a lane: the
// faces left of the first column and between the two columns are formed
// here (the left lane's second column comes by shuffles), the face right of
// the second column is the next lane's first face
HY_DEV void xdiv2(const float2* q, const Flux2& f, float2* div) {
  float2 qL[4], fL[4], F[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    qL[v] = make_float2(shfl_up1(q[v].y), q[v].x);
    fL[v] = make_float2(shfl_up1(f.fx[v].y), f.fx[v].x);
  }
  const float2 sL = make_float2(shfl_up1(f.sx.y), f.sx.x);
  rusanov2(qL, fL, sL, q, f.fx, f.sx, F);  // (left face, middle face)
#pragma unroll
  for (int v = 0; v < 4; ++v) div[v] = sub2(make_float2(F[v].y, shfl_dn1(F[v].x)), F[v]);
}

// Everything the kernel reads about the grid, in the form it uses: FP32
// constants (passed as a kernel parameter, so no conversion runs on the
// device) and the FP64 shock geometry for decisions near the front.
struct SweepCfg {
  int nx, ny, bc[4];
  int64_t nc;
  float g, nlx, nly;                         // gamma, -dt/(2 dx), -dt/(2 dy)
  float dx, dy, sn0, sn1, sd0, ssp, t0, t1;  // shock geometry and times
  float pre[4], post[4];
  double dxd, dyd, sn0d, sn1d, sd0d, sspd, t0d, t1d;
};

// exact planar-shock state at cell (gi, gj) at t0 (stage = 0) or t1: FP32
// where the cell is clearly on one side of the front, FP64 near it
HY_DEV void shock_f(const SweepCfg& c, int gi, int gj, int stage, float* out) {
  const float x = ((float)gi + 0.5f) * c.dx, y = ((float)gj + 0.5f) * c.dy;
  const float pr = c.sn0 * x + c.sn1 * y;
  const float fr = c.sd0 + c.ssp * (stage ? c.t1 : c.t0);
  bool post = pr < fr;
  if (fabsf(pr - fr) <= 1e-5f * (fabsf(pr) + fabsf(fr)) + 1e-6f) {
    const double xd = ((double)gi + 0.5) * c.dxd, yd = ((double)gj + 0.5) * c.dyd;
    post = c.sn0d * xd + c.sn1d * yd < c.sd0d + c.sspd * (stage ? c.t1d : c.t0d);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = post ? c.post[v] : c.pre[v];
}

// gamma_{k-1} at (gi, gj), as fetch() gives it at t0
HY_DEV void load_q1(const SweepCfg& c, const float* __restrict__ q, int gi, int gj, bool perx,
                    bool pery, float* out) {
  const bool outx = (gi < 0 || gi >= c.nx) && !perx;
  const bool outy = (gj < 0 || gj >= c.ny) && !pery;
  if (outx != outy) {
    const int side = outx ? (gi < 0 ? 0 : 1) : (gj < 0 ? 2 : 3);
    if (c.bc[side] == HYROM_BC_SHOCK) {
      shock_f(c, gi, gj, 0, out);
      return;
    }
  }
  if (perx) gi = imod(gi, c.nx);
  if (pery) gj = imod(gj, c.ny);
  gi = gi < 0 ? 0 : (gi >= c.nx ? c.nx - 1 : gi);
  gj = gj < 0 ? 0 : (gj >= c.ny ? c.ny - 1 : gj);
  const int64_t cell = (int64_t)gj * c.nx + gi;
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = __ldg(q + v * c.nc + cell);
}

// row gj of the lane's column pair.  Plain loads where the row (after a
// periodic wrap) and both columns are inside the domain, VEC: one 8-byte load
// per variable (an even nx keeps the pair inside one row); boundary values
// per column elsewhere.
template <bool VEC>
HY_DEV void load_row(const SweepCfg& c, const float* __restrict__ q, int cA, int gj,
                     bool interior, bool perx, bool pery, float2* Q) {
  int gjw = gj;
  bool plain = interior;
  if (!interior) {
    bool rowin = gj >= 0 && gj < c.ny;
    if (!rowin && pery) {
      gjw = imod(gj, c.ny);
      rowin = true;
    }
    plain = rowin && cA >= 0 && cA + 1 < c.nx;
  }
  if (plain) {
    const int64_t cell = (int64_t)gjw * c.nx + cA;
    if (VEC) {
#pragma unroll
      for (int v = 0; v < 4; ++v) Q[v] = __ldg(reinterpret_cast<const float2*>(q + v * c.nc + cell));
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v)
        Q[v] = make_float2(__ldg(q + v * c.nc + cell), __ldg(q + v * c.nc + cell + 1));
    }
  } else {
    float a[4], b[4];
    load_q1(c, q, cA, gj, perx, pery, a);
    load_q1(c, q, cA + 1, gj, perx, pery, b);
#pragma unroll
    for (int v = 0; v < 4; ++v) Q[v] = make_float2(a[v], b[v]);
  }
}

}  // namespace

// One warp's strip: columns x0 - 2 .. x0 + 61, output rows y0 .. y0 + H - 1.
// INTERIOR: every cell the strip touches lies inside the domain (plain loads,
// no boundary values); the boundary code is compiled only into the other
// instance.
template <bool VEC, bool INTERIOR>
HY_DEV void sweep_strip(const SweepCfg& c, const float* __restrict__ q, float* __restrict__ out,
                        int lane, int x0, int y0, int H) {
  constexpr bool interior = INTERIOR;
  const int cA = x0 - 2 + 2 * lane, cB = cA + 1;  // the lane's two columns
  const float g = c.g;
  const float2 nlx = splat(c.nlx), nly = splat(c.nly);
  const bool perx = c.bc[0] == HYROM_BC_PERIODIC, pery = c.bc[2] == HYROM_BC_PERIODIC;
  const bool ghostA = !perx && (cA < 0 || cA >= c.nx);
  const bool ghostB = !perx && (cB < 0 || cB >= c.nx);
  // some lane of the strip holds a ghost column (non-periodic x side)
  const bool any_ghost_x = !interior && __any_sync(0xffffffffu, ghostA || ghostB);
  const bool lane_out = lane >= 1 && lane <= 30;
  const bool wA = lane_out && cA < c.nx, wB = lane_out && cB < c.nx;
  const int yend = min(y0 + H, c.ny);  // last output row + 1
  const int rend = yend + 2;           // rows y0-2 .. yend+1 are loaded

  // Carried between rows (registers): for the y face above, the last row's
  // state, physical y flux and y wave speed, per stage (Qp, fyp, syp and
  // Q1p, fy1p, sy1p); and the partial updates that only wait for that face:
  //   A1 = q + nlx div_x - nly G_below   (stage 1 of the last row: + nly G_above)
  //   A2 = q/2 + (q* + nlx div*_x - nly G*_below)/2   (stage 2 of the row
  //        before it: + nly G*_above / 2)
  // with nlx = -dt/(2 dx), nly = -dt/(2 dy) and G twice the face flux.
  float2 Qp[4], fyp[4], A1[4], Q1p[4], fy1p[4], A2[4];
  float2 syp = splat(1.0f), sy1p = splat(1.0f);
#pragma unroll
  for (int v = 0; v < 4; ++v) Qp[v] = fyp[v] = A1[v] = Q1p[v] = fy1p[v] = A2[v] = splat(1.0f);
  const float2 hly = splat(0.5f * c.nly), mnly = splat(-c.nly);
  float2 Qn[4], Qnn[4];
  load_row<VEC>(c, q, cA, y0 - 2, interior, perx, pery, Qn);
  load_row<VEC>(c, q, cA, y0 - 1, interior, perx, pery, Qnn);
#pragma unroll kUnroll
  for (int gj = y0 - 2; gj < rend; ++gj) {
    float2 Q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      Q[v] = Qn[v];
      Qn[v] = Qnn[v];
    }
    if (gj + 2 < rend) load_row<VEC>(c, q, cA, gj + 2, interior, perx, pery, Qnn);
    // ---- stage 0: fluxes of row gj, x divergence, y face below the row
    Flux2 f;
    cell_flux2(Q, g, f);
    float2 div[4], G[4];
    xdiv2(Q, f, div);
    rusanov2(Qp, fyp, syp, Q, f.fy, f.sy, G);  // face between rows gj-1 and gj
    const int r1 = gj - 1;                      // stage-1 row
    if (r1 >= y0 - 1) {
      float2 Q1[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) Q1[v] = fma2(nly, G[v], A1[v]);
      bool bottom_outflow = false;
      if (!interior) {
        // stage-1 boundary values at t_k on non-periodic sides
        const bool outy = !pery && (r1 < 0 || r1 >= c.ny);  // the same on every lane
        if (outy) {
          const int side = r1 < 0 ? 2 : 3;
          if (c.bc[side] == HYROM_BC_SHOCK) {
            float a[4], b[4];
            shock_f(c, cA, r1, 1, a);
            shock_f(c, cB, r1, 1, b);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              if (!ghostA) Q1[v].x = a[v];
              if (!ghostB) Q1[v].y = b[v];
            }
          } else if (r1 >= c.ny) {  // outflow top: repeat row ny-1 (held in Q1p)
#pragma unroll
            for (int v = 0; v < 4; ++v) Q1[v] = Q1p[v];
          }
          // outflow bottom: row -1 takes row 0's values when row 0 is formed
        } else if (any_ghost_x) {
          float fromR[4], fromL[4], ownA[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            fromR[v] = shfl_dn1(Q1[v].x);  // the right lane's first column
            fromL[v] = shfl_up1(Q1[v].y);  // the left lane's second column
            ownA[v] = Q1[v].x;
          }
          if (ghostA) {
            if (c.bc[cA < 0 ? 0 : 1] == HYROM_BC_SHOCK) {
              float a[4];
              shock_f(c, cA, r1, 1, a);
#pragma unroll
              for (int v = 0; v < 4; ++v) Q1[v].x = a[v];
            } else {  // outflow: the next column inwards
#pragma unroll
              for (int v = 0; v < 4; ++v) Q1[v].x = cA < 0 ? Q1[v].y : fromL[v];
            }
          }
          if (ghostB) {
            if (c.bc[cB < 0 ? 0 : 1] == HYROM_BC_SHOCK) {
              float b[4];
              shock_f(c, cB, r1, 1, b);
#pragma unroll
              for (int v = 0; v < 4; ++v) Q1[v].y = b[v];
            } else {
#pragma unroll
              for (int v = 0; v < 4; ++v) Q1[v].y = cB < 0 ? fromR[v] : ownA[v];
            }
          }
        }
        bottom_outflow = !outy && r1 == 0 && !pery && c.bc[2] == HYROM_BC_OUTFLOW;
      }
      // ---- stage-1 state of row r1: fluxes, x divergence, y face below
      Flux2 f1;
      cell_flux2(Q1, g, f1);
      if (bottom_outflow) {  // the ghost row -1 (in Q1p) equals row 0
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          Q1p[v] = Q1[v];
          fy1p[v] = f1.fy[v];
        }
        sy1p = f1.sy;
      }
      float2 div1[4], G1[4];
      xdiv2(Q1, f1, div1);
      rusanov2(Q1p, fy1p, sy1p, Q1, f1.fy, f1.sy, G1);  // face between r1-1 and r1
      const int r2 = r1 - 1;                              // stage-2 row
      if (r2 >= y0 && r2 < yend && (wA || wB)) {
        float2 o[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) o[v] = fma2(hly, G1[v], A2[v]);
        const int64_t cell = (int64_t)r2 * c.nx + cA;
        if (VEC && wA && wB) {
#pragma unroll
          for (int v = 0; v < 4; ++v) *reinterpret_cast<float2*>(out + v * c.nc + cell) = o[v];
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            if (wA) out[v * c.nc + cell] = o[v].x;
            if (wB) out[v * c.nc + cell + 1] = o[v].y;
          }
        }
      }
      // A2 of row r1: q/2 + (q* + nlx div*_x - nly G*_below)/2
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float2 t = fma2(mnly, G1[v], fma2(nlx, div1[v], Q1[v]));
        A2[v] = fma2(splat(0.5f), Qp[v], mul2(splat(0.5f), t));
        Q1p[v] = Q1[v];
        fy1p[v] = f1.fy[v];
      }
      sy1p = f1.sy;
    }
    // A1 of row gj
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      A1[v] = fma2(mnly, G[v], fma2(nlx, div[v], Q[v]));
      Qp[v] = Q[v];
      fyp[v] = f.fy[v];
    }
    syp = f.sy;
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kWarps * 32, HY_SWEEP_MINB)
    k_rk2_euler_sweep(const __grid_constant__ SweepCfg c, const float* __restrict__ q,
                      float* __restrict__ out, int H, int strips_x, int nstrips) {
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (strip >= nstrips) return;  // whole warp leaves together
  // The strips along the domain's sides take the slower general path; they
  // are handed out first (bottom and top rows, then the left and right
  // columns), so that the launch does not end on them.
  const int strips_y = nstrips / strips_x;
  int sxi, syi;
  if (strips_x >= 3 && strips_y >= 3) {
    const int nb = 2 * strips_x + 2 * (strips_y - 2);
    if (strip < 2 * strips_x) {
      sxi = strip % strips_x;
      syi = strip < strips_x ? 0 : strips_y - 1;
    } else if (strip < nb) {
      const int e = strip - 2 * strips_x;
      sxi = e < strips_y - 2 ? 0 : strips_x - 1;
      syi = 1 + (e < strips_y - 2 ? e : e - (strips_y - 2));
    } else {
      const int e = strip - nb;
      sxi = 1 + e % (strips_x - 2);
      syi = 1 + e / (strips_x - 2);
    }
  } else {
    sxi = strip % strips_x;
    syi = strip / strips_x;
  }
  const int x0 = sxi * kStripW, y0 = syi * H;
  if (x0 - 2 >= 0 && x0 + 62 <= c.nx && y0 - 2 >= 0 && y0 + H + 2 <= c.ny)
    sweep_strip<VEC, true>(c, q, out, lane, x0, y0, H);
  else
    sweep_strip<VEC, false>(c, q, out, lane, x0, y0, H);
}

bool rk2_euler_sweep_ok(const DevCfg& c) {
  return c.nvar == 4 && c.ny > 1 && c.nx >= 4 && c.ny >= 4;
}

void launch_rk2_euler_sweep(const DevCfg& c, const float* q, float* out, int64_t k,
                            cudaStream_t s) {
  SweepCfg sc;
  sc.nx = c.nx;
  sc.ny = c.ny;
  for (int i = 0; i < 4; ++i) sc.bc[i] = c.bc[i];
  sc.nc = c.nc;
  sc.g = (float)c.gamma;
  sc.nlx = -(float)(0.5 * c.dt / c.dx);  // the 1/2 of the Rusanov flux
  sc.nly = -(float)(0.5 * c.dt / c.dy);
  sc.t0d = (double)(k - 1) * c.dt;
  sc.t1d = (double)k * c.dt;
  sc.dxd = c.dx;
  sc.dyd = c.dy;
  sc.sn0d = c.sn0;
  sc.sn1d = c.sn1;
  sc.sd0d = c.sd0;
  sc.sspd = c.sspeed;
  sc.dx = (float)c.dx;
  sc.dy = (float)c.dy;
  sc.sn0 = (float)c.sn0;
  sc.sn1 = (float)c.sn1;
  sc.sd0 = (float)c.sd0;
  sc.ssp = (float)c.sspeed;
  sc.t0 = (float)sc.t0d;
  sc.t1 = (float)sc.t1d;
  for (int i = 0; i < 4; ++i) {
    sc.pre[i] = (float)c.pre[i];
    sc.post[i] = (float)c.post[i];
  }
  // rows per strip: as many strips as fit on the GPU at once (one wave),
  // at least 16 rows each
  static int warps_per_sm[2] = {0, 0};
  const bool vec = (c.nx % 2) == 0;
  int& wps = warps_per_sm[vec];
  if (wps == 0) {
    int blocks = 0;
    if (vec)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_rk2_euler_sweep<true>, kWarps * 32, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_rk2_euler_sweep<false>, kWarps * 32, 0);
    wps = blocks > 0 ? blocks * kWarps : kWarps;
  }
  int sms = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int strips_x = (c.nx + kStripW - 1) / kStripW;
  int sy = (HY_SWEEP_WAVES * sms * wps) / strips_x;
  if (sy < 1) sy = 1;
  int H = (c.ny + sy - 1) / sy;
  if (H < HY_SWEEP_MINH) H = HY_SWEEP_MINH;
  const int strips_y = (c.ny + H - 1) / H;
  const int nstrips = strips_x * strips_y;
  const int blocks = (nstrips + kWarps - 1) / kWarps;
  if (vec)
    k_rk2_euler_sweep<true><<<blocks, kWarps * 32, 0, HY_S(s)>>>(sc, q, out, H, strips_x, nstrips);
  else
    k_rk2_euler_sweep<false><<<blocks, kWarps * 32, 0, HY_S(s)>>>(sc, q, out, H, strips_x, nstrips);
}

}  // namespace hy
