// Physics device functions shared by the HDM and filter kernels: boundary
// (ghost) values, the Godunov (Burgers) and Rusanov (Euler) fluxes and the
// semi-discrete operator f* at one cell (Sec. 2.2 and 3.1 of the paper).
// Every expression has one fixed evaluation order (see common.cuh).
#pragma once
#include <math.h>

#include "common.cuh"

namespace hy {

// ---------------------------------------------------------------------------
// boundary values
// ---------------------------------------------------------------------------

template <typename T>
HY_DEV void shock_state(const DevCfg& c, int gi, int gj, double t, T* out) {
  const double x = ((double)gi + 0.5) * c.dx;
  const double y = ((double)gj + 0.5) * c.dy;
  const double proj = c.sn0 * x + c.sn1 * y;
  const double front = c.sd0 + c.sspeed * t;
  const bool post = proj < front;
  for (int v = 0; v < 4; ++v) out[v] = (T)(post ? c.post[v] : c.pre[v]);
}

// State at grid position (gi, gj), which may lie one layer outside the
// domain: periodic sides wrap, outflow sides repeat the boundary cell, shock
// sides take the exact planar-shock state at time t.  Positions outside on
// both axes (corners) are never read by the 5-point stencils; they are
// clamped.
template <typename T, int NV>
HY_DEV void fetch(const DevCfg& c, const T* __restrict__ q, int gi, int gj, double t, T* out) {
  const bool twoD = c.ny > 1;
  if (!twoD) gj = 0;
  bool outx = false, outy = false;
  int side = -1;
  if (gi < 0 || gi >= c.nx) {
    if (c.bc[0] == HYROM_BC_PERIODIC) {
      gi = imod(gi, c.nx);
    } else {
      side = gi < 0 ? 0 : 1;
      outx = true;
    }
  }
  if (twoD && (gj < 0 || gj >= c.ny)) {
    if (c.bc[2] == HYROM_BC_PERIODIC) {
      gj = imod(gj, c.ny);
    } else {
      if (!outx) side = gj < 0 ? 2 : 3;
      outy = true;
    }
  }
  if ((outx || outy) && !(outx && outy) && c.bc[side] == HYROM_BC_SHOCK) {
    T s[4];
    shock_state<T>(c, gi, gj, t, s);
    for (int v = 0; v < NV; ++v) out[v] = s[v];
    return;
  }
  gi = gi < 0 ? 0 : (gi >= c.nx ? c.nx - 1 : gi);
  gj = gj < 0 ? 0 : (gj >= c.ny ? c.ny - 1 : gj);
  const int64_t cell = (int64_t)gj * c.nx + gi;
  for (int v = 0; v < NV; ++v) out[v] = q[v * c.nc + cell];
}

// ---------------------------------------------------------------------------
// fluxes (fixed evaluation order; see common.cuh)
// ---------------------------------------------------------------------------

template <typename T>
HY_DEV T godunov(T uL, T uR) {
  const T a = uL > (T)0 ? uL : (T)0;
  const T b = uR < (T)0 ? uR : (T)0;
  const T fa = (T)0.5 * a * a;
  const T fb = (T)0.5 * b * b;
  return fa > fb ? fa : fb;
}

template <typename T>
HY_DEV void prims(const T* q, T g, T& u, T& v, T& p, T& cs) {
  u = q[1] / q[0];
  v = q[2] / q[0];
  p = (g - (T)1) * (q[3] - (T)0.5 * q[0] * (u * u + v * v));
  const T a2 = g * p / q[0];
  cs = sqrt(a2 > (T)0 ? a2 : (T)0);
}

// Rusanov flux across a face normal to x (AX = 0) or y (AX = 1) from the
// two states and their primitive values w = (u, v, p, c) (prims()); a
// kernel that holds each cell's primitives evaluates each face once.
template <typename T, int AX>
HY_DEV void rusanov_p(const T* qL, const T* wL, const T* qR, const T* wR, T* F) {
  const T uL = wL[0], vL = wL[1], pL = wL[2], cL = wL[3];
  const T uR = wR[0], vR = wR[1], pR = wR[2], cR = wR[3];
  T fL[4], fR[4], a;
  if (AX == 0) {
    fL[0] = qL[1];
    fL[1] = qL[1] * uL + pL;
    fL[2] = qL[2] * uL;
    fL[3] = (qL[3] + pL) * uL;
    fR[0] = qR[1];
    fR[1] = qR[1] * uR + pR;
    fR[2] = qR[2] * uR;
    fR[3] = (qR[3] + pR) * uR;
    const T sl = fabs(uL) + cL, sr = fabs(uR) + cR;
    a = sl > sr ? sl : sr;
  } else {
    fL[0] = qL[2];
    fL[1] = qL[1] * vL;
    fL[2] = qL[2] * vL + pL;
    fL[3] = (qL[3] + pL) * vL;
    fR[0] = qR[2];
    fR[1] = qR[1] * vR;
    fR[2] = qR[2] * vR + pR;
    fR[3] = (qR[3] + pR) * vR;
    const T sl = fabs(vL) + cL, sr = fabs(vR) + cR;
    a = sl > sr ? sl : sr;
  }
  const T ha = (T)0.5 * a;
  for (int v = 0; v < 4; ++v) F[v] = (T)0.5 * (fL[v] + fR[v]) - ha * (qR[v] - qL[v]);
}

template <typename T, int AX>
HY_DEV void rusanov(const T* qL, const T* qR, T g, T* F) {
  T wL[4], wR[4];
  prims(qL, g, wL[0], wL[1], wL[2], wL[3]);
  prims(qR, g, wR[0], wR[1], wR[2], wR[3]);
  rusanov_p<T, AX>(qL, wL, qR, wR, F);
}

// f*(q) at one cell from its 5-point neighbourhood.
template <typename T, int NV>
HY_DEV void rhs_cell(const DevCfg& c, const T* qC, const T* qW, const T* qE, const T* qS,
                     const T* qN, T* out) {
  const T dx = (T)c.dx, dy = (T)c.dy;
  if (NV == 1) {
    const T Fl = godunov<T>(qW[0], qC[0]);
    const T Fr = godunov<T>(qC[0], qE[0]);
    out[0] = -(Fr - Fl) / dx;
  } else {
    const T g = (T)c.gamma;
    T Fl[4], Fr[4];
    rusanov<T, 0>(qW, qC, g, Fl);
    rusanov<T, 0>(qC, qE, g, Fr);
    for (int v = 0; v < 4; ++v) out[v] = -(Fr[v] - Fl[v]) / dx;
    if (c.ny > 1) {
      T Gb[4], Gt[4];
      rusanov<T, 1>(qS, qC, g, Gb);
      rusanov<T, 1>(qC, qN, g, Gt);
      for (int v = 0; v < 4; ++v) out[v] = out[v] - (Gt[v] - Gb[v]) / dy;
    }
  }
}

}  // namespace hy
