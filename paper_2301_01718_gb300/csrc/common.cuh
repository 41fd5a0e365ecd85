// Shared device helpers of libhyrom (sm_103a).
//
// Arithmetic convention: the library is compiled with -fmad=false, so every
// a*b+c written in source is a rounded multiply followed by a rounded add,
// exactly as written.  The HDM residual, flux, RK2 and filter expressions
// are written in one fixed order; in FP64 they reproduce, bit for bit, any
// implementation that evaluates the same expressions in the same order
// (IEEE-754 add/mul/div/sqrt are correctly rounded).  Reductions and small
// dense algebra use explicit fma() where speed matters.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hyrom.h"

#define HY_DEV __device__ __forceinline__

namespace hy {

// Kernel-launch counter: every launch passes its stream through HY_S(), a
// comma expression that counts the launch (for the benchmark's report).
void count_launch();
#define HY_S(stream) (::hy::count_launch(), (stream))

constexpr int kMaxVar = 4;

// Everything a kernel needs to know about the grid, PDE and boundaries.
struct DevCfg {
  int pde, scheme, nx, ny, nvar;
  int bc[4];
  double dx, dy, dt, gamma;
  double sn0, sn1, sd0, sspeed;
  double pre[4], post[4];
  int64_t nc, ndof;
};

inline DevCfg make_devcfg(const hyrom_config& c) {
  DevCfg d;
  d.pde = c.pde;
  d.scheme = c.scheme;
  d.nx = c.nx;
  d.ny = c.ny;
  d.nvar = c.pde == HYROM_PDE_BURGERS ? 1 : 4;
  for (int i = 0; i < 4; ++i) d.bc[i] = c.bc[i];
  d.dx = c.dx;
  d.dy = c.dy;
  d.dt = c.dt;
  d.gamma = c.gamma;
  d.sn0 = c.shock_n[0];
  d.sn1 = c.shock_n[1];
  d.sd0 = c.shock_d0;
  d.sspeed = c.shock_speed;
  for (int i = 0; i < 4; ++i) {
    d.pre[i] = c.shock_pre[i];
    d.post[i] = c.shock_post[i];
  }
  d.nc = (int64_t)c.nx * c.ny;
  d.ndof = d.nc * d.nvar;
  return d;
}

HY_DEV bool bit_get(const uint32_t* bm, int64_t c) { return (bm[c >> 5] >> (c & 31)) & 1u; }

HY_DEV int imod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// monotone map of a non-negative double to uint64 (for atomicMax)
HY_DEV unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
HY_DEV double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// Butterfly sum; lane 0's value is broadcast so that every lane holds the
// same bits (lanes would otherwise associate the terms differently).
// order-preserving map of a double to an unsigned 64-bit key (integer
// compares instead of FP64 compares, which run on the narrow FP64 pipe)
HY_DEV unsigned long long dkey(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Copy count values from global src to shared dst, the block's threads each
// issuing up to U loads before their first store (small kernels are
// otherwise bound by one global-memory latency per loop iteration).
template <int U = 8, typename T>
__device__ void stage_copy(T* dst, const T* __restrict__ src, int count) {
  for (int base = threadIdx.x; base < count; base += blockDim.x * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * blockDim.x;
      v[u] = i < count ? src[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * blockDim.x;
      if (i < count) dst[i] = v[u];
    }
  }
}

template <typename T>
HY_DEV T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// 1 / x in FP64 from an FP32 reciprocal seed and two Newton steps
// r <- r + r (1 - x r) (23 -> 46 -> 92 correct bits; within about an ulp),
// which takes 4 FP64 FMAs where an FP64 division takes a longer chain; FP64
// division where x is outside the FP32 normal range.
HY_DEV double rcp64(double x) {
  const float xf = (float)x;
  const float ax = fabsf(xf);
  if (!(ax >= 1.17549435e-38f && ax <= 1.7e38f)) return 1.0 / x;
  double r = (double)__frcp_rn(xf);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 1 / sqrt(a) for a > 0 in FP64 from an FP32 seed and two Newton steps
// y <- y (3/2 - a y^2 / 2) (about an ulp), in place of an FP64 square root
// and division; the FP64 square root and division outside the FP32 range.
HY_DEV double rsqrt64(double a) {
  const float af = (float)a;
  if (!(af >= 1.17549435e-38f && af <= 1.7e38f)) return 1.0 / sqrt(a);
  double y = (double)rsqrtf(af);
  y = y * fma(-0.5 * a * y, y, 1.5);
  y = y * fma(-0.5 * a * y, y, 1.5);
  return y;
}

// Programmatic dependent launch.  A kernel launched with programmatic
// stream serialization may be scheduled while its predecessor on the stream
// still runs; pdl_enter, its first statement, waits until the predecessor has
// completed and its writes are visible (griddepcontrol.wait; a no-op for an
// ordinary launch), then lets the next kernel be scheduled in turn.  Every
// kernel of such a chain therefore starts its work in stream order, only
// without the launch gap.
HY_DEV void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Bucket of a row's squared-norm bound v among 256 (ratio 2^(1/4) per
// bucket, bucket 255 for v = 0): the order ODEIM scans rows in.
constexpr int kNormBuckets = 256;
HY_DEV int nrm_bucket(float v) {
  if (!(v > 0.0f)) return kNormBuckets - 1;
  int b = (int)floorf(24.0f - 4.0f * log2f(v));
  return b < 0 ? 0 : (b > kNormBuckets - 2 ? kNormBuckets - 2 : b);
}

template <typename T>
HY_DEV T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Block-wide sum in a fixed order (deterministic); blockDim.x % 32 == 0,
// <= 1024.  All threads get the result.
template <typename T>
__device__ T block_sum(T v) {
  __shared__ T sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = (T)0;
  if (wid == 0) {
    r = lane < nw ? sh[lane] : (T)0;
    r = warp_sum(r);
    if (lane == 0) sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

template <typename T>
__device__ T block_max(T v) {
  __shared__ T sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T r = lane < nw ? sh[lane] : sh[0];
    r = warp_max(r);
    if (lane == 0) sh[0] = r;
  }
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

}  // namespace hy
