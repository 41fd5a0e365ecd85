// Diagnostics: the library's own FP64 reciprocal and reciprocal square root
// (common.cuh) on caller arrays, for tests against CUDA's division and sqrt;
// and a dense FP64 FMA loop whose timing gives this GPU's FP64 rate, the
// denominator of the FP64 stages' roofline.
#include <cuda_runtime.h>

#include "../../include/hyrom.h"
#include "common.cuh"

namespace {

__global__ void k_selftest_math(int which, const double* __restrict__ x, double* __restrict__ y,
                                int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = which == 0 ? hy::rcp64(x[i]) : hy::rsqrt64(x[i]);
}

// 8 independent FMA chains per thread, `iters` rounds: 16 * iters FP64
// flops per thread; the sum is stored so that nothing is dead code.
__global__ void k_fp64_rate(double* __restrict__ out, int iters, double a) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (double)(threadIdx.x + j) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, 0.5);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" hyrom_status hyrom_probe_fp64(double* out, int32_t blocks, int32_t iters,
                                         void* stream) {
  if (!out || blocks < 1 || iters < 1) return HYROM_EINVAL;
  k_fp64_rate<<<blocks, 256, 0, HY_S((cudaStream_t)stream)>>>(out, iters, 0.999999);
  return cudaGetLastError() == cudaSuccess ? HYROM_OK : HYROM_ECUDA;
}

extern "C" hyrom_status hyrom_selftest_math(int32_t which, const double* x, double* y, int64_t n,
                                            void* stream) {
  if (!x || !y || n < 0 || (which != 0 && which != 1)) return HYROM_EINVAL;
  if (n == 0) return HYROM_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_selftest_math<<<(int)blocks, 256, 0, HY_S((cudaStream_t)stream)>>>(which, x, y, n);
  return cudaGetLastError() == cudaSuccess ? HYROM_OK : HYROM_ECUDA;
}
