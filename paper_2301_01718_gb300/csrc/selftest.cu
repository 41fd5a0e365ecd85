// Diagnostics: the library's own FP64 reciprocal and reciprocal square root
// (common.cuh) on caller arrays, for tests against CUDA's division and sqrt.
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

}  // namespace

extern "C" hyrom_status hyrom_selftest_math(int32_t which, const double* x, double* y, int64_t n,
                                            void* stream) {
  if (!x || !y || n < 0 || (which != 0 && which != 1)) return HYROM_EINVAL;
  if (n == 0) return HYROM_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_selftest_math<<<(int)blocks, 256, 0, HY_S((cudaStream_t)stream)>>>(which, x, y, n);
  return cudaGetLastError() == cudaSuccess ? HYROM_OK : HYROM_ECUDA;
}
