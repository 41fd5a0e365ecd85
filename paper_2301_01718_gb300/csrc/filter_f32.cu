// Residual-gated explicit Shapiro filters for FP32 states (Sec. 2.3.4),
// the kernels of filter_impl.cuh compiled with contraction and approximate
// division and square root (see the build flags).
#include "filter_impl.cuh"

namespace hy {

template void launch_filter_sparse<float>(const DevCfg&, const int*, int, int, double, float*,
                                          const float*, int64_t, float*, uint32_t*, int*, int*,
                                          int*, double*, int*, void*, GraphSlot*, cudaStream_t,
                                          uint32_t*, int*, int*);

}  // namespace hy
