// Residual-gated explicit Shapiro filters for FP64 states (Sec. 2.3.4); the
// kernels are in filter_impl.cuh.
#include "filter_impl.cuh"

namespace hy {

template void launch_filter_sparse<double>(const DevCfg&, const int*, int, int, double, double*,
                                           const double*, int64_t, double*, uint32_t*, int*, int*,
                                           int*, double*, int*, void*, GraphSlot*, cudaStream_t,
                                           uint32_t*, int*, int*);

}  // namespace hy
