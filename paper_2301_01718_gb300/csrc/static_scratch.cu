// Gappy reduced coordinates without any device allocation.
//
// hyrom_stage_gappy (and the context it needs) allocate device memory.  Some
// callers cannot: a host application that budgets all device memory up front
// and hands the library only pointers into its own pools, a plugin that must
// not use the CUDA allocator of the program that loads it, or a time-critical
// loop where cudaMalloc / cudaFree would add an implicit device
// synchronisation.  This entry point computes the same
// y = (P^T Phi)^+ P^T (v - psi) with the same two kernels, but keeps its
// scratch (the m x n_p pseudo-inverse and the QR's rank-deficiency counter)
// in file-scope device arrays that exist once per GPU for the lifetime of the
// process.  The paper has no counterpart: this is a property of the library,
// not of the method.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/hyrom.h"
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int kStaticMaxM = 64;
constexpr int kStaticMaxNp = 128;

// m x n_p FP64 pseudo-inverse (64 x 128 doubles = 64 KB) and the counter the
// QR kernel increments when a pivot of R is numerically zero (P^T Phi
// rank-deficient); the second kernel then writes NaN into every y_j.
__device__ __align__(256) double g_pinv_scratch[kStaticMaxM * kStaticMaxNp];
__device__ __align__(256) int g_status_scratch[64];

struct DeviceScratch {
  double* pinv = nullptr;
  int* status = nullptr;
  bool ready = false;
};

constexpr int kMaxDevices = 64;
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

hyrom_status fail(char* err, int32_t err_len, hyrom_status s, const char* msg) {
  if (err && err_len > 0) snprintf(err, (size_t)err_len, "hyrom_gappy_static: %s", msg);
  return s;
}

// Device addresses of the scratch arrays on the current device.  In host
// code the array names are only stand-ins; kernels need the addresses that
// cudaGetSymbolAddress returns, looked up once per device with that device
// current and kept for later calls.
hyrom_status scratch_for_current_device(DeviceScratch** out, char* err, int32_t err_len) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(err, err_len, HYROM_ECUDA, "cudaGetDevice failed");
  }
  if (dev < 0 || dev >= kMaxDevices)
    return fail(err, err_len, HYROM_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  DeviceScratch& d = g_scratch[dev];
  if (!d.ready) {
    void* p = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pinv_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_status_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      char buf[160];
      snprintf(buf, sizeof buf, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return fail(err, err_len, HYROM_ECUDA, buf);
    }
    d.pinv = (double*)p;
    d.status = (int*)q;
    d.ready = true;
  }
  *out = &d;
  return HYROM_OK;
}

}  // namespace

extern "C" hyrom_status hyrom_gappy_static(const void* phi, int64_t ndof, int32_t m,
                                           const int32_t* points, int32_t n_p, const void* v,
                                           const void* psi, int32_t precision, double* y_out,
                                           void* stream, char* err, int32_t err_len) {
  if (err && err_len > 0) err[0] = '\0';
  if (!phi || !points || !v || !psi || !y_out || ndof <= 0)
    return fail(err, err_len, HYROM_EINVAL, "null pointer or empty state");
  if (precision != HYROM_PREC_F64 && precision != HYROM_PREC_F32)
    return fail(err, err_len, HYROM_EINVAL, "precision must be HYROM_PREC_F64 or HYROM_PREC_F32");
  if (m < 1 || m > kStaticMaxM || n_p < m || n_p > kStaticMaxNp || n_p > ndof) {
    char buf[160];
    snprintf(buf, sizeof buf,
             "needs 1 <= m <= %d and m <= n_p <= min(%d, ndof) (got m = %d, n_p = %d, ndof = %lld)",
             kStaticMaxM, kStaticMaxNp, m, n_p, (long long)ndof);
    return fail(err, err_len, HYROM_EINVAL, buf);
  }
  DeviceScratch* d = nullptr;
  hyrom_status st = scratch_for_current_device(&d, err, err_len);
  if (st != HYROM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // The counter must be zero when the QR starts; the pseudo-inverse needs no
  // clearing (the QR kernel writes all m x n_p entries before they are read).
  if (cudaMemsetAsync(d->status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return fail(err, err_len, HYROM_ECUDA, "clearing the rank-deficiency counter failed");
  }
  if (precision == HYROM_PREC_F32) {
    hy::launch_gappy_pinv<float>((const float*)phi, ndof, m, points, n_p, d->pinv, d->status, s);
    hy::launch_gappy_apply<float>(d->pinv, m, n_p, points, (const float*)v, (const float*)psi,
                                  y_out, nullptr, nullptr, s, d->status);
  } else {
    hy::launch_gappy_pinv<double>((const double*)phi, ndof, m, points, n_p, d->pinv, d->status,
                                  s);
    hy::launch_gappy_apply<double>(d->pinv, m, n_p, points, (const double*)v, (const double*)psi,
                                   y_out, nullptr, nullptr, s, d->status);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char buf[160];
    snprintf(buf, sizeof buf, "kernel launch failed: %s", cudaGetErrorString(e));
    return fail(err, err_len, HYROM_ECUDA, buf);
  }
  return HYROM_OK;
}
