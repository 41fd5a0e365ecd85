// Tensor-core forms of the sample-row normal matrix G = X^T X of the reduced
// solve (Sec. 2.2, reduced coordinates, regression on every dof row of the
// sample cells), X = Phi_S: rows = the dof rows of the sample cells
// (variable-major, as in reduced.cu), columns = the m <= 64 basis modes.
// FP32 states only.
//
// Each 16 KB shared-memory atom is a 128-row, 128-byte K-major operand whose
// K runs over sample rows.  Its 128 rows ("virtual columns" Y) are, by mode:
//   * TF32: X rounded to TF32 (nearest, ties away); rows 0-63 = X on the
//     atom's sample rows [0, 32), rows 64-127 = X on [32, 64);
//   * BF16: X rounded to BF16 (nearest even), 64 sample rows per half;
//   * split TF32: rows 0-63 = hi(X), rows 64-127 = lo(X) on 32 sample rows,
//     hi = x with its 13 low mantissa bits cleared, lo = TF32(x - hi).
// One tcgen05.mma (M = N = 128, A and B both the atom) accumulates Y^T Y in
// tensor memory.  G is the sum of its two diagonal 64 x 64 blocks (TF32,
// BF16: the two halves of the rows), or of all four blocks (split:
// (hi + lo)^T (hi + lo), FP32-level products).  The off-diagonal blocks of
// the two-half forms are products of different rows and are never read;
// keeping M = 128 keeps accumulator row i in tensor-memory lane i.
//
// One CTA per SM takes a contiguous range of sample rows in stages of 128:
//   * warps 1-16 (converters): each lane loads one sample row of 16 basis
//     columns (a warp: 32 consecutive rows of one column per load, coalesced
//     along the sorted cells), rounds, and writes the swizzled atoms;
//   * warp 0 (one thread): the MMAs of each full stage, committed to the
//     stage's empty barrier, and at the end to the accumulator's barrier;
//   * warps 1-4 (epilogue, after converting): tcgen05.ld of the accumulator,
//     block sums, and the CTA's FP64 partial G to part[b * 4096 ...]; the
//     partials are summed in FP64 by the caller.
// Every mbarrier wait is bounded; a timeout sets *err and ends every role's
// loop, and the tensor memory is freed only after the MMAs completed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace hy {
namespace {

using namespace tc;

constexpr int kThreads = 544;      // 17 warps
constexpr int kRowsStage = 128;    // sample rows per stage
constexpr int kColsWarp = 16;      // basis columns per converter warp and stage
constexpr int kAtomBytes = 16384;  // 128 rows x 128 bytes
constexpr int kRingBytes = 196608;
constexpr int kSmemBytes = kRingBytes + 1024;
constexpr uint32_t kTmemCols = 128;

enum { kTf32 = 1, kBf16 = 2, kSplit = 3 };  // the HYROM_RED_* values

template <int MODE>
struct Mode {
  // sample rows per atom, atoms per stage, stages in the ring
  static constexpr int kRowsAtom = MODE == kBf16 ? 128 : (MODE == kTf32 ? 64 : 32);
  static constexpr int kAtoms = kRowsStage / kRowsAtom;
  static constexpr int kStageBytes = kAtoms * kAtomBytes;
  static constexpr int kStages = kRingBytes / kStageBytes;
  // D FP32 (bits 4-5 = 1); A, B formats at bits 7-9, 10-12 (kind::tf32:
  // TF32 = 2, kind::f16: BF16 = 1); both K-major; N >> 3 at 17-22, M >> 4 at
  // 24-28; M = N = 128
  static constexpr uint32_t kFmt = MODE == kBf16 ? 1u : 2u;
  static constexpr uint32_t kIdesc =
      (1u << 4) | (kFmt << 7) | (kFmt << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
};

HY_DEV uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

HY_DEV int64_t sample_dof_tc(const int* __restrict__ cells, int ns, int64_t nc, int64_t r) {
  const int v = (int)(r / ns);
  return (int64_t)v * nc + cells[r - (int64_t)v * ns];
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_sample_gram_tc(const float* __restrict__ phi, int64_t N, int m,
                     const int* __restrict__ cells, int ns, int nvar, int64_t nc, int64_t rpc,
                     double* __restrict__ part, int* __restrict__ err) {
  using P = Mode<MODE>;
  extern __shared__ unsigned char smraw[];
  unsigned char* ring = smraw + ((1024 - (saddr(smraw) & 1023u)) & 1023u);  // 1024-aligned
  __shared__ uint64_t full[P::kStages], empty[P::kStages], d_full;
  __shared__ uint32_t tmem_s;
  __shared__ volatile int stop_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nrows = (int64_t)ns * nvar;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = r0 + rpc < nrows ? r0 + rpc : nrows;
  const int nst = r1 > r0 ? (int)((r1 - r0 + kRowsStage - 1) / kRowsStage) : 0;

  if (tid == 0) {
    for (int s = 0; s < P::kStages; ++s) {
      mbar_init(&full[s], 16);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&d_full, 1);
    stop_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_s, kTmemCols);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;
  auto fail = [&]() {
    if (lane == 0) atomicExch(err, 1);
    stop_s = 1;
  };

  if (warp == 0) {
    // ---- MMA issue (one thread) ----
    if (lane == 0) {
      for (int g = 0; g < nst && !stop_s; ++g) {
        const int s = g % P::kStages;
        if (!mbar_wait(&full[s], (uint32_t)((g / P::kStages) & 1))) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = saddr(ring + s * P::kStageBytes);
#pragma unroll
        for (int a = 0; a < P::kAtoms; ++a)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K per MMA
            const uint64_t d = sdesc(st + a * kAtomBytes + kk * 32);
            const uint32_t acc = (g > 0 || a > 0 || kk > 0) ? 1u : 0u;
            if (MODE == kBf16)
              mma_f16(tmem, d, d, P::kIdesc, acc);
            else
              mma_tf32(tmem, d, d, P::kIdesc, acc);
          }
        mma_commit(&empty[s]);
      }
      // the accumulator's barrier completes once every MMA above has; wait
      // for it here too so that no MMA is in flight when the memory is freed
      mma_commit(&d_full);
      if (!mbar_wait(&d_full, 0)) fail();
    }
  } else {
    // ---- converters: lane = sample row of a 32-row block, 16 columns ----
    const int cw = warp - 1;
    const int blk = cw & 3, j0 = cw >> 2;  // columns j0 + 4 t
    const int rl = blk * 32 + lane;        // row within the stage
    for (int g = 0; g < nst && !stop_s; ++g) {
      const int s = g % P::kStages;
      const int64_t r = r0 + (int64_t)g * kRowsStage + rl;
      float x[kColsWarp];
      if (r < r1) {
        const int64_t dof = sample_dof_tc(cells, ns, nc, r);
#pragma unroll
        for (int t = 0; t < kColsWarp; ++t) {
          const int j = j0 + 4 * t;
          x[t] = j < m ? phi[(int64_t)j * N + dof] : 0.f;
        }
      } else {
#pragma unroll
        for (int t = 0; t < kColsWarp; ++t) x[t] = 0.f;
      }
      if (g >= P::kStages && !mbar_wait(&empty[s], (uint32_t)((g / P::kStages - 1) & 1))) {
        fail();
        break;
      }
      unsigned char* st = ring + s * P::kStageBytes;
      if (MODE == kTf32) {
        unsigned char* at = st + (rl >> 6) * kAtomBytes;
        const int h = (rl >> 5) & 1;
#pragma unroll
        for (int t = 0; t < kColsWarp; ++t)
          *reinterpret_cast<uint32_t*>(at + sw128(h * 64 + j0 + 4 * t, lane)) = to_tf32(x[t]);
      } else if (MODE == kBf16) {
        const int h = rl >> 6, k = rl & 63;
#pragma unroll
        for (int t = 0; t < kColsWarp; ++t)
          *reinterpret_cast<__nv_bfloat16*>(st + sw128_h(h * 64 + j0 + 4 * t, k)) =
              __float2bfloat16_rn(x[t]);
      } else {
        unsigned char* at = st + blk * kAtomBytes;
#pragma unroll
        for (int t = 0; t < kColsWarp; ++t) {
          const uint32_t hi = __float_as_uint(x[t]) & 0xFFFFE000u;
          const uint32_t lo = to_tf32(x[t] - __uint_as_float(hi));
          *reinterpret_cast<uint32_t*>(at + sw128(j0 + 4 * t, lane)) = hi;
          *reinterpret_cast<uint32_t*>(at + sw128(64 + j0 + 4 * t, lane)) = lo;
        }
      }
      // generic-proxy writes become visible to the tensor core's async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
    }

    // ---- epilogue: warps 1-4, one lane quarter of the accumulator each ----
    if (warp <= 4) {
      const int q = warp & 3;             // lanes 32 q .. 32 q + 31
      const int i = (q & 1) * 32 + lane;  // row of G
      float (*gs)[65] = reinterpret_cast<float (*)[65]>(ring);  // 64 x 65, ring reused
      bool ok = nst == 0 || mbar_wait(&d_full, 0);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
      if (!ok) fail();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16);
      // rows 0-63 of the accumulator (q < 2) write their diagonal block
      // (columns 0-63), then rows 64-127 add theirs (columns 64-127); the
      // split form adds the off-diagonal block of each row as well
      const uint32_t own = q < 2 ? 0u : 64u;
      // the named barriers are passed unconditionally by all four warps (a
      // warp that gave up only skips its memory accesses)
      for (int phase = 0; phase < 2; ++phase) {
        if (ok && (q >= 2) == (phase == 1)) {
#pragma unroll 1
          for (int hc = 0; hc < 2; ++hc) {
            float v[32];
            if (nst == 0) {
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] = 0.f;
            } else {
              tmem_ld32(ta + own + 32 * hc, v);
              if (MODE == kSplit) {
                float o[32];
                tmem_ld32(ta + (64u - own) + 32 * hc, o);
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] += o[j];
              }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (phase == 0)
                gs[i][32 * hc + j] = v[j];
              else
                gs[i][32 * hc + j] += v[j];
            }
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
      if (!stop_s)
        for (int e = tid - 32; e < 64 * 64; e += 128)
          part[(int64_t)blockIdx.x * 4096 + e] = (double)gs[e >> 6][e & 63];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

template <int MODE>
void launch_mode(const float* phi, int64_t N, int m, const int* cells, int ns, int nvar,
                 int64_t nc, double* part, int* nb_out, int* err, cudaStream_t s) {
  const int64_t nrows = (int64_t)ns * nvar;
  int64_t nb = (nrows + kRowsStage - 1) / kRowsStage;
  if (nb > 152) nb = 152;
  if (nb < 1) nb = 1;
  int64_t rpc = (nrows + nb - 1) / nb;
  rpc = (rpc + kRowsStage - 1) / kRowsStage * kRowsStage;
  nb = rpc > 0 ? (nrows + rpc - 1) / rpc : 1;
  if (nb < 1) nb = 1;
  cudaFuncSetAttribute(k_sample_gram_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kSmemBytes);
  k_sample_gram_tc<MODE><<<(int)nb, kThreads, kSmemBytes, HY_S(s)>>>(phi, N, m, cells, ns, nvar,
                                                                     nc, rpc, part, err);
  *nb_out = (int)nb;
}

}  // namespace

int launch_sample_gram_tc(const float* phi, int64_t N, int m, const int* cells, int ns, int nvar,
                          int64_t nc, int red, double* part, int* err, cudaStream_t s) {
  int nb = 0;
  if (red == kTf32)
    launch_mode<kTf32>(phi, N, m, cells, ns, nvar, nc, part, &nb, err, s);
  else if (red == kBf16)
    launch_mode<kBf16>(phi, N, m, cells, ns, nvar, nc, part, &nb, err, s);
  else
    launch_mode<kSplit>(phi, N, m, cells, ns, nvar, nc, part, &nb, err, s);
  return nb;
}

}  // namespace hy
