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
// The tensor core's FP32 accumulation is not unbiased: over n accumulating
// MMAs the error of a sum grows like n times the FP32 unit.  So no tensor
// memory accumulator runs for more than kPeriod stages: two accumulators
// alternate, and each finished one is drained into compensated (Kahan) FP32
// sums in shared memory while the MMAs fill the other.
//
// One CTA per SM takes a contiguous range of sample rows in stages (128
// rows; 64 for the split form):
//   * warps 1-16 (converters): each lane loads one sample row of 16 (split:
//     8) basis columns (a warp: 32 consecutive rows of one column per load,
//     coalesced along the sorted cells), rounds, and writes the swizzled
//     atoms;
//   * warp 0 (one thread): the MMAs of each full stage into the period's
//     accumulator, committed to the stage's empty barrier and at a period's
//     end to the accumulator's full barrier;
//   * warps 17-20 (epilogue, one lane quarter of the accumulators each):
//     tcgen05.ld of each finished accumulator, block sums, Kahan updates of
//     their rows, release of the accumulator; at the end the CTA's FP64
//     partial G to part[b * 4096 ...], summed in FP64 by the caller.
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

constexpr int kThreads = 672;      // 21 warps: MMA, 16 converters, 4 epilogue
constexpr int kAtomBytes = 16384;  // 128 rows x 128 bytes
constexpr int kRingBytes = 163840;
constexpr int kKahanBytes = 2 * 128 * 65 * 4;  // sums and compensations, 128 x 64 (+1 pad)
constexpr int kSmemBytes = kRingBytes + kKahanBytes + 1024;
constexpr int kPeriod = 2;         // stages per accumulator period
constexpr uint32_t kTmemCols = 256;  // two 128 x 128 FP32 accumulators

enum { kTf32 = 1, kBf16 = 2, kSplit = 3 };  // the HYROM_RED_* values

template <int MODE>
struct Mode {
  // sample rows per atom and per stage, atoms per stage, stages in the ring
  static constexpr int kRowsAtom = MODE == kBf16 ? 128 : (MODE == kTf32 ? 64 : 32);
  static constexpr int kRowsStage = MODE == kSplit ? 64 : 128;
  static constexpr int kAtoms = kRowsStage / kRowsAtom;
  static constexpr int kStageBytes = kAtoms * kAtomBytes;
  static constexpr int kStages = kRingBytes / kStageBytes;
  // converter warps: 32-row blocks per stage, columns per warp, column step
  static constexpr int kBlk = kRowsStage / 32;
  static constexpr int kColsWarp = 4 * kBlk;
  static constexpr int kColStep = 16 / kBlk;
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
  float (*ks)[65] = reinterpret_cast<float (*)[65]>(ring + kRingBytes);  // Kahan sums
  float (*kc)[65] = ks + 128;                                            // compensations
  __shared__ uint64_t full[P::kStages], empty[P::kStages], d_full[2], d_empty[2], d_all;
  __shared__ uint32_t tmem_s;
  __shared__ volatile int stop_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nrows = (int64_t)ns * nvar;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = r0 + rpc < nrows ? r0 + rpc : nrows;
  const int nst = r1 > r0 ? (int)((r1 - r0 + P::kRowsStage - 1) / P::kRowsStage) : 0;
  const int nper = (nst + kPeriod - 1) / kPeriod;

  if (tid == 0) {
    for (int s = 0; s < P::kStages; ++s) {
      mbar_init(&full[s], 16);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d_full[b], 1);
      mbar_init(&d_empty[b], 4);
    }
    mbar_init(&d_all, 1);
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
        const int p = g / kPeriod, b = p & 1;
        const bool first = g % kPeriod == 0;
        if (first && p >= 2 && !mbar_wait(&d_empty[b], (uint32_t)(((p >> 1) - 1) & 1))) {
          fail();
          break;
        }
        if (!mbar_wait(&full[s], (uint32_t)((g / P::kStages) & 1))) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = saddr(ring + s * P::kStageBytes);
        const uint32_t d = tmem + 128u * (uint32_t)b;
#pragma unroll
        for (int a = 0; a < P::kAtoms; ++a)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K per MMA
            const uint64_t desc = sdesc(st + a * kAtomBytes + kk * 32);
            const uint32_t acc = (!first || a > 0 || kk > 0) ? 1u : 0u;
            if (MODE == kBf16)
              mma_f16(d, desc, desc, P::kIdesc, acc);
            else
              mma_tf32(d, desc, desc, P::kIdesc, acc);
          }
        mma_commit(&empty[s]);
        if (g % kPeriod == kPeriod - 1 || g == nst - 1) mma_commit(&d_full[b]);
      }
      // completes once every MMA above has: none is in flight when the
      // tensor memory is freed
      mma_commit(&d_all);
      if (!mbar_wait(&d_all, 0)) fail();
    }
  } else if (warp <= 16) {
    // ---- converters: lane = sample row of a 32-row block ----
    const int cw = warp - 1;
    const int blk = cw % P::kBlk, j0 = cw / P::kBlk;  // columns j0 + kColStep t
    const int rl = blk * 32 + lane;                   // row within the stage
    // the gathers of stage g + 1 are issued before stage g waits for its
    // ring slot, so two stages of loads are in flight per thread
    auto gather = [&](int g, float* x) {
      const int64_t r = r0 + (int64_t)g * P::kRowsStage + rl;
      if (g < nst && r < r1) {
        const int64_t dof = sample_dof_tc(cells, ns, nc, r);
#pragma unroll
        for (int t = 0; t < P::kColsWarp; ++t) {
          const int j = j0 + P::kColStep * t;
          x[t] = j < m ? phi[(int64_t)j * N + dof] : 0.f;
        }
      } else {
#pragma unroll
        for (int t = 0; t < P::kColsWarp; ++t) x[t] = 0.f;
      }
    };
    float xn[P::kColsWarp];
    gather(0, xn);
    for (int g = 0; g < nst && !stop_s; ++g) {
      const int s = g % P::kStages;
      float x[P::kColsWarp];
#pragma unroll
      for (int t = 0; t < P::kColsWarp; ++t) x[t] = xn[t];
      gather(g + 1, xn);
      if (g >= P::kStages && !mbar_wait(&empty[s], (uint32_t)((g / P::kStages - 1) & 1))) {
        fail();
        break;
      }
      unsigned char* st = ring + s * P::kStageBytes;
      if (MODE == kTf32) {
        unsigned char* at = st + (rl >> 6) * kAtomBytes;
        const int h = (rl >> 5) & 1;
#pragma unroll
        for (int t = 0; t < P::kColsWarp; ++t)
          *reinterpret_cast<uint32_t*>(at + sw128(h * 64 + j0 + P::kColStep * t, lane)) =
              to_tf32(x[t]);
      } else if (MODE == kBf16) {
        const int h = rl >> 6, k = rl & 63;
#pragma unroll
        for (int t = 0; t < P::kColsWarp; ++t)
          *reinterpret_cast<__nv_bfloat16*>(st + sw128_h(h * 64 + j0 + P::kColStep * t, k)) =
              __float2bfloat16_rn(x[t]);
      } else {
        unsigned char* at = st + blk * kAtomBytes;
#pragma unroll
        for (int t = 0; t < P::kColsWarp; ++t) {
          const uint32_t hi = __float_as_uint(x[t]) & 0xFFFFE000u;
          const uint32_t lo = to_tf32(x[t] - __uint_as_float(hi));
          const int j = j0 + P::kColStep * t;
          *reinterpret_cast<uint32_t*>(at + sw128(j, lane)) = hi;
          *reinterpret_cast<uint32_t*>(at + sw128(64 + j, lane)) = lo;
        }
      }
      // generic-proxy writes become visible to the tensor core's async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
    }
  } else {
    // ---- epilogue: warps 17-20, lanes 32 q .. 32 q + 31 of each accumulator ----
    const int q = warp & 3;
    const int drow = 32 * q + lane;  // accumulator row = tensor-memory lane
    // accumulator rows 0-63 take their diagonal block (columns 0-63), rows
    // 64-127 theirs (64-127); the split form adds the other block too
    const uint32_t own = q < 2 ? 0u : 64u;
#pragma unroll 8
    for (int j = 0; j < 64; ++j) ks[drow][j] = kc[drow][j] = 0.f;
    for (int p = 0; p < nper && !stop_s; ++p) {
      const int b = p & 1;
      bool ok = mbar_wait(&d_full[b], (uint32_t)((p >> 1) & 1));
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
      if (!ok) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + 128u * (uint32_t)b;
#pragma unroll 1
      for (int hc = 0; hc < 2; ++hc) {
        float v[32];
        tmem_ld32(ta + own + 32 * hc, v);
        if (MODE == kSplit) {
          float o[32];
          tmem_ld32(ta + (64u - own) + 32 * hc, o);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += o[j];
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float sj = ks[drow][32 * hc + j];
          const float y = v[j] - kc[drow][32 * hc + j];
          const float t = sj + y;
          kc[drow][32 * hc + j] = (t - sj) - y;
          ks[drow][32 * hc + j] = t;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_empty[b]);
    }
    // passed unconditionally by all four epilogue warps
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (!stop_s)
      for (int e = tid - 17 * 32; e < 64 * 64; e += 128) {
        const int i = e >> 6, j = e & 63;
        part[(int64_t)blockIdx.x * 4096 + e] =
            ((double)ks[i][j] - (double)kc[i][j]) + ((double)ks[64 + i][j] - (double)kc[64 + i][j]);
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
  constexpr int kRS = Mode<MODE>::kRowsStage;
  const int64_t nrows = (int64_t)ns * nvar;
  int64_t nb = (nrows + kRS - 1) / kRS;
  if (nb > 152) nb = 152;
  if (nb < 1) nb = 1;
  int64_t rpc = (nrows + nb - 1) / nb;
  rpc = (rpc + kRS - 1) / kRS * kRS;
  nb = rpc > 0 ? (nrows + rpc - 1) / rpc : 1;
  if (nb < 1) nb = 1;
  smem_at_least((const void*)k_sample_gram_tc<MODE>, kSmemBytes);
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
