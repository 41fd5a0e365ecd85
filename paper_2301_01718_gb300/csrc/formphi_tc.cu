// The POD basis product Phi = (X - psi 1^T) C and the next reference state
// psi_next = mean of the window (Sec. 2.2, POD and window mean) on the
// 5th-generation tensor cores.
//
// X is the snapshot window (N rows x w slots of the FP32 ring), C the w x m
// coefficient matrix V Sigma^{-1} (m <= 64, w <= 128).  The product is a
// dense contraction of 2 N w m flops over 4 N (w + m + 2) bytes, so on the
// tensor cores it is bound by HBM.  FP32 accuracy is kept with TF32 and an
// error-compensated split: with a = a_hi + a_lo (a_hi = a with its 13 low
// mantissa bits cleared, a_lo exact), a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// (error ~2^-21 |a||b|): B's hi and lo splits form one 128-column operand, so
// that a_hi times both is one MMA (N = 128) and a_lo b_hi a second (N = 64)
// into the first 64 columns; the epilogue adds the two halves.
//
// One persistent CTA per SM takes 128-row tiles, with warp-specialised
// roles handing chunks of 32 window slots to each other through mbarriers:
//   * warp 0 (producer): a chunk (128 rows x 32 window slots) into a 4-stage
//     ring of raw FP32 chunks by one 2D tensor copy (cp.async.bulk.tensor
//     over the snapshot ring, rows x slots) when its slots are consecutive
//     in the ring, else by bulk copies of one 512-byte slot per lane;
//   * warps 8-11 (converters, one thread per row): Kahan window sum, centring
//     by psi, TF32 hi/lo split, writes into a 2-stage ring of A tiles in the
//     128-byte-swizzled K-major layout the tensor core reads; at a tile's
//     end each writes its row of psi_next;
//   * warp 1 (MMA): per chunk 4 x 2 tcgen05.mma (M = 128, N = 128 and 64,
//     K = 8, kind::tf32) into one of two 128 x 128 FP32 accumulators in
//     tensor memory (tiles alternate), committed to the chunk's and tile's
//     mbarriers;
//   * warps 4-7 (epilogue): tcgen05.ld of a finished accumulator (warp w:
//     rows 32 (w % 4) ..), the sum of its halves, release, and coalesced
//     stores of Phi; when
//     asked, also each row's squared-norm bound and bucket for ODEIM (the
//     FP32 sum in column order, as ODEIM's own row-norm pass forms it), with
//     per-CTA bucket counts and maxima in shared memory flushed at the end.
// C is split and staged once per CTA.  Every mbarrier wait is bounded (about
// a second); a timeout sets *err and a shared stop flag that ends every
// role's loop, and the tensor memory is freed before the CTA returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace hy {
namespace {

using namespace tc;
static_assert(kNormBucketCount == kNormBuckets, "row-norm buckets");

constexpr int kRows = 128;     // tile rows (UMMA M)
constexpr int kCols = 64;      // basis columns (UMMA N), zero padded beyond m_eff
constexpr int kChunk = 32;     // window slots per chunk: one 128-byte atom of TF32
constexpr int kMaxW = 128;
constexpr int kThreads = 384;  // 12 warps: producer, MMA, 2 idle, 4 epilogue, 4 converters
constexpr int kRawStages = 4;
constexpr int kAStages = 2;
constexpr int kBBytes = (kMaxW / kChunk) * (kCols / 8) * kAtomGroup;  // 32 KB
constexpr int kABytes = (kRows / 8) * kAtomGroup;                    // 16 KB
constexpr int kRawBytes = kChunk * kRows * 4;                        // 16 KB
constexpr int kSmemBytes = 2 * kBBytes + kAStages * 2 * kABytes + kRawStages * kRawBytes + 1024;
constexpr uint32_t kTmemCols = 256;  // two 128-column accumulators (hi.hi + lo.hi | hi.lo)

// kind::tf32: D in FP32 (bits 4-5 = 1), A and B TF32 (format 2 at bits 7-9
// and 10-12), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                            ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

// the same with N = 128: B's hi and lo halves as one operand
constexpr uint32_t kIdesc2 = (1u << 4) | (2u << 7) | (2u << 10) |
                             ((uint32_t)((2 * kCols) >> 3) << 17) |
                             ((uint32_t)(kRows >> 4) << 24);

HY_DEV void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_form_phi_tc(const __grid_constant__ CUtensorMap tmap, int use_tma,
                  const float* __restrict__ ring, int64_t N, const int* __restrict__ win, int w,
                  const float* __restrict__ psi, const float* __restrict__ C, int m,
                  const int* __restrict__ m_eff_dev, float* __restrict__ phi,
                  float* __restrict__ psi_next, int* __restrict__ err, OdeimNorms nout) {
  extern __shared__ unsigned char smraw[];
  unsigned char* base =
      smraw + ((1024 - (saddr(smraw) & 1023u)) & 1023u);  // 1024-byte aligned
  // B per chunk of 32 window slots: its hi split in rows 0..63, its lo split
  // in rows 64..127 of one 128-row operand (16 KB)
  unsigned char* Bcat = base;
  unsigned char* Aarea = Bcat + 2 * kBBytes;                             // kAStages x (hi, lo)
  float* raw = reinterpret_cast<float*>(Aarea + kAStages * 2 * kABytes);  // kRawStages chunks
  __shared__ uint64_t raw_full[kRawStages], raw_empty[kRawStages];
  __shared__ uint64_t a_full[kAStages], a_empty[kAStages], d_full[2], d_empty[2];
  __shared__ uint32_t tmem_s;
  __shared__ int ws[kMaxW];
  __shared__ volatile int stop_s;
  __shared__ int hcnt[kNormBuckets];
  __shared__ unsigned int hmax[kNormBuckets];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int me = *m_eff_dev;
  const int nch = (w + kChunk - 1) / kChunk;
  const int64_t ntile = (N + kRows - 1) / kRows;
  const int64_t my_tiles = ntile > blockIdx.x ? (ntile - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * nch;  // chunks this CTA processes

  // C split into TF32 hi/lo, K-major swizzled: B[n][k], one block per atom of k
  for (int i = tid; i < kMaxW * kCols; i += kThreads) {
    const int k = i / kCols, n = i % kCols;
    const float c = (k < w && n < m && n < me) ? C[k * m + n] : 0.f;
    float hi, lo;
    split_tf32(c, hi, lo);
    const int off = (k / kChunk) * 2 * (kCols / 8) * kAtomGroup;
    *reinterpret_cast<float*>(Bcat + off + sw128(n, k % kChunk)) = hi;
    *reinterpret_cast<float*>(Bcat + off + sw128(n + kCols, k % kChunk)) = lo;
  }
  for (int i = tid; i < w; i += kThreads) ws[i] = win[i];
  for (int i = tid; i < kNormBuckets; i += kThreads) {
    hcnt[i] = 0;
    hmax[i] = 0u;
  }
  if (tid == 0) {
    for (int s = 0; s < kRawStages; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], 4);
    }
    for (int s = 0; s < kAStages; ++s) {
      mbar_init(&a_full[s], 4);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&d_full[s], 1);
      mbar_init(&d_empty[s], 4);
    }
    stop_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&tmem_s)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // generic-proxy writes of B become visible to the tensor core's async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;
  auto fail = [&]() {
    if (lane == 0) atomicExch(err, 1);
    stop_s = 1;
  };

  if (warp == 0) {
    // ---- producer: raw chunk g into stage g % kRawStages ----
    for (int64_t g = 0; g < total && !stop_s; ++g) {
      const int s = (int)(g % kRawStages);
      if (g >= kRawStages &&
          !mbar_wait(&raw_empty[s], (uint32_t)((g / kRawStages - 1) & 1))) {
        fail();
        break;
      }
      const int64_t tile = blockIdx.x + (g / nch) * (int64_t)gridDim.x;
      const int c = (int)(g % nch);
      const int64_t row0 = tile * kRows;
      const int rows = (int)(N - row0 < kRows ? N - row0 : kRows);
      const int k0 = c * kChunk;
      const int nk = w - k0 < kChunk ? w - k0 : kChunk;
      float* dst = raw + s * (kRawBytes / 4);
      const bool cons =
          use_tma && __all_sync(0xffffffffu, lane >= nk || ws[k0 + lane] == ws[k0] + lane);
      if (cons) {
        // one box of 128 rows x 32 slots, laid out like the per-slot copies
        // (slot-major); rows past N and slots past the ring read as zero
        if (lane == 0) {
          mbar_expect_tx(&raw_full[s], (uint32_t)kRawBytes);
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
              "l"(reinterpret_cast<uint64_t>(&tmap)), "r"((int)row0), "r"(ws[k0]),
              "r"(saddr(&raw_full[s]))
              : "memory");
        }
      } else {
        if (lane == 0) mbar_expect_tx(&raw_full[s], (uint32_t)(nk * rows * 4));
        __syncwarp();
        if (lane < nk)
          bulk_g2s(dst + lane * kRows, ring + (int64_t)ws[k0 + lane] * N + row0,
                   (uint32_t)(rows * 4), &raw_full[s]);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue (one thread) ----
    if (lane == 0) {
      for (int64_t g = 0; g < total && !stop_s; ++g) {
        const int64_t t = g / nch;
        const int c = (int)(g % nch);
        const int as = (int)(g % kAStages), b = (int)(t & 1);
        if (!mbar_wait(&a_full[as], (uint32_t)((g / kAStages) & 1))) {
          fail();
          break;
        }
        if (c == 0 && t >= 2 && !mbar_wait(&d_empty[b], (uint32_t)(((t >> 1) - 1) & 1))) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(2 * kCols * b);
        unsigned char* Ahi = Aarea + as * 2 * kABytes;
        const uint32_t ahi = saddr(Ahi), alo = saddr(Ahi + kABytes);
        const uint32_t bcat = saddr(Bcat) + (uint32_t)(c * 2 * (kCols / 8) * kAtomGroup);
#pragma unroll
        for (int kk = 0; kk < kChunk / 8; ++kk) {
          const uint32_t ko = kk * 32;  // 8 TF32 = 32 bytes along k inside the atom
          const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
          // columns 0..63 += a_hi b_hi, 64..127 += a_hi b_lo; then 0..63 += a_lo b_hi
          mma_tf32(d, sdesc(ahi + ko), sdesc(bcat + ko), kIdesc2, acc0);
          mma_tf32(d, sdesc(alo + ko), sdesc(bcat + ko), kIdesc, 1u);
        }
        mma_commit(&a_empty[as]);
        if (c == nch - 1) mma_commit(&d_full[b]);
      }
    }
  } else if (warp >= 8) {
    // ---- converters: thread = row, all 32 slots of each chunk ----
    const int row = tid - 8 * 32;
    // four Kahan accumulators (slot index mod 4) keep the dependent chains short
    float ksum[4] = {0.f, 0.f, 0.f, 0.f}, kcomp[4] = {0.f, 0.f, 0.f, 0.f};
    float pr = 0.f, pr_next = 0.f;
    if (my_tiles > 0) {
      const int64_t r0 = (int64_t)blockIdx.x * kRows + row;
      pr_next = r0 < N ? psi[r0] : 0.f;
    }
    for (int64_t g = 0; g < total; ++g) {
      if (__any_sync(0xffffffffu, stop_s != 0)) break;  // warp-uniform (__syncwarp below)
      const int64_t t = g / nch;
      const int c = (int)(g % nch);
      const int64_t row0 = (blockIdx.x + t * (int64_t)gridDim.x) * kRows;
      const bool valid = row0 + row < N;
      if (c == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) ksum[u] = kcomp[u] = 0.f;
        pr = pr_next;
        const int64_t rn = row0 + (int64_t)gridDim.x * kRows + row;  // next tile's row
        pr_next = (t + 1 < my_tiles && rn < N) ? psi[rn] : 0.f;
      }
      const int rs = (int)(g % kRawStages), as = (int)(g % kAStages);
      if (!__all_sync(0xffffffffu, mbar_wait(&raw_full[rs], (uint32_t)((g / kRawStages) & 1)))) {
        fail();
        break;
      }
      const float* rv = raw + rs * (kRawBytes / 4);
      const int k0 = c * kChunk;
      float x[kChunk];
#pragma unroll
      for (int kl = 0; kl < kChunk; ++kl) {
        float v = 0.f;
        if (k0 + kl < w && valid) {
          const float gv = rv[kl * kRows + row];
          const int u = kl & 3;
          const float yk = gv - kcomp[u], tk = ksum[u] + yk;
          kcomp[u] = (tk - ksum[u]) - yk;
          ksum[u] = tk;
          v = gv - pr;
        }
        x[kl] = v;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&raw_empty[rs]);
      if (g >= kAStages &&
          !__all_sync(0xffffffffu, mbar_wait(&a_empty[as], (uint32_t)((g / kAStages - 1) & 1)))) {
        fail();
        break;
      }
      unsigned char* Ahi = Aarea + as * 2 * kABytes;
      unsigned char* Alo = Ahi + kABytes;
#pragma unroll
      for (int q = 0; q < kChunk / 4; ++q) {
        float hi4[4], lo4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_tf32(x[4 * q + e], hi4[e], lo4[e]);
        const int off = sw128(row, 4 * q);
        *reinterpret_cast<float4*>(Ahi + off) = make_float4(hi4[0], hi4[1], hi4[2], hi4[3]);
        *reinterpret_cast<float4*>(Alo + off) = make_float4(lo4[0], lo4[1], lo4[2], lo4[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_full[as]);
      if (c == nch - 1 && valid) {
        // Kahan-add the four partial sums (each carried with its compensation)
        float sum = 0.f, comp = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float yk = (ksum[u] - kcomp[u]) - comp, tk = sum + yk;
          comp = (tk - sum) - yk;
          sum = tk;
        }
        psi_next[row0 + row] = (sum - comp) / (float)w;
      }
    }
  } else if (warp >= 4) {
    // ---- epilogue: accumulator of tile t -> Phi ----
    const int lanegrp = warp & 3;
    // loop decisions are warp-uniform: the loads and ballots below are
    // warp-collective
    for (int64_t t = 0; t < my_tiles; ++t) {
      if (__any_sync(0xffffffffu, stop_s != 0)) break;
      const int b = (int)(t & 1);
      if (!__all_sync(0xffffffffu, mbar_wait(&d_full[b], (uint32_t)((t >> 1) & 1)))) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v0[32], v1[32];
      const uint32_t ta = tmem + ((uint32_t)(32 * lanegrp) << 16) + (uint32_t)(2 * kCols * b);
      {  // column j of Phi: (a_hi b_hi + a_lo b_hi) in column j, a_hi b_lo in 64 + j
        float u[32];
        tmem_ld32(ta, v0);
        tmem_ld32(ta + 64, u);
#pragma unroll
        for (int j = 0; j < 32; ++j) v0[j] += u[j];
        tmem_ld32(ta + 32, v1);
        tmem_ld32(ta + 96, u);
#pragma unroll
        for (int j = 0; j < 32; ++j) v1[j] += u[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_empty[b]);
      const int64_t r = (blockIdx.x + t * (int64_t)gridDim.x) * kRows + 32 * lanegrp + lane;
      if (r < N) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j < me) phi[(int64_t)j * N + r] = v0[j];
          if (32 + j < me) phi[(int64_t)(32 + j) * N + r] = v1[j];
        }
      }
      if (nout.nrm) {
        const bool valid = r < N;
        float acc = 0.f;  // columns past m_eff are zero
#pragma unroll
        for (int j = 0; j < 32; ++j) acc = fmaf(v0[j], v0[j], acc);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc = fmaf(v1[j], v1[j], acc);
        // an upper bound of the exact squared norm (m terms of relative
        // error <= 2^-24 each; 1e-5 covers m <= 128)
        const float up = __double2float_ru((double)acc * (1.0 + 1e-5));
        const int b = nrm_bucket(up);
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (valid) {
          nout.nrm[r] = up;
          nout.bkt[r] = (unsigned char)b;
          const unsigned peers = __match_any_sync(vm, b);
          const unsigned mx = __reduce_max_sync(peers, __float_as_uint(up));
          if (lane == __ffs(peers) - 1) {
            atomicAdd(&hcnt[b], __popc(peers));
            atomicMax(&hmax[b], mx);
          }
        }
      }
    }
  }
  // all roles done; in-flight MMAs ended before their last commit was seen
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (nout.nrm)
    for (int i = tid; i < kNormBuckets; i += kThreads)
      if (hcnt[i]) {
        atomicAdd(&nout.bcnt[i], hcnt[i]);
        atomicMax(&nout.bmax[i], hmax[i]);
      }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

}  // namespace

bool form_phi_tc_ok(int64_t N, int w, int m) {
  return N > 0 && (N & 3) == 0 && w >= 1 && w <= kMaxW && m >= 1 && m <= kCols;
}

// the driver's tensor-map encoder, through the runtime (no link to libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

void launch_form_phi_tc(const float* ring, int64_t N, int nslot, const int* win, int w,
                        const float* psi, const float* C, int m, const int* m_eff_dev,
                        float* phi, float* psi_next, int* err, OdeimNorms norms,
                        cudaStream_t s) {
  smem_at_least((const void*)k_form_phi_tc, kSmemBytes);
  int64_t tiles = (N + kRows - 1) / kRows;
  const int grid = (int)(tiles < 152 ? tiles : 152);
  // the ring as a 2D tensor: rows (contiguous, N) x slots (stride 4 N bytes),
  // boxes of kRows x kChunk; the per-slot copies serve if it cannot be made
  CUtensorMap tmap;
  int use_tma = 0;
  if (PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder()) {
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)nslot};
    const cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kRows, (cuuint32_t)kChunk};
    const cuuint32_t estr[2] = {1, 1};
    use_tma = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ring), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  if (!use_tma) memset(&tmap, 0, sizeof(tmap));
  k_form_phi_tc<<<grid, kThreads, kSmemBytes, HY_S(s)>>>(tmap, use_tma, ring, N, win, w, psi, C,
                                                         m, m_eff_dev, phi, psi_next, err, norms);
}

}  // namespace hy
