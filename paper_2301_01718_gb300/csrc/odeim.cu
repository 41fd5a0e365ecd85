// ODEIM_{n_p}(Phi) (Eq. odeim of the paper): the DEIM points, then greedy
// oversampling points, each maximising lambda_min(A^T A + phi_i phi_i^T)
// (A = P^T Phi over the points so far, phi_i a candidate row).
//
// Each greedy step is an exact arg-max over all N rows (ties within
// relative tie_tol go to the lowest row), but the exact FP64 score is only
// evaluated on rows that can still win:
//   * rows are bucketed once per basis by an upper bound of their squared
//     norm nrm_i = |Phi[i, :]|^2 (buckets of a factor 2^(1/4), in
//     decreasing order; each bucket records its largest bound);
//   * DEIM step l: |r_i| <= sqrt(nrm_i) sqrt(1 + |c|^2) for the interpolation
//     residual r = phi_l - Phi_{:, <l} c, so rows with
//     nrm_i < s*^2 (1 - 2 tie_tol)^2 / (1 + |c|^2) cannot reach the best score
//     s* found on a probe of the largest-norm rows;
//   * ODEIM step: lambda_min(M + phi phi^T) <= lambda_1(M) + |phi|^2 and
//     <= min(lambda_2, lambda_1 + (w_1 . phi)^2) (Rayleigh quotient on the
//     eigenvector w_1, and interlacing), so rows below either bound are
//     skipped; survivors get the smallest root of the secular equation
//     1 + sum_j z_j^2 / (lambda_j - mu) = 0, z = W^T phi, by bisection.
// Every decision is taken in FP64 on the same quantity an FP64 reference
// computes, so the chosen points do not depend on the pruning.
#include <math.h>

#include <new>
#include <utility>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace hy {

constexpr int kNB = 256;       // norm buckets
constexpr int kProbe = 2048;   // rows scored before the bound is applied
constexpr int kLdw = 65;       // odd leading dimension of W in shared memory
constexpr int kCompact = 524288;  // leading ordered rows kept row-major (FP32, 64 wide)
// the step's eigensystem in FP32 for the screens: W^T (64 x 64), then the
// poles relative to lam_1 (dn, du, dd) and to lam_2 (en, eu, ed), then
// lam_2 - lam_1 (rounded to nearest, upward, downward)
constexpr int kW32 = 64 * 64 + 7 * 64;

struct OdCtl {
  unsigned long long smax;  // bits of the best score so far (>= 0)
  int argmin;               // winning row (lowest index within the tie window)
  int n_c;                  // ordered rows to score
  double cn2;               // 1 + |c|^2            (DEIM)
  double lam1, lam2, lmax;  // eigenvalues of M (ODEIM)
  int n_list;                // rows passed on by the z_1 filter (ODEIM)
  int eig_sweeps;            // Jacobi sweeps of the first eigensystem (ODEIM)
  unsigned long long slo;    // bits of the best certified lower bound (ODEIM)
  int ncand;                 // candidates listed in the step
  int n_x;                   // rows listed for exact scores (ODEIM)
  unsigned ticket;           // CTAs finished in the current pass
  // counters over one ODEIM call: DEIM rows scored, ODEIM rows given the
  // full FP32 bound, ODEIM exact scores, greedy steps
  unsigned long long stat[4];
};

size_t odeim_ctl_bytes() { return 256; }

// counters of the last ODEIM call (the control block heads the workspace)
void odeim_stats(const void* ws, unsigned long long* out4, cudaStream_t s) {
  const OdCtl* c = (const OdCtl*)ws;
  cudaMemcpyAsync(out4, c->stat, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
}

// Jacobi sweeps of the last ODEIM call's first eigensystem
void odeim_eig_sweeps(const void* ws, int* out, cudaStream_t s) {
  const OdCtl* c = (const OdCtl*)ws;
  cudaMemcpyAsync(out, &c->eig_sweeps, sizeof(int), cudaMemcpyDeviceToHost, s);
}

// sqrt(x) for x >= 0 from the approximate reciprocal square root: the FP32
// model steps of the root solvers and screens only steer their iterates
// (every bound is certified apart, every root finished in FP64)
HY_DEV float fsqrt_fast(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// ---- row norms and buckets --------------------------------------------------

static_assert(kNB == kNormBuckets, "row-norm buckets");

template <typename T>
__global__ void k_rownorm(const T* __restrict__ phi, int64_t N, int m, float* __restrict__ nrm,
                          unsigned char* __restrict__ bkt, int* __restrict__ bcnt,
                          unsigned int* __restrict__ bmax) {
  __shared__ int sc[kNB];
  __shared__ unsigned int sm[kNB];
  for (int i = threadIdx.x; i < kNB; i += blockDim.x) {
    sc[i] = 0;
    sm[i] = 0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    T acc = (T)0;
    for (int j = 0; j < m; ++j) {
      const T x = phi[(int64_t)j * N + i];
      acc = fma(x, x, acc);
    }
    // an upper bound of the exact squared norm (m terms of relative error
    // <= 2^-24 each for FP32 data; 1e-5 covers m <= 128)
    const float up = __double2float_ru((double)acc * (1.0 + 1e-5));
    nrm[i] = up;
    const int b = nrm_bucket(up);
    bkt[i] = (unsigned char)b;
    atomicAdd(&sc[b], 1);
    atomicMax(&sm[b], __float_as_uint(up));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNB; i += blockDim.x) {
    if (sc[i]) {
      atomicAdd(&bcnt[i], sc[i]);
      atomicMax(&bmax[i], sm[i]);
    }
  }
}

__global__ void k_bucket_scan(const int* __restrict__ bcnt, int* __restrict__ bstart,
                              int* __restrict__ bcur) {
  if (threadIdx.x == 0) {
    int a = 0;
    for (int b = 0; b < kNB; ++b) {
      bstart[b] = a;
      bcur[b] = a;
      a += bcnt[b];
    }
    bstart[kNB] = a;
  }
}

// warp-aggregated: lanes with the same bucket share one atomic
__global__ void k_bucket_scatter(int64_t N, const unsigned char* __restrict__ bkt, int* bcur,
                                 int* __restrict__ ord) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; base < N;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + lane;
    const bool valid = i < N;
    const int b = valid ? bkt[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int pos = 0;
    if (valid && lane == leader) pos = atomicAdd(&bcur[b], __popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (valid) ord[pos + rank] = (int)i;
  }
}

// ---- DEIM -------------------------------------------------------------------

// Rows ord[0 .. C) of Phi copied once per call into a row-major FP32 array
// R (64 values per row, zero beyond m), so that the per-step scoring passes
// read each candidate row as 256 contiguous bytes instead of m scattered
// sectors of the column-major basis.  One warp per row.
template <typename T>
__global__ void k_gather_rows(const T* __restrict__ phi, int64_t N, int m,
                              const int* __restrict__ ord, int C, float* __restrict__ R) {
  const int lane = threadIdx.x & 31;
  for (int pos = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pos < C;
       pos += gridDim.x * (blockDim.x >> 5)) {
    const int i = ord[pos];
    const float x0 = lane < m ? (float)phi[(int64_t)lane * N + i] : 0.f;
    const float x1 = lane + 32 < m ? (float)phi[(int64_t)(lane + 32) * N + i] : 0.f;
    R[(int64_t)pos * 64 + lane] = x0;
    R[(int64_t)pos * 64 + lane + 32] = x1;
  }
}

// Value a of row i of Phi: from the row copy where the row's ordered
// position is inside it (it holds the FP32 values exactly), else from Phi.
template <typename T>
HY_DEV double phi_at(const T* __restrict__ phi, int64_t N, int a, int i, int pos,
                     const float* __restrict__ R, int C) {
  if (sizeof(T) == 4 && pos >= 0 && pos < C) return (double)R[(int64_t)pos * 64 + a];
  return (double)phi[(int64_t)a * N + i];
}

// The last non-empty bucket whose largest squared-norm bound reaches tau
// bounds the ordered rows still to score: every row after it has a smaller
// bound.  Returns max(that end, probe_end); all threads of the CTA get it.
HY_DEV int plan_end(const unsigned int* __restrict__ bmax, const int* __restrict__ bstart,
                    int probe_end, double tau) {
  __shared__ int red[32];
  int blast = -1;
  for (int b = threadIdx.x; b < kNB; b += blockDim.x)
    if (bstart[b + 1] > bstart[b] && (double)__uint_as_float(bmax[b]) >= tau) blast = b;
  for (int o = 16; o > 0; o >>= 1) blast = max(blast, __shfl_xor_sync(0xffffffffu, blast, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = blast;
  __syncthreads();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) blast = max(blast, red[w]);
  const int n = blast >= 0 ? bstart[blast + 1] : 0;
  __syncthreads();
  return n > probe_end ? n : probe_end;
}

// Block-wide maximum of unsigned 64-bit keys (integer compares: the FP64
// compare runs on the narrow FP64 pipe).  All threads get the result.
HY_DEV unsigned long long block_max_u64(unsigned long long v) {
  __shared__ unsigned long long sh[32];
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = sh[w] > v ? sh[w] : v;
  __syncthreads();
  return v;
}

HY_DEV unsigned long long block_min_u64(unsigned long long v) {
  __shared__ unsigned long long sh[32];
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u < v ? u : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = sh[w] < v ? sh[w] : v;
  __syncthreads();
  return v;
}

// One pass of a greedy step's scoring, block-synchronous (every thread of
// the CTA calls it with its score sc, or -1 for none): the best score of the
// pass raises the step's best ctl->smax, and scores that reach the tie
// window of the best known to this CTA (its own passes and the global best
// returned by the atomic) are appended to the candidate list.  The final
// winner's tie window lies inside every such window, so the list holds every
// row that can still win (and some that cannot, which the final pick drops).
// run: this CTA's running best (dbits of a non-negative double).
HY_DEV void note_scores(double sc, int pos, double tie_tol, unsigned long long& run, OdCtl* ctl,
                        int* __restrict__ cand) {
  __shared__ unsigned long long runs;
  const unsigned long long k = sc > 0.0 ? dbits(sc) : 0ull;
  const unsigned long long bm = block_max_u64(k);
  if (threadIdx.x == 0) {
    unsigned long long r = run > bm ? run : bm;
    if (bm > run) {
      const unsigned long long old = atomicMax(&ctl->smax, bm);
      r = old > r ? old : r;
    }
    runs = r;
  }
  __syncthreads();
  run = runs;
  const bool keep = sc >= 0.0 && sc >= bitsd(run) * (1.0 - tie_tol);
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  if (bal) {
    const int lane = threadIdx.x & 31;
    int first = 0;
    if (lane == __ffs(bal) - 1) first = atomicAdd(&ctl->ncand, __popc(bal));
    first = __shfl_sync(0xffffffffu, first, __ffs(bal) - 1);
    if (keep) cand[first + __popc(bal & ((1u << lane) - 1u))] = pos;
  }
  __syncthreads();
}

// True in the CTA that finishes a grid of nb CTAs last (all threads); its
// reads of what the other CTAs wrote see their writes.
HY_DEV bool last_block(unsigned* ticket, unsigned nb) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == nb - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

// The step's winner: the lowest row index among the candidates whose score
// reaches the tie window of the step's best, picked and recorded as point
// l.  Returns (row << 32 | ordered position) to all threads, ~0 if no
// candidate qualifies (then nothing is recorded).
HY_DEV unsigned long long pick_winner(const double* __restrict__ scores,
                                      const int* __restrict__ ord, const int* __restrict__ cand,
                                      OdCtl* ctl, double tie_tol, int l, int* __restrict__ pts,
                                      unsigned char* __restrict__ picked) {
  const double lim = bitsd(*(volatile unsigned long long*)&ctl->smax) * (1.0 - tie_tol);
  const int nc = *(volatile int*)&ctl->ncand;
  unsigned long long best = ~0ull;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const int pos = cand[k];
    const double sc = scores[pos];
    if (sc >= 0.0 && sc >= lim) {
      const unsigned long long key = ((unsigned long long)(unsigned)ord[pos] << 32) | (unsigned)pos;
      best = key < best ? key : best;
    }
  }
  best = block_min_u64(best);
  if (threadIdx.x == 0 && best != ~0ull) {
    const int p = (int)(best >> 32);
    pts[l] = p;
    picked[p] = 1;
    ctl->argmin = p;
  }
  return best;
}

// Several points of one pass (the cheaper variant): nbp rounds of the
// single pick over the same exact scores, each excluding the rows picked
// before it (the best of the rest, its tie window, the lowest row in the
// window).  Points l, l + 1, ... are recorded, their ordered positions in
// pick_pos[0..) and their count in pick_pos[16].  Returns the first pick's
// key (row << 32 | position), ~0 if none.
HY_DEV unsigned long long pick_several(const double* __restrict__ scores,
                                       const int* __restrict__ ord, const int* __restrict__ cand,
                                       OdCtl* ctl, double tie_tol, int l, int nbp,
                                       int* __restrict__ pts, unsigned char* __restrict__ picked,
                                       int* __restrict__ pick_pos) {
  const int nc = *(volatile int*)&ctl->ncand;
  unsigned long long first = ~0ull;
  int got = 0;
  for (int r = 0; r < nbp; ++r) {
    // keys 1 + bits of a score >= 0 (ordered like the score), 0 for none
    unsigned long long mx = 0ull;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      const int pos = cand[k];
      const double sc = scores[pos];
      if (sc >= 0.0 && !picked[ord[pos]]) {
        const unsigned long long b = sc > 0.0 ? dbits(sc) + 1ull : 1ull;
        mx = b > mx ? b : mx;
      }
    }
    mx = block_max_u64(mx);
    if (mx == 0ull) break;
    const double lim = (mx > 1ull ? bitsd(mx - 1ull) : 0.0) * (1.0 - tie_tol);
    unsigned long long best = ~0ull;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      const int pos = cand[k];
      const double sc = scores[pos];
      if (sc >= 0.0 && sc >= lim && !picked[ord[pos]]) {
        const unsigned long long key = ((unsigned long long)(unsigned)ord[pos] << 32) | (unsigned)pos;
        best = key < best ? key : best;
      }
    }
    best = block_min_u64(best);
    if (best == ~0ull) break;
    if (threadIdx.x == 0) {
      const int p = (int)(best >> 32);
      pts[l + r] = p;
      picked[p] = 1;
      pick_pos[r] = (int)(best & 0xffffffffull);
      if (r == 0) ctl->argmin = p;
    }
    if (r == 0) first = best;
    ++got;
    __syncthreads();
  }
  if (threadIdx.x == 0) pick_pos[16] = got;
  __syncthreads();
  return first;
}

// DEIM residual |r_i| of column l for ordered position pos (-1: picked),
// by the four lanes of a quad (lane c = threadIdx.x % 4 sums the terms
// j = c mod 4; an FP64 instruction holds its SM sub-partition for 64 cycles
// whatever the number of active lanes, so the row's terms are spread over
// lanes, and rows over more warps).  All four lanes return the score.
template <typename T>
HY_DEV double deim_score(const T* __restrict__ phi, int64_t N, int l, const double* cs,
                         const int* __restrict__ ord, const unsigned char* __restrict__ picked,
                         int pos, const float* __restrict__ R, int C) {
  const int c = threadIdx.x & 3;
  const int i = ord[pos];
  const bool row = sizeof(T) == 4 && pos < C;  // the copy holds the FP32 values exactly
  const float* rr = R + (int64_t)(row ? pos : 0) * 64;
  auto x = [&](int j) { return row ? (double)rr[j] : (double)phi[(int64_t)j * N + i]; };
  double sc = 0.0;
  for (int j = c; j < l; j += 4) sc = fma(x(j), cs[j], sc);
  sc = sc + __shfl_xor_sync(0xffffffffu, sc, 1);  // (s0 + s1), (s2 + s3)
  sc = sc + __shfl_xor_sync(0xffffffffu, sc, 2);
  return picked[i] ? -1.0 : fabs(x(l) - sc);
}

// DEIM step l, pass 1: exact |r_i| of the probe rows (the largest-norm
// ordered rows [0, probe), a quad of lanes per row, 16 rows per CTA of 64
// threads so that they spread over the SMs); the CTA that finishes last sets the rows still
// to score: |r_i| <= |phi_i| sqrt(1 + |c|^2), so only rows with
// |phi_i|^2 >= lim^2 / (1 + |c|^2) can reach the tie window of the best.
template <typename T>
__global__ void __launch_bounds__(256) k_deim_probe(
    const T* __restrict__ phi, int64_t N, int l, const double* __restrict__ cvec,
    const int* __restrict__ ord, const unsigned char* __restrict__ picked, int probe,
    const unsigned int* __restrict__ bmax, const int* __restrict__ bstart, double tie_tol,
    OdCtl* ctl, double* __restrict__ scores, int* __restrict__ cand, const float* __restrict__ R,
    int C) {
  pdl_enter();
  __shared__ double cs[64];
  for (int j = threadIdx.x; j < l; j += blockDim.x) cs[j] = cvec[j];
  __syncthreads();
  unsigned long long run = 0ull;
  const int rows = blockDim.x >> 2;  // one quad per row
  for (int base = blockIdx.x * rows; base < probe; base += gridDim.x * rows) {
    const int pos = base + (threadIdx.x >> 2);
    // every lane takes part in the quad's shuffles (rows past the end
    // score row `base` again and drop it)
    const bool valid = pos < probe;
    const double s0 = deim_score<T>(phi, N, l, cs, ord, picked, valid ? pos : base, R, C);
    double sc = -1.0;
    if (valid && (threadIdx.x & 3) == 0) {
      sc = s0;
      scores[pos] = sc;
    }
    note_scores(sc, pos, tie_tol, run, ctl, cand);
  }
  if (!last_block(&ctl->ticket, gridDim.x)) return;
  const double s = bitsd(*(volatile unsigned long long*)&ctl->smax);
  const double lim = s * (1.0 - 2.0 * tie_tol);
  const double cn2 = l == 0 ? 1.0 : ctl->cn2;
  const int n = plan_end(bmax, bstart, probe, lim * lim / (cn2 * (1.0 + 1e-5)));
  if (threadIdx.x == 0) {
    ctl->n_c = n;
    ctl->ticket = 0u;
    ctl->stat[0] += (unsigned long long)(n - probe);
  }
}

// DEIM step l, pass 2: the rows [probe, n_c); the CTA that finishes last
// picks point l and, for l + 1 < m, borders the factors with it and forms
// the coefficients of step l + 1.
//
// With A_l = P^T Phi[:, :l] = L U (rows in pick order; the DEIM picks are
// the partial-pivoting order of A_l, so no pivoting is needed) the CTA keeps
// the inverses Li = L^{-1} and Ui = U^{-1} (64 x 64 row-major):
//   step coefficients   y = Li b, c = Ui y      (b = Phi[P, l])
//   new point p         ell = Ui^T a (a = Phi[p, :l]), beta = Phi[p, l] - ell . y,
//                       Li row l = [-ell^T Li, 1], Ui column l = [-c / beta; 1 / beta]
// (Ui y = c).  Each product is a 64 x 64 matrix-vector product spread over
// the CTA's eight warps, in place of the dependent chains of forward and
// back substitution (an FP64 instruction holds its SM sub-partition for 64
// cycles, so those chains cost more than all the scoring).
HY_DEV void matvec_part(const double* __restrict__ A, bool trans, const double* x, int k0, int k1,
                        int n, double (*part)[64]) {
  // part[h][r] = sum over k in the h-th quarter of [k0, k1) of A(r, k) x_k
  // (A(r, k) = A[r * 64 + k], or A[k * 64 + r] when trans), r < n
  const int r = threadIdx.x & 63, h = threadIdx.x >> 6;
  const int len = (k1 - k0 + 3) / 4, a0 = k0 + h * len, a1 = a0 + len < k1 ? a0 + len : k1;
  double p0 = 0.0, p1 = 0.0;
  if (r < n) {
    int k = a0;
    for (; k + 1 < a1; k += 2) {
      p0 = fma(trans ? A[k * 64 + r] : A[r * 64 + k], x[k], p0);
      p1 = fma(trans ? A[(k + 1) * 64 + r] : A[r * 64 + k + 1], x[k + 1], p1);
    }
    if (k < a1) p0 = fma(trans ? A[k * 64 + r] : A[r * 64 + k], x[k], p0);
  }
  part[h][r] = p0 + p1;
}

template <typename T>
__global__ void __launch_bounds__(256) k_deim_rest(
    const T* __restrict__ phi, int64_t N, int l, int m, const double* __restrict__ cvec_in,
    const int* __restrict__ ord, unsigned char* __restrict__ picked, int probe, double tie_tol,
    OdCtl* ctl, double* __restrict__ scores, int* __restrict__ cand, const float* __restrict__ R,
    int C, int* __restrict__ pts, double* __restrict__ Li, double* __restrict__ Ui,
    double* __restrict__ yv, double* __restrict__ cvec) {
  pdl_enter();
  __shared__ double cs[64];
  for (int j = threadIdx.x; j < l; j += blockDim.x) cs[j] = cvec_in[j];
  __syncthreads();
  const int end = ctl->n_c;
  unsigned long long run = ctl->smax;
  const int rows = blockDim.x >> 2;  // one quad per row
  for (int base = probe + blockIdx.x * rows; base < end; base += gridDim.x * rows) {
    const int pos = base + (threadIdx.x >> 2);
    // every lane takes part in the quad's shuffles (rows past the end
    // score row `base` again and drop it)
    const bool valid = pos < end;
    const double s0 = deim_score<T>(phi, N, l, cs, ord, picked, valid ? pos : base, R, C);
    double sc = -1.0;
    if (valid && (threadIdx.x & 3) == 0) {
      sc = s0;
      scores[pos] = sc;
    }
    note_scores(sc, pos, tie_tol, run, ctl, cand);
  }
  if (!last_block(&ctl->ticket, gridDim.x)) return;
  // ---- the pick, then the factors of step l + 1 (this CTA alone) ----
  const int tid = threadIdx.x;
  const unsigned long long key = pick_winner(scores, ord, cand, ctl, tie_tol, l, pts, picked);
  const int p = (int)(key >> 32), wpos = (int)(key & 0xffffffffull);
  __shared__ double a[64], ell[64], y[64], b[64], c[64];
  __shared__ double part[4][64];
  __shared__ double beta_s;
  if (l + 1 < m && key != ~0ull) {
    // a = Phi[p, :l], its entry l, y and c of step l
    if (tid <= l) a[tid] = phi_at<T>(phi, N, tid, p, wpos, R, C);
    if (tid < l) {
      y[tid] = yv[tid];
      c[tid] = cvec_in[tid];
    }
    __syncthreads();
    // ell = Ui^T a: ell_k = sum_{r <= k} Ui[r][k] a_r
    matvec_part(Ui, true, a, 0, l, l, part);
    __syncthreads();
    if (tid < l) ell[tid] = (part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]);
    __syncthreads();
    double dot = tid < l ? ell[tid] * y[tid] : 0.0;
    dot = block_sum(dot);
    if (tid == 0) beta_s = a[l] - dot;
    // Li row l = -ell^T Li (Li lower triangular)
    matvec_part(Li, true, ell, 0, l, l, part);
    __syncthreads();
    const double beta = beta_s;
    const double ib = 1.0 / beta;
    if (tid < l) {
      Li[l * 64 + tid] = -((part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]));
      Ui[tid * 64 + l] = -c[tid] * ib;
    }
    if (tid == 0) {
      Li[l * 64 + l] = 1.0;
      Ui[l * 64 + l] = ib;
    }
    // step l + 1: b = Phi[P, l + 1] over the l + 1 points
    const int k = l + 1;
    if (tid < k) b[tid] = (double)phi[(int64_t)k * N + pts[tid]];
    __syncthreads();
    // y = Li b (rows r < k; Li lower triangular, zero beyond the diagonal)
    matvec_part(Li, false, b, 0, k, k, part);
    __syncthreads();
    if (tid < k) y[tid] = (part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]);
    __syncthreads();
    // c = Ui y
    matvec_part(Ui, false, y, 0, k, k, part);
    __syncthreads();
    double cn = 0.0;
    if (tid < k) {
      const double ci = (part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]);
      cvec[tid] = ci;
      yv[tid] = y[tid];
      cn = ci * ci;
    }
    cn = block_sum(cn);
    if (tid == 0) ctl->cn2 = 1.0 + cn;
  }
  if (tid == 0) {
    ctl->smax = 0ull;
    ctl->ncand = 0;
    ctl->ticket = 0u;
    ctl->n_c = 0;
  }
}

// ---- ODEIM oversampling -----------------------------------------------------

// M = A^T A over the first l points (m x m, FP64)
template <typename T>
__global__ void __launch_bounds__(256) k_odeim_gram(const T* __restrict__ phi, int64_t N, int m,
                                                    const int* __restrict__ pts, int l,
                                                    double* __restrict__ M) {
  // M = A^T A, A = the l sampled rows of Phi (l x m): every CTA stages A in
  // shared memory (eight loads in flight per thread), CTA c forms the rows
  // a = c, c + G, ... of M, one entry per thread, four chains over the l
  // terms (fma(x, y) = fma(y, x), so M is exactly symmetric)
  __shared__ double A[64][65];
  const int tid = threadIdx.x;
  for (int base = tid; base < l * m; base += blockDim.x * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      const int r = idx / m, a = idx - r * m;
      v[u] = idx < l * m ? (double)phi[(int64_t)a * N + pts[r]] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < l * m) A[idx / m][idx % m] = v[u];
    }
  }
  __syncthreads();
  for (int e = tid; e < 4 * 64; e += blockDim.x) {
    const int a = blockIdx.x + gridDim.x * (e >> 6), b = e & 63;
    if (a >= m || b >= m) continue;
    double p4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r = 0; r < l; ++r) p4[r & 3] = fma(A[r][a], A[r][b], p4[r & 3]);
    M[a * m + b] = (p4[0] + p4[1]) + (p4[2] + p4[3]);
  }
}

// sort the Jacobi eigenpairs ascending: lam_s, W_s (m x m column-major);
// reset the step's control block
// The screens read the eigensystem in FP32, written once per step where it
// changes: wt32[a * 64 + j] = W_ja (zero for j >= m), then dn[64], du[64]
// and dd[64] at wt32 + 4096: d_j = lam_j - lam_1 (sorted) rounded to
// nearest, upward and downward for 1 <= j < m, +inf otherwise (slot 0
// carries z_1 itself); en, eu, ed: e_j = lam_j - lam_2 likewise for j < m
// (+inf beyond; e_1 < 0, e_2 = 0); d2[3]: lam_2 - lam_1.  One CTA.
HY_DEV void w32_tail(const double* __restrict__ lam_sorted, int m, float* __restrict__ wt32) {
  for (int idx = threadIdx.x; idx < m * (64 - m); idx += blockDim.x) {
    const int a = idx / (64 - m), j = m + idx % (64 - m);
    wt32[a * 64 + j] = 0.f;
  }
  float* dn = wt32 + 64 * 64;
  float* du = dn + 64;
  float* dd = du + 64;
  float* en = dd + 64;
  float* eu = en + 64;
  float* ed = eu + 64;
  float* d2 = ed + 64;
  const double l1 = lam_sorted[0];
  const double l2 = m > 1 ? lam_sorted[1] : 0.0;
  for (int j = threadIdx.x; j < 64; j += blockDim.x) {
    if (j >= 1 && j < m) {
      dn[j] = (float)(lam_sorted[j] - l1);
      du[j] = __double2float_ru(__dsub_ru(lam_sorted[j], l1));
      dd[j] = __double2float_rd(__dsub_rd(lam_sorted[j], l1));
    } else {
      dn[j] = INFINITY;
      du[j] = INFINITY;
      dd[j] = INFINITY;
    }
    if (m > 1 && j < m) {
      en[j] = (float)(lam_sorted[j] - l2);
      eu[j] = __double2float_ru(__dsub_ru(lam_sorted[j], l2));
      ed[j] = __double2float_rd(__dsub_rd(lam_sorted[j], l2));
    } else {
      en[j] = INFINITY;
      eu[j] = INFINITY;
      ed[j] = INFINITY;
    }
  }
  if (threadIdx.x == 0) {
    d2[0] = m > 1 ? (float)(l2 - l1) : INFINITY;
    d2[1] = m > 1 ? __double2float_ru(__dsub_ru(l2, l1)) : INFINITY;
    d2[2] = m > 1 ? __double2float_rd(__dsub_rd(l2, l1)) : INFINITY;
  }
}

__global__ void k_odeim_sort(const double* __restrict__ lam, const double* __restrict__ V, int n,
                             int m, double* __restrict__ lam_s, double* __restrict__ W_s,
                             OdCtl* ctl, float* __restrict__ wt32) {
  __shared__ int perm[128];
  __shared__ unsigned long long key[128];
  for (int i = threadIdx.x; i < m; i += blockDim.x) key[i] = dkey(lam[i]);
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {  // ascending rank
    int r = 0;
    for (int i = 0; i < m; ++i) r += (key[i] < key[j]) || (key[i] == key[j] && i < j);
    perm[r] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) lam_s[i] = lam[perm[i]];
    ctl->lam1 = lam[perm[0]];
    ctl->lam2 = m > 1 ? lam[perm[1]] : INFINITY;
    ctl->lmax = lam[perm[m - 1]];
    ctl->smax = 0ull;
    ctl->slo = 0ull;
    ctl->n_list = 0;
    ctl->n_x = 0;
    ctl->ncand = 0;
    ctl->ticket = 0u;
    ctl->argmin = 0x7fffffff;
    ctl->n_c = 0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int j = idx / m, a = idx % m;
    const double v = V[(int64_t)perm[j] * n + a];
    W_s[idx] = v;
    wt32[a * 64 + j] = (float)v;
  }
  w32_tail(lam_s, m, wt32);
}

// Smallest root mu of the secular equation
//   f(mu) = 1 + sum_j z_j^2 / (lam_j - mu)   (lam ascending, m <= 64),
// i.e. lambda_min(diag(lam) + z z^T), one warp (lane: terms j = lane and
// lane + 32; z and lam in shared memory).  The root lies in (lam_1, lam_2).
// It is found in coordinates shifted to the nearer of the two poles (the
// sign of f at their midpoint tells which), mu = lam_o + t, so that both
// t and every lam_j - mu keep full relative accuracy; the steps solve the
// two-pole model of f ("middle way" of Li's secular-equation solver, as in
// LAPACK's dlaed4): with psi the term of pole 1 and phi the others,
//   f ~ c + s / (del_1 - t') + S / (del_2 - t'),
//   s = psi' (del_1 - t)^2, S = phi' (del_2 - t)^2,
//   c = f - psi' (del_1 - t) - phi' (del_2 - t),
// a quadratic whose root in the interval is taken; steps stay inside a
// shrinking bracket (bisection otherwise).  FP32 steps first (an FP64
// instruction holds its SM sub-partition for 64 cycles), then FP64 steps
// until |f| is within the rounding error of its evaluation, the step is
// below 2 ulp, or the bracket has collapsed.  The greedy's best rows lift
// lambda_min to just below lam_2, where a root in unshifted coordinates
// took about seven FP64 steps (the poles' differences lost their digits);
// shifted, it takes two.  Special cases: m = 1 (mu = lam_1 + z_1^2), and
// z_1 = 0 or lam_1 = lam_2 (mu = lam_1: no eigenvalue falls below it).
__device__ double secular_root_warp(const double* __restrict__ z, const double* __restrict__ lam,
                                    int m, double l1, double l2) {
  const int lane = threadIdx.x & 31;
  double dv[2], z2[2];
  for (int u = 0; u < 2; ++u) {
    const int i = lane + 32 * u;
    dv[u] = i < m ? lam[i] : 0.0;
    const double zi = i < m ? z[i] : 0.0;
    z2[u] = zi * zi;
  }
  const double zf = __shfl_sync(0xffffffffu, z2[0], 0);  // z_1^2
  if (m == 1) return l1 + zf;
  if (zf == 0.0 || !(l2 > l1)) return l1;
  const double mid = 0.5 * (l1 + l2);
  double f = 0.0;
  for (int u = 0; u < 2; ++u)
    if (lane + 32 * u < m) f = f + z2[u] / (dv[u] - mid);
  f = 1.0 + warp_sum(f);
  const bool left = f >= 0.0;  // the root lies in (lam_1, mid]
  const double dorg = left ? l1 : l2;
  double lo = left ? 0.0 : mid - l2, hi = left ? mid - l1 : 0.0;
  double del[2];
  for (int u = 0; u < 2; ++u) del[u] = dv[u] - dorg;
  const double delj = l1 - dorg, deln = l2 - dorg;
  double t = left ? 0.5 * hi : 0.5 * lo;
  const double eps = 2.220446049250313e-16;
  {  // FP32 model steps to a start for the FP64 ones, which keep their own bracket
    const float fe = 1.1920929e-7f;
    float fdel[2], fz2[2];
    for (int u = 0; u < 2; ++u) {
      fdel[u] = (float)del[u];
      fz2[u] = (float)z2[u];
    }
    const float fdelj = (float)delj, fdeln = (float)deln;
    float ft = (float)t, flo = (float)lo, fhi = (float)hi;
    for (int it = 0; it < 16; ++it) {
      float ff = 0.f, fa = 0.f, dps = 0.f, dph = 0.f;
      for (int u = 0; u < 2; ++u) {
        const int i = lane + 32 * u;
        if (i < m) {
          const float r = __frcp_rn(fdel[u] - ft);
          const float q = fz2[u] * r;
          ff += q;
          fa += fabsf(q);
          if (i == 0)
            dps = fmaf(q, r, dps);
          else
            dph = fmaf(q, r, dph);
        }
      }
      ff = 1.f + warp_sum(ff);
      fa = warp_sum(fa);
      dps = warp_sum(dps);
      dph = warp_sum(dph);
      if (fabsf(ff) <= 8.f * fe * (1.f + fa + fabsf(ft) * (dps + dph))) break;
      if (ff < 0.f)
        flo = ft;
      else
        fhi = ft;
      if (fhi - flo <= 2.f * fe * fmaxf(fabsf(fhi), fabsf(flo))) {
        ft = 0.5f * (flo + fhi);
        break;
      }
      const float Dj = fdelj - ft, Dn = fdeln - ft;
      const float sL = dps * Dj * Dj, sR = dph * Dn * Dn;
      const float A = ff - dps * Dj - dph * Dn;
      const float B = A * (Dj + Dn) + sL + sR;
      const float Cq = ff * Dj * Dn;
      float eta = NAN;
      if (A == 0.f) {
        if (B != 0.f) eta = __fdividef(Cq, B);
      } else {
        const float qq = 0.5f * (B + copysignf(fsqrt_fast(fmaxf(B * B - 4.f * A * Cq, 0.f)), B));
        const float e1 = __fdividef(qq, A), e2 = qq != 0.f ? __fdividef(Cq, qq) : NAN;
        if (e1 > Dj && e1 < Dn) eta = e1;
        if (e2 > Dj && e2 < Dn) eta = e2;
      }
      float nt = ft + eta;
      if (fabsf(nt - ft) <= 2.f * fe * fabsf(ft)) {
        ft = nt;
        break;
      }
      if (!(nt > flo && nt < fhi)) nt = 0.5f * (flo + fhi);
      ft = nt;
    }
    const double tc = (double)ft;
    if (tc > lo && tc < hi) t = tc;
  }
  for (int it = 0; it < 100; ++it) {
    double ff = 0.0, fa = 0.0, dps = 0.0, dph = 0.0;
    for (int u = 0; u < 2; ++u) {
      const int i = lane + 32 * u;
      if (i < m) {
        const double r = 1.0 / (del[u] - t);
        const double q = z2[u] * r;
        ff = ff + q;
        fa = fa + fabs(q);
        if (i == 0)
          dps = dps + q * r;
        else
          dph = dph + q * r;
      }
    }
    ff = 1.0 + warp_sum(ff);
    fa = warp_sum(fa);
    dps = warp_sum(dps);
    dph = warp_sum(dph);
    if (fabs(ff) <= 8.0 * eps * (1.0 + fa + fabs(t) * (dps + dph))) break;
    if (ff < 0.0)
      lo = t;
    else
      hi = t;
    if (hi - lo <= 2.0 * eps * fmax(fabs(hi), fabs(lo))) {
      t = 0.5 * (lo + hi);
      break;
    }
    const double Dj = delj - t, Dn = deln - t;
    const double sL = dps * Dj * Dj, sR = dph * Dn * Dn;
    const double A = ff - dps * Dj - dph * Dn;
    const double B = A * (Dj + Dn) + sL + sR;
    const double Cq = ff * Dj * Dn;
    double eta = NAN;  // A eta^2 - B eta + Cq = 0: the root in (Dj, Dn)
    if (A == 0.0) {
      if (B != 0.0) eta = Cq / B;
    } else {
      const double q = 0.5 * (B + copysign(sqrt(fmax(B * B - 4.0 * A * Cq, 0.0)), B));
      const double e1 = q / A, e2 = q != 0.0 ? Cq / q : NAN;
      if (e1 > Dj && e1 < Dn) eta = e1;
      if (e2 > Dj && e2 < Dn) eta = e2;
    }
    double nt = t + eta;
    if (fabs(nt - t) <= 2.0 * eps * fabs(t)) {  // before the bracket test: a
      t = nt;                                    // converged step may sit on it
      break;
    }
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    t = nt;
  }
  return dorg + t;
}

// z = W^T rb for the m x m eigenvector block W (column j at W + j ldw) by the
// whole CTA (blockDim a multiple of 64): thread t forms component t % 64 over
// one of blockDim / 64 contiguous parts of the m terms (four chains), the
// parts are then added in a fixed order.  A warp-wide FP64 instruction
// occupies an SM sub-partition for 64 cycles, so the 64 x 64 product is
// spread over all the CTA's warps.  Synchronises the CTA on entry and exit.
HY_DEV void z_block(const double* W, int ldw, const double* rb, int m, double* zp, double* z) {
  const int t = threadIdx.x, j = t & 63, h = t >> 6, parts = blockDim.x >> 6;
  const int len = (m + parts - 1) / parts;
  const int a0 = h * len, a1 = a0 + len < m ? a0 + len : m;
  __syncthreads();
  double p[4] = {0.0, 0.0, 0.0, 0.0};
  if (j < m) {
    const double* w = W + j * ldw;
    int a = a0;
    for (; a + 3 < a1; a += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) p[u] = fma(w[a + u], rb[a + u], p[u]);
    }
    for (; a < a1; ++a) p[0] = fma(w[a], rb[a], p[0]);
  }
  zp[h * 64 + j] = (p[0] + p[1]) + (p[2] + p[3]);
  __syncthreads();
  if (t < 64) {
    double sm = 0.0;
    for (int q = 0; q < parts; ++q) sm += zp[q * 64 + t];
    z[t] = t < m ? sm : 0.0;
  }
  __syncthreads();
}

// ---- ODEIM scoring: certified FP32 bounds, then exact FP64 scores ---------
//
// With z = W^T phi, d_j = l_j - l1 and mu = l1 + tau, tau is the root in
// [0, d_2) of the increasing function
//   h(tau) = tau (1 + sum_{j>=2} z_j^2 / (d_j - tau)) - z_1^2,
// so tau <= z_1^2 and tau <= d_2 (interlacing).  FP32 dot products of m <= 64
// terms on operands rounded to FP32 are within dl = 8e-6 |phi| of the exact
// components ((m + 2) 2^-24 |W_j| |phi| = 3.9e-6 |phi|; the factor 2 covers
// the rounding of the stored norm), so with b1 = |z~_1| + dl and
// a_j = max(|z~_j| - dl, 0) the function
//   h_L(t) = t (1 + sum_{j>=2} a_j^2 / (d_j - t)) - b1^2  <=  h(t),
// and h_L(t) >= 0 proves tau <= t: an upper bound U of the exact score.
// Symmetrically, with B1 = max(|z~_1| - dl, 0), A_j = |z~_j| + dl and the
// poles rounded down,
//   h_U(t) = t (1 + sum_{j>=2} A_j^2 / (d_j - t)) - B1^2  >=  h(t),
// and h_U(t) <= 0 proves tau >= t: a lower bound L.  Every bound is
// evaluated with directed rounding.  The largest L found raises the step's
// pruning limit before any exact score is known.
//
// A step's rows are taken in three passes: the probe rows (the largest
// norms) get both bounds, and the exact score of the row with the best U;
// the rows whose norm can still reach the limit get the bound from z_1
// alone, and those it does not exclude both full bounds; the rows whose U
// reaches the limit get the exact score.  The last pass also picks the point
// and prepares the eigensystem update.


// stage a CTA's copy of W (m x m, column j = eigenvector j) with an odd
// leading dimension, and the eigenvalues
HY_DEV void stage_w(const double* __restrict__ W_s, const double* __restrict__ lam_s, int m,
                    double* W, double* lam) {
  for (int base = threadIdx.x; base < m * m; base += blockDim.x * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * blockDim.x;
      v[u] = i < m * m ? W_s[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * blockDim.x;
      if (i < m * m) {
        const int j = i / m, a = i - j * m;
        W[j * kLdw + a] = v[u];
      }
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = lam_s[i];
}

HY_DEV double limit_of(const OdCtl* ctl, double tie_tol) {
  const unsigned long long a = *(const volatile unsigned long long*)&ctl->smax;
  const unsigned long long b = *(const volatile unsigned long long*)&ctl->slo;
  return bitsd(a > b ? a : b) * (1.0 - 2.0 * tie_tol);
}

// Pass 2a, one thread per ordered row in [probe, n_c): bounds from z_1 and
// z_2 alone (two m-term dot products): U1 = min(l1 + b1^2, l2), and, below
// l2, l2 - s for the s at which the two-term secular function
//   f2(s) = 1 + z_2^2 / s - z_1^2 / (d2 - s)
// is certified non-negative (the true f has further positive terms, so
// f(s) >= f2(s) >= 0 and sigma >= s; s from f2's root less a margin for the
// FP32 errors of z).  Rows whose bound reaches the limit are appended to
// `list` for pass 2b.
template <typename T>
HY_DEV void odeim_z1_body(int bid, int nb,
    const T* __restrict__ phi, int64_t N, int m, const float* __restrict__ wt32,
    const float* __restrict__ nrm, const int* __restrict__ ord,
    const unsigned char* __restrict__ picked, int p0, double tie_tol, OdCtl* ctl,
    double* __restrict__ scores, int* __restrict__ list, const float* __restrict__ R, int C) {
  pdl_enter();
  __shared__ float w1[64], w2[64];
  for (int a = threadIdx.x; a < 64; a += blockDim.x) {
    w1[a] = a < m ? wt32[a * 64] : 0.f;
    w2[a] = a < m && m > 1 ? wt32[a * 64 + 1] : 0.f;
  }
  __syncthreads();
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  const double lim = limit_of(ctl, tie_tol);
  const int end = ctl->n_c;
  const int lane = threadIdx.x & 31;
  const float d2n = wt32[4096 + 384], d2d = wt32[4096 + 384 + 2];
  for (int base = p0 + bid * blockDim.x; base < end; base += nb * blockDim.x) {
    const int pos = base + threadIdx.x;
    bool pass = false;
    if (pos < end) {
      const int i = ord[pos];
      double U = -1.0;
      if (!picked[i]) {
        float z1 = 0.f, z2 = 0.f;
        if (pos < C) {  // contiguous copy (zero beyond m: the m columns suffice)
          const float4* rp = reinterpret_cast<const float4*>(R + (int64_t)pos * 64);
          auto term = [&](const float4 v, int q) {
            z1 = fmaf(w1[4 * q], v.x, z1);
            z1 = fmaf(w1[4 * q + 1], v.y, z1);
            z1 = fmaf(w1[4 * q + 2], v.z, z1);
            z1 = fmaf(w1[4 * q + 3], v.w, z1);
            z2 = fmaf(w2[4 * q], v.x, z2);
            z2 = fmaf(w2[4 * q + 1], v.y, z2);
            z2 = fmaf(w2[4 * q + 2], v.z, z2);
            z2 = fmaf(w2[4 * q + 3], v.w, z2);
          };
          const int nq = (m + 3) >> 2;
          if (nq == 16) {  // all 16 loads in flight at once
#pragma unroll
            for (int q = 0; q < 16; ++q) term(rp[q], q);
          } else {
#pragma unroll 4
            for (int q = 0; q < nq; ++q) term(rp[q], q);
          }
        } else {
          for (int a = 0; a < m; ++a) {
            const float x = (float)phi[(int64_t)a * N + i];
            z1 = fmaf(w1[a], x, z1);
            z2 = fmaf(w2[a], x, z2);
          }
        }
        const float dl = __fmul_ru(8e-6f, __fsqrt_ru(nrm[i]));
        const float b1 = __fadd_ru(fabsf(z1), dl);
        const float bh = __fmul_ru(b1, b1);
        U = fmin(__dadd_ru(l1, (double)bh), l2);
        const float al = fmaxf(__fsub_rd(fabsf(z2), dl), 0.f);
        if (m > 1 && d2n > 0.f && al > 0.f) {
          const float a = z2 * z2, b = z1 * z1, p = d2n - a - b;
          const float rt = fsqrt_fast(fmaf(p, p, 4.f * a * d2n));
          const float s0 = p >= 0.f ? 0.5f * (p + rt) : __fdividef(2.f * a * d2n, rt - p);
          const float kap = fminf(__fdividef(6.f * dl, fmaxf(fabsf(z2), 1e-30f)) +
                                      __fdividef(6.f * dl, fmaxf(fabsf(z1), 1e-30f)) +
                                      1.0f / 32768.f,
                                  0.75f);
          const float sl = __fmul_rd(s0, 1.f - kap);
          if (sl > 0.f && sl < d2d) {
            const float ta = __fmul_rd(__fmul_rd(al, al), __frcp_rd(sl));
            const float tb = __fmul_ru(bh, __frcp_ru(__fsub_rd(d2d, sl)));
            if (__fsub_rd(__fadd_rd(1.f, ta), tb) >= 0.f) U = fmin(U, __dsub_ru(l2, (double)sl));
          }
        }
        pass = U >= lim;
      }
      scores[pos] = U;
    }
    // warp-aggregated append
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    if (bal) {
      int first = 0;
      if (lane == 0) first = atomicAdd(&ctl->n_list, __popc(bal));
      first = __shfl_sync(0xffffffffu, first, 0);
      if (pass) list[first + __popc(bal & ((1u << lane) - 1u))] = pos;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_odeim_z1(
    const T* __restrict__ phi, int64_t N, int m, const float* __restrict__ wt32,
    const float* __restrict__ nrm, const int* __restrict__ ord,
    const unsigned char* __restrict__ picked, int p0, double tie_tol, OdCtl* ctl,
    double* __restrict__ scores, int* __restrict__ list, const float* __restrict__ R, int C) {
  odeim_z1_body<T>(blockIdx.x, gridDim.x, phi, N, m, wt32, nrm, ord, picked, p0, tie_tol, ctl,
                   scores, list, R, C);
}

// ---- certified bounds, eight lanes per row ----------------------------------
//
// The probe pass and the full-bound pass take their rows in tiles of kTile
// rows per CTA of kTile * kGrp threads: the tile's rows are gathered
// (row-major FP32, 256 contiguous bytes each) into shared memory, z = W^T phi
// of every row is formed as a small matrix product (thread: one row, eight
// components), and then the kGrp lanes of a row certify its bounds, lane g
// taking the components j = g mod kGrp and the sums closing with three
// shuffles.  A warp per row spent most of its time in five-level shuffle
// sums; a thread per row in long dependent chains.

constexpr int kTile = 32;        // rows per CTA
constexpr int kGrp = 8;          // lanes per row
constexpr int kTileThreads = kTile * kGrp;
constexpr int kTileLd = 65;      // odd row stride of the tile in shared memory

struct TileSm {
  float Wt[64][64];
  float dn[64], du[64], dd[64];
  float en[64], eu[64], ed[64], d2[4];
  float zt[kTile * kTileLd];     // the rows, then their z
  int pos[kTile], row[kTile];
  float nrm[kTile];
};

HY_DEV void stage_tile_tables(const float* __restrict__ wt32, int m, TileSm& S) {
  const float4* src = reinterpret_cast<const float4*>(wt32);
  float4* dst = reinterpret_cast<float4*>(&S.Wt[0][0]);
  for (int i = threadIdx.x; i < m * 16; i += blockDim.x) dst[i] = src[i];
  for (int j = threadIdx.x; j < 64; j += blockDim.x) {
    S.dn[j] = wt32[4096 + j];
    S.du[j] = wt32[4096 + 64 + j];
    S.dd[j] = wt32[4096 + 128 + j];
    S.en[j] = wt32[4096 + 192 + j];
    S.eu[j] = wt32[4096 + 256 + j];
    S.ed[j] = wt32[4096 + 320 + j];
  }
  if (threadIdx.x < 3) S.d2[threadIdx.x] = wt32[4096 + 384 + threadIdx.x];
}

// The tile's rows (S.pos[r] >= 0; -1: no row) into S.zt, then their z in
// place (zero beyond m).  blockDim.x == kTileThreads.
template <typename T>
HY_DEV void tile_z(const T* __restrict__ phi, int64_t N, int m, const float* __restrict__ R,
                   int C, TileSm& S) {
  const int t = threadIdx.x;
  for (int idx = t; idx < kTile * 16; idx += kTileThreads) {  // float4 k of row r
    const int r = idx >> 4, k = idx & 15;
    const int pos = S.pos[r];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pos >= 0 && 4 * k < m) {  // (the product below reads the first m only)
      if (pos < C) {
        v = reinterpret_cast<const float4*>(R + (int64_t)pos * 64)[k];
      } else {
        const int i = S.row[r];
        const int a = 4 * k;
        v.x = a < m ? (float)phi[(int64_t)a * N + i] : 0.f;
        v.y = a + 1 < m ? (float)phi[(int64_t)(a + 1) * N + i] : 0.f;
        v.z = a + 2 < m ? (float)phi[(int64_t)(a + 2) * N + i] : 0.f;
        v.w = a + 3 < m ? (float)phi[(int64_t)(a + 3) * N + i] : 0.f;
      }
    }
    float* d = S.zt + r * kTileLd + 4 * k;
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
  }
  __syncthreads();
  const int r = t / kGrp, c0 = (t % kGrp) * 8;
  float acc[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) acc[v] = 0.f;
  for (int a = 0; a < m; ++a) {
    const float x = S.zt[r * kTileLd + a];
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[v] = fmaf(S.Wt[a][c0 + v], x, acc[v]);
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < 8; ++v) S.zt[r * kTileLd + c0 + v] = c0 + v < m ? acc[v] : 0.f;
  __syncthreads();
}

// Sums over a row's kGrp lanes (mask: the group's lanes); the group's first
// lane's result is given to all, so that every lane takes the same branches.
HY_DEV float grp_sum(float v, unsigned mask, int base) {
#pragma unroll
  for (int o = kGrp / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return __shfl_sync(mask, v, base);
}
HY_DEV float grp_sum_rd(float v, unsigned mask, int base) {
#pragma unroll
  for (int o = kGrp / 2; o > 0; o >>= 1) v = __fadd_rd(v, __shfl_xor_sync(mask, v, o));
  return __shfl_sync(mask, v, base);
}
HY_DEV float grp_sum_ru(float v, unsigned mask, int base) {
#pragma unroll
  for (int o = kGrp / 2; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(mask, v, o));
  return __shfl_sync(mask, v, base);
}

// Both certified bounds, U >= mu >= L, of one row from its FP32 z (zr, m
// values) and squared-norm bound, by one thread.  The root is approached in
// the coordinates of the nearer pole (the sign of the secular function at
// the midpoint of (l1, l2) tells which): tau = mu - l1 as above, or
// sigma = l2 - mu, where
//   f(sigma) = 1 + sum_j z_j^2 / (e_j + sigma),  e_j = lam_j - l2,
// is decreasing on (0, l2 - l1) (the j = 1 term is the negative one), so a
// certified lower bound f_lo(s) >= 0 proves sigma >= s (mu <= l2 - s) and a
// certified upper bound f_hi(s) <= 0 proves sigma <= s.  The greedy's best
// rows lift lambda_min to just below l2, where only these coordinates
// resolve sigma: in tau the bounds would stop at l2 itself.  sigma scales
// with z_2^2 (and z_1^2), whose FP32 errors are about 2 dl / |z_2| and
// 2 dl / |z_1| relative: the first margin tried is three times that.
HY_DEV void bounds_row(const TileSm& S, int m, double l1, double l2, const float* zr,
                       float nrm_i, unsigned mask, int base, int g, double& U, double& L) {
  const float dl = __fmul_ru(8e-6f, __fsqrt_ru(nrm_i));
  const float zf = zr[0];
  const float b1 = __fadd_ru(fabsf(zf), dl);
  const float b1s = __fmul_ru(b1, b1);
  const float B1 = fmaxf(__fsub_rd(fabsf(zf), dl), 0.f);
  const float B1s = __fmul_rd(B1, B1);
  U = fmin(__dadd_ru(l1, (double)b1s), l2);
  L = l1;
  if (m == 1) {
    L = __dadd_rd(l1, (double)B1s);
    return;
  }
  const float d2n = S.dn[1], d2u = S.du[1], d2d = S.dd[1];
  if (!(d2n > 0.f)) return;  // a double eigenvalue: mu = l1
  auto alo = [&](int j) {    // z_j^2 from below
    const float x = fmaxf(__fsub_rd(fabsf(zr[j]), dl), 0.f);
    return __fmul_rd(x, x);
  };
  auto chi = [&](int j) {    // z_j^2 from above
    const float x = __fadd_ru(fabsf(zr[j]), dl);
    return __fmul_ru(x, x);
  };
  const float hm = 0.5f * d2n;
  float fm = 0.f;
  for (int j = g; j < m; j += kGrp) fm += __fdividef(zr[j] * zr[j], S.en[j] + hm);
  const float fmid = 1.f + grp_sum(fm, mask, base);
  const int j1 = g == 0 ? kGrp : g;  // this lane's first component j >= 1
  if (fmid >= 0.f) {
    // the root in (l1, mid]: tau coordinates
    float t = 0.f, lo = 0.f, hi = fminf(d2n, b1s);
    float g0 = 0.f, dg0 = 0.f;
    for (int j = j1; j < m; j += kGrp) {
      const float a = alo(j), r = __fdividef(1.f, S.dn[j]);
      g0 = fmaf(a, r, g0);
      dg0 = fmaf(a * r, r, dg0);
    }
    float gs = grp_sum(g0, mask, base), dgs = grp_sum(dg0, mask, base);
    for (int it = 0; it < 16; ++it) {
      if (it > 0) {
        float q0 = 0.f, d0 = 0.f;
        for (int j = j1; j < m; j += kGrp) {
          const float r = __frcp_rn(S.dn[j] - t);
          const float q = alo(j) * r;
          q0 += q;
          d0 = fmaf(q, r, d0);
        }
        gs = grp_sum(q0, mask, base);
        dgs = grp_sum(d0, mask, base);
        const float h = fmaf(t, 1.f + gs, -b1s);
        if (fabsf(h) <= 32.f * 1.1920929e-7f * (t * (1.f + gs) + b1s)) break;
        if (h < 0.f)
          lo = t;
        else
          hi = t;
      }
      const float gap = d2n - t;
      const float C = 1.f + (gs - dgs * gap);
      const float B = C * d2n + b1s + dgs * gap * gap;
      const float nt =
          __fdividef(2.f * b1s * d2n, B + fsqrt_fast(fmaxf(B * B - 4.f * C * b1s * d2n, 0.f)));
      if (it > 0 && fabsf(nt - t) <= 4.f * 1.1920929e-7f * t) {
        t = nt;
        break;
      }
      t = (nt > lo && nt < hi) ? nt : 0.5f * (lo + hi);
    }
    for (int tr = 0; tr < 2; ++tr) {  // h_L(t') >= 0 above the iterate
      const float tu = __fmul_ru(t, tr == 0 ? 1.f + 1.0f / 32768.f : 1.f + 1.0f / 2048.f);
      if (!(tu < d2u)) break;
      float sl = 0.f;
      for (int j = j1; j < m; j += kGrp)
        sl = __fadd_rd(sl, __fmul_rd(alo(j), __frcp_rd(__fsub_ru(S.du[j], tu))));
      const float hl = __fsub_rd(__fmul_rd(tu, __fadd_rd(1.f, grp_sum_rd(sl, mask, base))), b1s);
      if (hl >= 0.f) {
        U = fmin(U, __dadd_ru(l1, (double)tu));
        break;
      }
    }
    if (!(B1s > 0.f)) return;
    for (int tr = 0; tr < 3; ++tr) {  // h_U(t') <= 0 below the iterate
      const float td = __fmul_rd(t, tr == 0 ? 1.f - 1.0f / 32768.f
                                            : (tr == 1 ? 1.f - 1.0f / 2048.f : 1.f - 1.0f / 128.f));
      if (!(td > 0.f && td < d2d)) continue;
      float su = 0.f;
      for (int j = j1; j < m; j += kGrp)
        su = __fadd_ru(su, __fmul_ru(chi(j), __frcp_ru(__fsub_rd(S.dd[j], td))));
      const float hu = __fsub_ru(__fmul_ru(td, __fadd_ru(1.f, grp_sum_ru(su, mask, base))), B1s);
      if (hu <= 0.f) {
        L = __dadd_rd(l1, (double)td);
        return;
      }
    }
    return;
  }
  // the root in (mid, l2): sigma = -t, model steps around the poles
  // e_1 = -d2 and e_2 = 0
  const float fe = 1.1920929e-7f;
  const float fdelj = -d2n;
  float ft = -0.5f * hm, flo = -hm, fhi = 0.f;
  for (int it = 0; it < 16; ++it) {
    const float r0 = __frcp_rn(S.en[0] - ft);
    const float ql = zf * zf * r0;
    float q0 = 0.f, d0 = 0.f;
    for (int j = j1; j < m; j += kGrp) {
      const float r = __frcp_rn(S.en[j] - ft);
      const float q = zr[j] * zr[j] * r;
      q0 += q;
      d0 = fmaf(q, r, d0);
    }
    const float ff = 1.f + ql + grp_sum(q0, mask, base);
    const float dph = grp_sum(d0, mask, base);
    const float dps = ql * r0;
    const float fa = (ff - 1.f) - 2.f * ql;
    if (fabsf(ff) <= 8.f * fe * (1.f + fa + fabsf(ft) * (dps + dph))) break;
    if (ff < 0.f)
      flo = ft;
    else
      fhi = ft;
    if (fhi - flo <= 2.f * fe * fmaxf(fabsf(fhi), fabsf(flo))) {
      ft = 0.5f * (flo + fhi);
      break;
    }
    const float Dj = fdelj - ft, Dn = -ft;
    const float sL = dps * Dj * Dj, sR = dph * Dn * Dn;
    const float A = ff - dps * Dj - dph * Dn;
    const float B = A * (Dj + Dn) + sL + sR;
    const float Cq = ff * Dj * Dn;
    float eta = NAN;
    if (A == 0.f) {
      if (B != 0.f) eta = __fdividef(Cq, B);
    } else {
      const float qq = 0.5f * (B + copysignf(fsqrt_fast(fmaxf(B * B - 4.f * A * Cq, 0.f)), B));
      const float e1 = __fdividef(qq, A), e2 = qq != 0.f ? __fdividef(Cq, qq) : NAN;
      if (e1 > Dj && e1 < Dn) eta = e1;
      if (e2 > Dj && e2 < Dn) eta = e2;
    }
    float nt = ft + eta;
    if (fabsf(nt - ft) <= 2.f * fe * fabsf(ft)) {
      ft = nt;
      break;
    }
    if (!(nt > flo && nt < fhi)) nt = 0.5f * (flo + fhi);
    ft = nt;
  }
  const float sg = -ft;
  if (!(sg > 0.f)) return;
  const float kap = fminf(__fdividef(6.f * dl, fmaxf(fabsf(zr[1]), 1e-30f)) +
                              __fdividef(6.f * dl, fmaxf(fabsf(zf), 1e-30f)) + 1.0f / 32768.f,
                          0.5f);
  for (int tr = 0; tr < 2; ++tr) {  // U: f_lo(s) >= 0 below the iterate
    const float sl = __fmul_rd(sg, 1.f - (tr == 0 ? kap : fminf(4.f * kap, 0.75f)));
    if (!(sl > 0.f)) continue;
    float part = 0.f;
    for (int j = j1; j < m; j += kGrp)
      part = __fadd_rd(part, __fmul_rd(alo(j), __frcp_rd(__fadd_ru(S.eu[j], sl))));
    const float neg = __fmul_ru(b1s, __frcp_ru(__fsub_rd(d2d, sl)));
    const float fl = __fadd_rd(__fsub_rd(1.f, neg), grp_sum_rd(part, mask, base));
    if (fl >= 0.f) {
      U = fmin(U, __dsub_ru(l2, (double)sl));
      break;
    }
  }
  for (int tr = 0; tr < 3; ++tr) {  // L: f_hi(s) <= 0 above the iterate
    const float su = tr == 0 ? __fmul_ru(sg, 1.f + kap)
                             : (tr == 1 ? __fmul_ru(sg, 1.f + 4.f * kap)
                                        : __fadd_ru(sg, __fmul_ru(d2u, 1.0f / 32768.f)));
    if (!(su < d2d)) continue;
    float part = 0.f;
    for (int j = j1; j < m; j += kGrp)
      part = __fadd_ru(part, __fmul_ru(chi(j), __frcp_ru(__fadd_rd(S.ed[j], su))));
    const float pos_ = __fmul_rd(B1s, __frcp_rd(__fsub_ru(d2u, su)));
    const float fh = __fadd_ru(__fsub_ru(1.f, pos_), grp_sum_ru(part, mask, base));
    if (fh <= 0.f) {
      L = fmax(L, __dsub_rd(l2, (double)su));
      break;
    }
  }
}

// Pass 1: both bounds of the probe rows [0, probe), a tile of kTile rows per
// CTA; the best L raises the limit.  The CTA that finishes last sets the
// rows the next pass takes: mu - l1 <= z_1^2 <= |phi_i|^2, so only rows
// with |phi_i|^2 >= lim - l1 can reach the limit.
template <typename T>
HY_DEV void odeim_probe_body(int bid, int nb,
    const T* __restrict__ phi, int64_t N, int m, const float* __restrict__ wt32,
    const float* __restrict__ nrm, const int* __restrict__ ord,
    const unsigned char* __restrict__ picked, int probe, const unsigned int* __restrict__ bmax,
    const int* __restrict__ bstart, double tie_tol, OdCtl* ctl, double* __restrict__ scores,
    const float* __restrict__ R, int C, int bsel, double* __restrict__ Lbuf) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char tsm[];
  TileSm& S = *reinterpret_cast<TileSm*>(tsm);
  const int t = threadIdx.x, r = t / kGrp, g = t % kGrp;
  const int gbase = (t & 31) & ~(kGrp - 1);
  const unsigned gmask = ((1u << kGrp) - 1u) << gbase;
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  stage_tile_tables(wt32, m, S);
  unsigned long long bestL = 0ull, cnt = 0;
  for (int b0 = bid * kTile; b0 < probe; b0 += nb * kTile) {
    const int pos = b0 + r;
    if (g == 0) {
      int i = -1;
      if (pos < probe) {
        i = ord[pos];
        if (picked[i]) {
          scores[pos] = -1.0;
          if (bsel > 1) Lbuf[pos] = -1.0;
          i = -1;
        }
      }
      S.pos[r] = i >= 0 ? pos : -1;
      S.row[r] = i;
      S.nrm[r] = i >= 0 ? nrm[i] : 0.f;
    }
    __syncthreads();
    tile_z<T>(phi, N, m, R, C, S);
    if (S.pos[r] >= 0) {
      double U, L;
      bounds_row(S, m, l1, l2, S.zt + r * kTileLd, S.nrm[r], gmask, gbase, g, U, L);
      if (g == 0) {
        scores[pos] = U;
        ++cnt;
        bestL = dbits(L) > bestL ? dbits(L) : bestL;
        if (bsel > 1) Lbuf[pos] = L;
      }
    }
    __syncthreads();
  }
  bestL = block_max_u64(bestL);
  cnt = block_sum(cnt);
  if (t == 0) {
    if (bestL && bsel <= 1) atomicMax(&ctl->slo, bestL);
    if (cnt) atomicAdd(&ctl->stat[1], cnt);
  }
  if (!last_block(&ctl->ticket, nb)) return;
  if (bsel > 1) {
    // several points per pass: the limit is the bsel-th largest lower bound
    // L of the probe rows (bsel rows score at least that much, so every row
    // among the pass's bsel best reaches it), counted with multiplicity
    unsigned long long above = ~0ull, kth = 0ull;
    long long seen = 0;
    for (int round = 0; round < bsel; ++round) {
      unsigned long long mx = 0ull;
      // keys: the bits of L > 0 (ordered like L), 0 for L <= 0; -1 marks a
      // picked row
      for (int q = t; q < probe; q += blockDim.x) {
        const double v = Lbuf[q];
        const unsigned long long k = v > 0.0 ? dbits(v) : 0ull;
        if (v != -1.0 && k < above) mx = k > mx ? k : mx;
      }
      mx = block_max_u64(mx);
      unsigned long long c = 0;
      for (int q = t; q < probe; q += blockDim.x) {
        const double v = Lbuf[q];
        c += (v != -1.0 && (v > 0.0 ? dbits(v) : 0ull) == mx && mx < above) ? 1ull : 0ull;
      }
      c = block_sum(c);
      if (c == 0) break;  // fewer than bsel probe rows: no limit from them
      seen += (long long)c;
      if (seen >= bsel) {
        kth = mx;
        break;
      }
      above = mx;
    }
    if (t == 0) ctl->slo = kth;
    __syncthreads();
  }
  const double lim = limit_of(ctl, tie_tol);
  const int n = plan_end(bmax, bstart, probe, (lim - l1) / (1.0 + 1e-5));
  if (t == 0) {
    ctl->n_c = n;
    ctl->ticket = 0u;
    ctl->stat[3] += 1;
  }
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_odeim_probe(
    const T* __restrict__ phi, int64_t N, int m, const float* __restrict__ wt32,
    const float* __restrict__ nrm, const int* __restrict__ ord,
    const unsigned char* __restrict__ picked, int probe, const unsigned int* __restrict__ bmax,
    const int* __restrict__ bstart, double tie_tol, OdCtl* ctl, double* __restrict__ scores,
    const float* __restrict__ R, int C, int bsel, double* __restrict__ Lbuf) {
  odeim_probe_body<T>(blockIdx.x, gridDim.x, phi, N, m, wt32, nrm, ord, picked, probe, bmax,
                      bstart, tie_tol, ctl, scores, R, C, bsel, Lbuf);
}

// Pass 2b: both full bounds of the rows pass 2a listed, a tile of kTile
// rows per CTA (U replaces the row's score); the best L raises the limit.
// The rows whose U reaches the limit of the time, and the probe rows whose
// U does, are listed in xlist for the exact pass.
template <typename T>
HY_DEV void odeim_screen_body(int bid, int nb,
    const T* __restrict__ phi, int64_t N, int m, const float* __restrict__ wt32,
    const float* __restrict__ nrm, const int* __restrict__ ord, const int* __restrict__ list,
    int probe, double tie_tol, OdCtl* ctl, double* __restrict__ scores, int* __restrict__ xlist,
    const float* __restrict__ R, int C, int bsel) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char tsm[];
  TileSm& S = *reinterpret_cast<TileSm*>(tsm);
  const int t = threadIdx.x, lane = t & 31, r = t / kGrp, g = t % kGrp;
  const int gbase = lane & ~(kGrp - 1);
  const unsigned gmask = ((1u << kGrp) - 1u) << gbase;
  const int count = ctl->n_list;
  {  // the probe rows
    const double lim = limit_of(ctl, tie_tol);
    for (int base = bid * kTileThreads; base < probe; base += nb * kTileThreads) {
      const int pos = base + t;
      const bool x = pos < probe && scores[pos] >= lim;
      const unsigned bal = __ballot_sync(0xffffffffu, x);
      if (bal) {
        int first = 0;
        if (lane == __ffs(bal) - 1) first = atomicAdd(&ctl->n_x, __popc(bal));
        first = __shfl_sync(0xffffffffu, first, __ffs(bal) - 1);
        if (x) xlist[first + __popc(bal & ((1u << lane) - 1u))] = pos;
      }
    }
  }
  if ((int)bid * kTile >= count) return;  // no listed row for this CTA
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  stage_tile_tables(wt32, m, S);
  unsigned long long bestL = 0ull, cnt = 0;
  for (int b0 = bid * kTile; b0 < count; b0 += nb * kTile) {
    if (g == 0) {
      const int e = b0 + r;
      const int pos = e < count ? list[e] : -1;
      const int i = pos >= 0 ? ord[pos] : -1;
      S.pos[r] = pos;
      S.row[r] = i;
      S.nrm[r] = i >= 0 ? nrm[i] : 0.f;
    }
    __syncthreads();
    tile_z<T>(phi, N, m, R, C, S);
    const int pos = S.pos[r];
    if (pos >= 0) {
      double U, L;
      bounds_row(S, m, l1, l2, S.zt + r * kTileLd, S.nrm[r], gmask, gbase, g, U, L);
      if (g == 0) {
        scores[pos] = U;
        ++cnt;
        bestL = dbits(L) > bestL ? dbits(L) : bestL;
        if (U >= limit_of(ctl, tie_tol)) xlist[atomicAdd(&ctl->n_x, 1)] = pos;
      }
    }
    __syncthreads();
  }
  bestL = block_max_u64(bestL);
  cnt = block_sum(cnt);
  if (t == 0) {
    if (bestL && bsel <= 1) atomicMax(&ctl->slo, bestL);  // (several points: the limit stays)
    if (cnt) atomicAdd(&ctl->stat[1], cnt);
  }
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_odeim_screen(
    const T* __restrict__ phi, int64_t N, int m, const float* __restrict__ wt32,
    const float* __restrict__ nrm, const int* __restrict__ ord, const int* __restrict__ list,
    int probe, double tie_tol, OdCtl* ctl, double* __restrict__ scores, int* __restrict__ xlist,
    const float* __restrict__ R, int C, int bsel) {
  odeim_screen_body<T>(blockIdx.x, gridDim.x, phi, N, m, wt32, nrm, ord, list, probe, tie_tol,
                       ctl, scores, xlist, R, C, bsel);
}

// ---- rank-one update of the eigensystem of M (one per oversampling step) ----
//
// M' = M + phi phi^T with M = W diag(d) W^T (d ascending).  In the basis W,
// M' = diag(d) + z z^T, z = W^T phi; its eigenvalues are the roots of the
// secular equation 1 + sum_i z_i^2 / (d_i - lambda) = 0 (Golub 1973), one in
// each (d_j, d_{j+1}) and the last in (d_n, d_n + |z|^2).  Components with a
// negligible z_i, and pairs of nearly equal d, are deflated first (a Givens
// rotation folds one z component into its neighbour), as in the
// divide-and-conquer eigensolver (Bunch, Nielsen & Sorensen 1978).  Each
// root is found by bisection in coordinates shifted to its nearer pole, so
// that d_i - lambda_j is known to full relative accuracy; z is then
// recomputed from the roots by Loewner's formula (Gu & Eisenstat 1994), which
// makes the eigenvectors (d_i - lambda_j)^{-1} z_i numerically orthogonal.

struct R1Work {
  int nK;          // non-deflated count
  int nD;          // deflated count
  int K[64];       // original indices (ascending d) of the non-deflated
  int D[64];       // deflated indices
  double dK[64];   // their (possibly rotated) d
  double zK[64];   // their z
  double dD[64];   // deflated eigenvalues
  int org[64];     // root j: origin index into K
  double tau[64];  // root j = dK[org[j]] + tau[j]
  double zh[64];   // Loewner z of the non-deflated components
};

// The eigensystem update's preparation for the point p just picked (one
// CTA, blockDim a multiple of 64): z = W^T phi_p, then deflation of the
// negligible z components and of nearly equal poles (a Givens rotation
// folds one z component into its neighbour), as in the divide-and-conquer
// eigensolver (Bunch, Nielsen & Sorensen 1978).  W (stride kLdw) and the
// eigenvalues ds are the CTA's shared copies (both may be rotated); the
// kept components go to wk, the possibly rotated W to Wrot (stride m).
HY_DEV void r1_prepare_block(double* W, double* ds, const double* ph, int m, double* zp,
                             double* z, R1Work* wk, double* __restrict__ Wrot) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  z_block(W, kLdw, ph, m, zp, z);
  __shared__ int nonsmall[64], nns, anyclose;
  __shared__ double tol_s, nz_s;
  {
    double r = 0.0, dm = 0.0;
    for (int j = tid; j < m; j += blockDim.x) {
      r = fma(z[j], z[j], r);
      dm = fmax(dm, fabs(ds[j]));
    }
    r = block_sum(r);
    dm = block_max(dm);
    if (tid == 0) {
      nz_s = sqrt(r);
      tol_s = 8.0 * 2.220446049250313e-16 * fmax(dm, r);
      anyclose = 0;
    }
  }
  __syncthreads();
  const double tol = tol_s, nz = nz_s;
  if (tid < 64) {  // ordered list of the non-negligible z (two warps, ballots)
    const bool keep = tid < m && !(fabs(z[tid]) * nz <= tol);
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    __shared__ int wcnt[2];
    if (lane == 0) wcnt[wid] = __popc(b);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    const int off = (wid == 1 ? wcnt[0] : 0) + __popc(b & ((1u << lane) - 1u));
    if (keep) nonsmall[off] = tid;
    if (tid == 0) nns = wcnt[0] + wcnt[1];
  }
  __syncthreads();
  for (int k = 1 + tid; k < nns; k += blockDim.x) {  // adjacent pairs, in parallel
    const int ip = nonsmall[k - 1], i = nonsmall[k];
    const double t = hypot(z[ip], z[i]);
    const double c = z[i] / t, sn = z[ip] / t;
    if (fabs(c * sn * (ds[i] - ds[ip])) <= tol) anyclose = 1;
  }
  __syncthreads();
  if (!anyclose) {
    // fast path: no rotation; K = the non-negligible entries, D = the rest
    for (int k = tid; k < nns; k += blockDim.x) {
      const int i = nonsmall[k];
      wk->K[k] = i;
      wk->dK[k] = ds[i];
      wk->zK[k] = z[i];
    }
    if (tid == 0) {
      int nD = 0;
      for (int i = 0, k = 0; i < m; ++i) {
        if (k < nns && nonsmall[k] == i) {
          ++k;
          continue;
        }
        wk->D[nD] = i;
        wk->dD[nD++] = ds[i];
      }
      wk->nK = nns;
      wk->nD = nD;
    }
  } else if (tid == 0) {
    int nK = 0, nD = 0, prev = -1;
    for (int i = 0; i < m; ++i) {
      if (fabs(z[i]) * nz <= tol) {
        wk->D[nD] = i;
        wk->dD[nD++] = ds[i];
        continue;
      }
      if (prev < 0) {
        prev = i;
        continue;
      }
      const double t = hypot(z[prev], z[i]);
      const double c = z[i] / t, sn = z[prev] / t;
      if (fabs(c * sn * (ds[i] - ds[prev])) <= tol) {
        // fold z[prev] into z[i]; prev becomes an eigenpair
        const double dp = c * c * ds[prev] + sn * sn * ds[i];
        const double di = sn * sn * ds[prev] + c * c * ds[i];
        for (int a2 = 0; a2 < m; ++a2) {
          const double wp = W[prev * kLdw + a2], wi = W[i * kLdw + a2];
          W[prev * kLdw + a2] = c * wp - sn * wi;
          W[i * kLdw + a2] = sn * wp + c * wi;
        }
        z[prev] = 0.0;
        z[i] = t;
        ds[i] = di;
        wk->D[nD] = prev;
        wk->dD[nD++] = dp;
        prev = i;
      } else {
        wk->K[nK] = prev;
        wk->dK[nK] = ds[prev];
        wk->zK[nK++] = z[prev];
        prev = i;
      }
    }
    if (prev >= 0) {
      wk->K[nK] = prev;
      wk->dK[nK] = ds[prev];
      wk->zK[nK++] = z[prev];
    }
    wk->nK = nK;
    wk->nD = nD;
  }
  __syncthreads();
  for (int i = tid; i < m * m; i += blockDim.x) {
    const int j = i / m, a = i - j * m;
    Wrot[i] = W[j * kLdw + a];
  }
}

// Pass 3: exact scores of the rows listed in xlist (U reached the limit of
// its time), spread over the CTAs round-robin (row k of the list to CTA
// k mod G) so that the FP64 work spreads over the SMs, four at a time per
// CTA: z by the whole CTA for each, then warp w solves the secular equation
// of the w-th row.  Before each group the limit is raised to the best
// exact score any CTA has found so far (and the best L); rows whose bound
// no longer reaches it get -1 (they cannot reach the tie window of the
// best).  Every exact score is listed as a candidate.  The CTA that finishes
// last picks point l (the lowest row in the tie window of the best exact
// score) and, for l + 1 < n_p, prepares the eigensystem update with it; it
// then resets the step's control block.
constexpr int kExactThreads = 128;
template <typename T>
HY_DEV void odeim_exact_body(int bid, int nb,
    const T* __restrict__ phi, int64_t N, int m, const double* __restrict__ lam_s,
    const double* __restrict__ W_s, const int* __restrict__ ord, const int* __restrict__ xlist,
    double tie_tol, OdCtl* ctl, double* __restrict__ scores, int* __restrict__ cand, int l,
    int np, int* __restrict__ pts, unsigned char* __restrict__ picked,
    const float* __restrict__ R, int C, R1Work* wk, double* __restrict__ Wrot, int bsel,
    int* __restrict__ pick_pos) {
  pdl_enter();
  extern __shared__ double sh[];
  double* W = sh;               // 64 x kLdw
  double* lam = W + 64 * kLdw;  // 64
  double* rb = lam + 64;        // 4 x 64: rows of the group
  double* zp = rb + 4 * 64;     // 2 x 64
  double* zs = zp + 2 * 64;     // 4 x 64
  __shared__ int grp[4];  // the group's positions still to score
  __shared__ int ngrp;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double l1 = ctl->lam1, l2 = ctl->lam2;
  const int nx = ctl->n_x;
  const int G = nb;
  double best = 0.0;
  unsigned long long cnt = 0;
  bool staged = false;
  for (int k0 = bid; k0 < nx; k0 += 4 * G) {
    if (tid == 0) {
      const double lnow = limit_of(ctl, tie_tol);
      int k = 0;
      for (int q = 0; q < 4; ++q) {
        const int e = k0 + q * G;
        if (e >= nx) break;
        const int pos = xlist[e];
        if (scores[pos] >= lnow)
          grp[k++] = pos;
        else
          scores[pos] = -1.0;
      }
      ngrp = k;
    }
    __syncthreads();
    const int ng = ngrp;
    if (ng > 0 && !staged) {
      stage_w(W_s, lam_s, m, W, lam);
      staged = true;
    }
    for (int idx = tid; idx < ng * 64; idx += kExactThreads) {
      const int q = idx >> 6, a = idx & 63;
      rb[idx] = a < m ? phi_at<T>(phi, N, a, ord[grp[q]], grp[q], R, C) : 0.0;
    }
    for (int q = 0; q < ng; ++q) z_block(W, kLdw, rb + 64 * q, m, zp, zs + 64 * q);
    if (wid < ng) {
      const double mu = secular_root_warp(zs + 64 * wid, lam, m, l1, l2);
      if (lane == 0) {
        scores[grp[wid]] = mu;
        if (bsel <= 1) atomicMax(&ctl->smax, dbits(mu));  // raises the limit of later groups
        cand[atomicAdd(&ctl->ncand, 1)] = grp[wid];
      }
      best = mu > best ? mu : best;
      ++cnt;
    }
    __syncthreads();
  }
  best = block_max(best);
  if (tid == 0 && bsel <= 1) atomicMax(&ctl->smax, dbits(best));
  if (lane == 0 && cnt) atomicAdd(&ctl->stat[2], cnt);
  if (!last_block(&ctl->ticket, nb)) return;
  // ---- the pick(s), then the update's preparation (this CTA alone) ----
  const unsigned long long key =
      bsel <= 1 ? pick_winner(scores, ord, cand, ctl, tie_tol, l, pts, picked)
                : pick_several(scores, ord, cand, ctl, tie_tol, l, np - l < bsel ? np - l : bsel,
                               pts, picked, pick_pos);
  if (l + 1 < np && key != ~0ull) {
    const int p = (int)(key >> 32), wpos = (int)(key & 0xffffffffull);
    if (!staged) stage_w(W_s, lam_s, m, W, lam);
    for (int a = tid; a < 64; a += blockDim.x)
      rb[a] = a < m ? phi_at<T>(phi, N, a, p, wpos, R, C) : 0.0;
    r1_prepare_block(W, lam, rb, m, zp, zs, wk, Wrot);
  }
  __syncthreads();
  if (tid == 0) {
    ctl->smax = 0ull;
    ctl->slo = 0ull;
    ctl->n_list = 0;
    ctl->n_x = 0;
    ctl->ncand = 0;
    ctl->ticket = 0u;
    ctl->n_c = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kExactThreads) k_odeim_exact(
    const T* __restrict__ phi, int64_t N, int m, const double* __restrict__ lam_s,
    const double* __restrict__ W_s, const int* __restrict__ ord, const int* __restrict__ xlist,
    double tie_tol, OdCtl* ctl, double* __restrict__ scores, int* __restrict__ cand, int l,
    int np, int* __restrict__ pts, unsigned char* __restrict__ picked,
    const float* __restrict__ R, int C, R1Work* wk, double* __restrict__ Wrot, int bsel,
    int* __restrict__ pick_pos) {
  odeim_exact_body<T>(blockIdx.x, gridDim.x, phi, N, m, lam_s, W_s, ord, xlist, tie_tol, ctl,
                      scores, cand, l, np, pts, picked, R, C, wk, Wrot, bsel, pick_pos);
}

// The update's preparation for the r-th point (r >= 1) of a pass that took
// several, once the eigensystem holds the earlier ones (one CTA).  Where the
// pass found fewer points, the update is the identity: every component
// deflated, the eigenpairs unchanged.
template <typename T>
__global__ void __launch_bounds__(kExactThreads) k_r1_prepare(
    const T* __restrict__ phi, int64_t N, int m, const double* __restrict__ lam_s,
    const double* __restrict__ W_s, const int* __restrict__ pts, int idx,
    const int* __restrict__ pick_pos, int r, const float* __restrict__ R, int C, R1Work* wk,
    double* __restrict__ Wrot) {
  pdl_enter();
  extern __shared__ double sh[];
  double* W = sh;               // 64 x kLdw
  double* lam = W + 64 * kLdw;  // 64
  double* rb = lam + 64;        // 64
  double* zp = rb + 4 * 64;     // 2 x 64
  double* zs = zp + 2 * 64;     // 64
  const int tid = threadIdx.x;
  stage_w(W_s, lam_s, m, W, lam);
  const int p = pts[idx], wpos = pick_pos[r];
  if (r >= pick_pos[16] || p < 0 || p >= N || wpos < 0 || wpos >= N) {
    __syncthreads();
    if (tid == 0) {
      wk->nK = 0;
      wk->nD = m;
    }
    for (int j = tid; j < m; j += blockDim.x) {
      wk->D[j] = j;
      wk->dD[j] = lam[j];
    }
    for (int i = tid; i < m * m; i += blockDim.x) {
      const int j = i / m, a = i - j * m;
      Wrot[i] = W[j * kLdw + a];
    }
    return;
  }
  for (int a = tid; a < 64; a += blockDim.x) rb[a] = a < m ? phi_at<T>(phi, N, a, p, wpos, R, C) : 0.0;
  __syncthreads();
  r1_prepare_block(W, lam, rb, m, zp, zs, wk, Wrot);
}

// One warp per root (CTA j); Delta[i * 64 + j] = d_i - lambda_j.
// Root j lies in (d_j, d_{j+1}) (the last one in (d_n, d_n + |z|^2)); it is
// computed as tau in coordinates shifted to the nearer pole o, so that
// d_i - lambda_j = (d_i - d_o) - tau keeps full relative accuracy.  Each
// step solves the two-pole model of f(tau) = 1 + sum_i z_i^2 / (del_i - tau)
// (the "middle way" of Li's secular solver, as in LAPACK's dlaed4): with
// psi the terms with poles at or left of d_j and phi the rest,
//   f ~ c + s / (del_j - tau') + S / (del_{j+1} - tau'),
//   s = psi' (del_j - tau)^2, S = phi' (del_{j+1} - tau)^2,
//   c = f - psi' (del_j - tau) - phi' (del_{j+1} - tau),
// a quadratic in the correction whose root in the interval is taken
// (the last root has no right pole: tau' = del_n + s / c).  Steps are kept
// inside a shrinking bracket (bisection otherwise); the iteration stops once
// |f| is within the rounding error of its evaluation, the step is below
// 2 ulp, or the bracket has collapsed.
HY_DEV void r1_roots_body(int bid, R1Work* wk, double* __restrict__ Delta) {
  pdl_enter();
  const int j = bid, lane = threadIdx.x;
  const int nK = wk->nK;
  if (j >= nK) return;
  double dv[2], z2[2];
  for (int u = 0; u < 2; ++u) {
    const int i = lane + 32 * u;
    dv[u] = i < nK ? wk->dK[i] : 0.0;
    const double zi = i < nK ? wk->zK[i] : 0.0;
    z2[u] = zi * zi;
  }
  const double rho = warp_sum(z2[0] + z2[1]);
  const double dj = wk->dK[j];
  const bool last = j == nK - 1;
  int o;
  double lo, hi;
  if (last) {
    o = j;
    lo = 0.0;
    hi = rho;
  } else {
    const double dn = wk->dK[j + 1];
    const double mid = 0.5 * (dj + dn);
    double f = 0.0;
    for (int u = 0; u < 2; ++u)
      if (lane + 32 * u < nK) f = f + z2[u] / (dv[u] - mid);
    f = 1.0 + warp_sum(f);
    if (f >= 0.0) {
      o = j;
      lo = 0.0;
      hi = mid - dj;
    } else {
      o = j + 1;
      lo = mid - dn;
      hi = 0.0;
    }
  }
  const double dorg = wk->dK[o];
  double del[2];
  for (int u = 0; u < 2; ++u) del[u] = dv[u] - dorg;
  const double delj = dj - dorg, deln = last ? 0.0 : wk->dK[j + 1] - dorg;
  double t = (o == j) ? 0.5 * hi : 0.5 * lo;
  const double eps = 2.220446049250313e-16;
  {  // the same model steps in FP32 (cheap) to a start for the FP64 ones,
     // which keep their own bracket
    const float fe = 1.1920929e-7f;
    float fdel[2], fz2[2];
    for (int u = 0; u < 2; ++u) {
      fdel[u] = (float)del[u];
      fz2[u] = (float)z2[u];
    }
    const float fdelj = (float)delj, fdeln = (float)deln;
    float ft = (float)t, flo = (float)lo, fhi = (float)hi;
    for (int it = 0; it < 16; ++it) {
      float f = 0.f, fa = 0.f, dps = 0.f, dph = 0.f;
      for (int u = 0; u < 2; ++u) {
        const int i = lane + 32 * u;
        if (i < nK) {
          const float r = __frcp_rn(fdel[u] - ft);
          const float q = fz2[u] * r;
          f += q;
          fa += fabsf(q);
          if (i <= j)
            dps = fmaf(q, r, dps);
          else
            dph = fmaf(q, r, dph);
        }
      }
      f = 1.f + warp_sum(f);
      fa = warp_sum(fa);
      dps = warp_sum(dps);
      dph = warp_sum(dph);
      if (fabsf(f) <= 8.f * fe * (1.f + fa + fabsf(ft) * (dps + dph))) break;
      if (f < 0.f)
        flo = ft;
      else
        fhi = ft;
      if (fhi - flo <= 2.f * fe * fmaxf(fabsf(fhi), fabsf(flo))) {
        ft = 0.5f * (flo + fhi);
        break;
      }
      const float Dj = fdelj - ft;
      float eta = NAN;
      if (last) {
        const float sL = dps * Dj * Dj, cq = f - dps * Dj;
        if (cq > 0.f) eta = Dj + __fdividef(sL, cq);
      } else {
        const float Dn = fdeln - ft;
        const float sL = dps * Dj * Dj, sR = dph * Dn * Dn;
        const float A = f - dps * Dj - dph * Dn;
        const float B = A * (Dj + Dn) + sL + sR;
        const float Cq = f * Dj * Dn;
        if (A == 0.f) {
          if (B != 0.f) eta = __fdividef(Cq, B);
        } else {
          const float qq = 0.5f * (B + copysignf(fsqrt_fast(fmaxf(B * B - 4.f * A * Cq, 0.f)), B));
          const float e1 = __fdividef(qq, A), e2 = qq != 0.f ? __fdividef(Cq, qq) : NAN;
          if (e1 > Dj && e1 < Dn) eta = e1;
          if (e2 > Dj && e2 < Dn) eta = e2;
        }
      }
      float nt = ft + eta;
      if (fabsf(nt - ft) <= 2.f * fe * fabsf(ft)) {
        ft = nt;
        break;
      }
      if (!(nt > flo && nt < fhi)) nt = 0.5f * (flo + fhi);
      ft = nt;
    }
    const double tc = (double)ft;
    if (tc > lo && tc < hi) t = tc;
  }
  for (int it = 0; it < 100; ++it) {
    double f = 0.0, fa = 0.0, dps = 0.0, dph = 0.0;
    for (int u = 0; u < 2; ++u) {
      const int i = lane + 32 * u;
      if (i < nK) {
        const double r = rcp64(del[u] - t);
        const double q = z2[u] * r;
        f = f + q;
        fa = fa + fabs(q);
        if (i <= j)
          dps = dps + q * r;
        else
          dph = dph + q * r;
      }
    }
    f = 1.0 + warp_sum(f);
    fa = warp_sum(fa);
    dps = warp_sum(dps);
    dph = warp_sum(dph);
    if (fabs(f) <= 8.0 * eps * (1.0 + fa + fabs(t) * (dps + dph))) break;
    if (f < 0.0)
      lo = t;
    else
      hi = t;
    if (hi - lo <= 2.0 * eps * fmax(fabs(hi), fabs(lo))) {
      t = 0.5 * (lo + hi);
      break;
    }
    const double Dj = delj - t;  // < 0
    double eta = NAN;
    if (last) {
      const double sL = dps * Dj * Dj, c = f - dps * Dj;
      if (c > 0.0) eta = Dj + sL / c;
    } else {
      const double Dn = deln - t;  // > 0
      const double sL = dps * Dj * Dj, sR = dph * Dn * Dn;
      const double A = f - dps * Dj - dph * Dn;
      const double B = A * (Dj + Dn) + sL + sR;
      const double Cq = f * Dj * Dn;
      // A eta^2 - B eta + Cq = 0: the root in (Dj, Dn)
      if (A == 0.0) {
        if (B != 0.0) eta = Cq / B;
      } else {
        const double q = 0.5 * (B + copysign(sqrt(fmax(B * B - 4.0 * A * Cq, 0.0)), B));
        const double e1 = q / A, e2 = q != 0.0 ? Cq / q : NAN;
        if (e1 > Dj && e1 < Dn) eta = e1;
        if (e2 > Dj && e2 < Dn) eta = e2;
      }
    }
    double nt = t + eta;
    if (fabs(nt - t) <= 2.0 * eps * fabs(t)) {  // before the bracket test: a
      t = nt;                                    // converged step may sit on it
      break;
    }
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    t = nt;
  }
  for (int u = 0; u < 2; ++u) {
    const int i = lane + 32 * u;
    if (i < nK) Delta[i * 64 + j] = del[u] - t;
  }
  if (lane == 0) {
    wk->org[j] = o;
    wk->tau[j] = t;
  }
}

__global__ void k_r1_roots(R1Work* wk, double* __restrict__ Delta) {
  r1_roots_body(blockIdx.x, wk, Delta);
}

// Loewner's z (Gu & Eisenstat): with Delta_iq = d_i - lambda_q,
//   zh_i^2 = (lambda_i - d_i) prod_{q != i} (lambda_q - d_i) / (d_q - d_i),
// signed like z_i.  One warp per component i (lane: q and q + 32), a product
// tree over the lanes.
HY_DEV void r1_loewner_body(int bid, R1Work* wk, const double* __restrict__ Delta) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int i = bid * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nK = wk->nK;
  if (i >= nK) return;
  const double di = wk->dK[i];
  double pr = 1.0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = lane + 32 * u;
    if (q < nK) {
      const double lq = -Delta[i * 64 + q];  // lambda_q - d_i
      pr *= q == i ? lq : lq * rcp64(wk->dK[q] - di);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pr *= __shfl_xor_sync(0xffffffffu, pr, o);
  if (lane == 0) {
    const double zz = sqrt(fmax(pr, 0.0));
    wk->zh[i] = wk->zK[i] >= 0.0 ? zz : -zz;
  }
}

__global__ void __launch_bounds__(128) k_r1_loewner(R1Work* wk, const double* __restrict__ Delta) {
  r1_loewner_body(blockIdx.x, wk, Delta);
}

// Eigenpair j of M + phi phi^T, written straight to its place in ascending
// order (CTA j of m).  For j < nK, the new pair: the root
// lambda_j = dK[org_j] + tau_j and the vector v_i = zh_i / (d_i - lambda_j)
// mapped back through W (the product split over the CTA's eight warps,
// thread t: row a = t % 64 over a quarter of the components); for j >= nK
// the deflated pair (dD, Wrot column D) unchanged.  Its rank among all m
// eigenvalues (ties by index) is the column it takes in W_out and wt32.
// CTA 0 also writes the sorted eigenvalues' control entries and the FP32
// tails of wt32.
HY_DEV void r1_vectors_body(int bid, const R1Work* __restrict__ wk,
                                const double* __restrict__ Delta,
                                const double* __restrict__ Wrot, int m,
                                double* __restrict__ d_out, double* __restrict__ W_out,
                                OdCtl* ctl, float* __restrict__ wt32) {
  pdl_enter();
  __shared__ double v[64];
  __shared__ double Wk[64 * 65];  // rows K[i] of Wrot, stride 65
  __shared__ double part[4][64];
  __shared__ int Ks[64];
  __shared__ double lv[64];
  __shared__ unsigned long long key[64];
  const int j = bid, tid = threadIdx.x;
  const int nK = wk->nK;
  for (int i = tid; i < m; i += blockDim.x) {
    const double x = i < nK ? wk->dK[wk->org[i]] + wk->tau[i] : wk->dD[i - nK];
    lv[i] = x;
    key[i] = dkey(x);
  }
  __syncthreads();
  int r = 0;
  for (int i = 0; i < m; ++i) r += (key[i] < key[j]) || (key[i] == key[j] && i < j);
  if (j < nK) {
    for (int i = tid; i < nK; i += blockDim.x) Ks[i] = wk->K[i];
    __syncthreads();
    for (int base = tid; base < nK * 64; base += blockDim.x * 8) {
      double wv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * blockDim.x;
        const int i = idx >> 6, a = idx & 63;
        wv[u] = idx < nK * 64 && a < m ? Wrot[Ks[i] * m + a] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < nK * 64) Wk[(idx >> 6) * 65 + (idx & 63)] = wv[u];
      }
    }
    double vi = 0.0;
    if (tid < 64) {
      if (tid < nK) vi = wk->zh[tid] * rcp64(Delta[tid * 64 + j]);
      v[tid] = vi;
    }
    __syncthreads();
    double nrm = tid < 64 ? vi * vi : 0.0;
    nrm = block_sum(nrm);
    const double inv = 1.0 / sqrt(nrm);
    {
      const int a = tid & 63, h = tid >> 6;
      const int i0 = h * 16, i1 = i0 + 16 < nK ? i0 + 16 : nK;
      double acc0 = 0.0, acc1 = 0.0;
      int i = i0;
      for (; i + 1 < i1; i += 2) {
        acc0 = fma(Wk[i * 65 + a], v[i], acc0);
        acc1 = fma(Wk[(i + 1) * 65 + a], v[i + 1], acc1);
      }
      if (i < i1) acc0 = fma(Wk[i * 65 + a], v[i], acc0);
      part[h][a] = acc0 + acc1;
    }
    __syncthreads();
    if (tid < m) {
      const double x = ((part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid])) * inv;
      W_out[r * m + tid] = x;
      wt32[tid * 64 + r] = (float)x;
    }
  } else {
    const int src = wk->D[j - nK];
    for (int a = tid; a < m; a += blockDim.x) {
      const double x = Wrot[src * m + a];
      W_out[r * m + a] = x;
      wt32[a * 64 + r] = (float)x;
    }
  }
  if (tid == 0) d_out[r] = lv[j];
  if (j == 0) {
    __shared__ double ls[64];
    for (int i = tid; i < m; i += blockDim.x) {
      int ri = 0;
      for (int q = 0; q < m; ++q) ri += (key[q] < key[i]) || (key[q] == key[i] && q < i);
      ls[ri] = lv[i];
    }
    __syncthreads();
    if (tid == 0) {
      ctl->lam1 = ls[0];
      ctl->lam2 = m > 1 ? ls[1] : INFINITY;
      ctl->lmax = ls[m - 1];
    }
    w32_tail(ls, m, wt32);
  }
}

__global__ void __launch_bounds__(256) k_r1_vectors(const R1Work* __restrict__ wk,
                                                    const double* __restrict__ Delta,
                                                    const double* __restrict__ Wrot, int m,
                                                    double* __restrict__ d_out,
                                                    double* __restrict__ W_out, OdCtl* ctl,
                                                    float* __restrict__ wt32) {
  r1_vectors_body(blockIdx.x, wk, Delta, Wrot, m, d_out, W_out, ctl, wt32);
}

__global__ void k_pad_sym2(const double* __restrict__ M, int m, int n, double* __restrict__ P) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int a = idx / n, b = idx % n;
    P[idx] = (a < m && b < m) ? M[a * m + b] : 0.0;
  }
}

// ---- driver -----------------------------------------------------------------

struct OdeimBufs {
  int* list;
  int* cand;
  int* xlist;
  float* rows;
  float* nrm;
  unsigned char* bkt;
  unsigned char* picked;
  int* ord;
  int* bcnt;
  int* bstart;
  int* bcur;
  unsigned int* bmax;
  double* scores;
  double* cvec;
  double* M;
  double* V;
  double* lam;
  double* lam_s;
  double* W_s;
  double* Mp;
  double* Wrot;
  double* Wnew;
  double* lamnew;
  double* Delta;
  double* lam_s2;
  double* W_s2;
  R1Work* r1;
  double* jbuf;
  double* jscale;
  int* jflag;
  double* Lbuf;   // several points per pass: the probe rows' lower bounds
  int* pick_pos;  // the pass's picked positions, [16] = how many
  double* Li;  // DEIM: inverses of the bordered factors (64 x 64 row-major)
  double* Ui;
  double* yv;
  OdCtl* ctl;
  float* wt32;  // the step's eigensystem in FP32 for the screens (kW32 floats)
};

size_t odeim_ws_bytes(int64_t N, int m) {
  size_t b = 0;
  b += N * sizeof(float) + N + N + 4 * N * sizeof(int) + N * sizeof(double) + 768;
  b += (size_t)(N < kCompact ? N : kCompact) * 64 * sizeof(float) + 256;
  b += (3 * (kNB + 1) + kNB) * sizeof(int);
  b += sizeof(double) * (64 + 6 * (size_t)(m + 1) * (m + 1) + 4 * m + 64);
  b += 16 * 256;
  b += sizeof(double) * (5 * 64 * 64 + 3 * 64) + sizeof(R1Work) + 16 * 256;
  b += sizeof(double) * (psd_eig_scratch_doubles(m + 1) + 2 * (m + 1) * (m + 1) + 512) + 3 * 256;
  b += sizeof(double) * (2 * 64 * 64 + 64) + 3 * 256;
  b += sizeof(float) * kW32 + 256;
  b += sizeof(double) * kProbe + 256 + 32 * sizeof(int) + 256;
  return b + 4096;
}

static OdeimBufs carve(void* ws, int64_t N, int m) {
  OdeimBufs o;
  char* p = (char*)ws;
  auto take = [&](size_t n) {
    char* r = p;
    p += (n + 255) & ~(size_t)255;
    return r;
  };
  o.ctl = (OdCtl*)take(256);
  o.scores = (double*)take(N * sizeof(double));
  o.nrm = (float*)take(N * sizeof(float));
  o.ord = (int*)take(N * sizeof(int));
  o.list = (int*)take(N * sizeof(int));
  o.cand = (int*)take(N * sizeof(int));
  o.xlist = (int*)take(N * sizeof(int));
  o.rows = (float*)take((size_t)(N < kCompact ? N : kCompact) * 64 * sizeof(float));
  o.bkt = (unsigned char*)take(N);
  o.picked = (unsigned char*)take(N);
  o.bcnt = (int*)take((kNB + 1) * sizeof(int));
  o.bstart = (int*)take((kNB + 1) * sizeof(int));
  o.bcur = (int*)take((kNB + 1) * sizeof(int));
  o.bmax = (unsigned int*)take(kNB * sizeof(int));
  o.cvec = (double*)take(64 * sizeof(double));
  o.M = (double*)take((size_t)m * m * sizeof(double));
  o.V = (double*)take((size_t)(m + 1) * (m + 1) * sizeof(double));
  o.lam = (double*)take((m + 1) * sizeof(double));
  o.lam_s = (double*)take((m + 1) * sizeof(double));
  o.W_s = (double*)take((size_t)m * m * sizeof(double));
  o.Mp = (double*)take((size_t)(m + 1) * (m + 1) * sizeof(double));
  o.Wrot = (double*)take((size_t)64 * 64 * sizeof(double));
  o.Wnew = (double*)take((size_t)64 * 64 * sizeof(double));
  o.lamnew = (double*)take(64 * sizeof(double));
  o.Delta = (double*)take((size_t)64 * 64 * sizeof(double));
  o.lam_s2 = (double*)take(64 * sizeof(double));
  o.W_s2 = (double*)take((size_t)64 * 64 * sizeof(double));
  o.r1 = (R1Work*)take(sizeof(R1Work));
  o.jbuf = (double*)take((psd_eig_scratch_doubles(m + 1) + (size_t)2 * (m + 1) * (m + 1) + 512) *
                         sizeof(double));
  o.jscale = (double*)take(64);
  o.jflag = (int*)take(64);
  o.Li = (double*)take((size_t)64 * 64 * sizeof(double));
  o.Ui = (double*)take((size_t)64 * 64 * sizeof(double));
  o.yv = (double*)take(64 * sizeof(double));
  o.wt32 = (float*)take(kW32 * sizeof(float));
  o.Lbuf = (double*)take(kProbe * sizeof(double));
  o.pick_pos = (int*)take(32 * sizeof(int));
  return o;
}

OdeimNorms odeim_norm_bufs(void* ws, int64_t N) {
  const OdeimBufs o = carve(ws, N, 1);  // these buffers precede every m-dependent one
  return OdeimNorms{o.nrm, o.bkt, o.bcnt, o.bmax};
}

void odeim_graphs_free(OdeimGraphs* g) {
  graph_slot_free(&g->deim);
  graph_slot_free(&g->over);
  g->N = -1;
  g->m = g->np = g->bs = -1;
}

// Launch with programmatic stream serialization (the kernel starts with
// pdl_enter(), which keeps stream order); where the attribute is refused,
// an ordinary launch.  The arguments are converted to the kernel's
// parameter types as in a triple-chevron launch.
template <typename... KArgs, typename... Args>
void pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
         Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  if (cudaLaunchKernelEx(&cfg, kern, args...) != cudaSuccess) {
    cudaGetLastError();
    cfg.numAttrs = 0;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  }
}

template <typename T>
int launch_odeim(const T* phi, int64_t N, int m, int np, double tie_tol, int* pts, void* ws,
                 void* host_pinned, cudaStream_t s, void (*mark)(void*, int), void* mark_arg,
                 bool norms_ready, OdeimGraphs* graphs, OdeimOver* over, int bsel) {
  if (over) over->active = 0;
  if (m <= 0) return 0;
  if (np > N) np = (int)N;
  const int bs = bsel > 1 ? bsel : 1;
  if (bs > 1) over = nullptr;  // (the multi-instance loops take one point per pass)
  OdeimBufs o = carve(ws, N, m);
  if (graphs && (graphs->N != N || graphs->m != m || graphs->np != np || graphs->bs != bs)) {
    odeim_graphs_free(graphs);
    graphs->N = N;
    graphs->m = m;
    graphs->np = np;
    graphs->bs = bs;
  }
  auto M_ = [&](int id) {
    if (mark) mark(mark_arg, id);
  };
  M_(12);
  cudaMemsetAsync(o.ctl, 0, sizeof(OdCtl), s);
  cudaMemsetAsync(o.picked, 0, N, s);
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (!norms_ready) {  // else the basis product's epilogue formed them
    cudaMemsetAsync(o.bcnt, 0, (kNB + 1) * sizeof(int), s);
    cudaMemsetAsync(o.bmax, 0, kNB * sizeof(int), s);
    k_rownorm<T><<<(int)blocks, 256, 0, HY_S(s)>>>(phi, N, m, o.nrm, o.bkt, o.bcnt, o.bmax);
  }
  k_bucket_scan<<<1, 32, 0, HY_S(s)>>>(o.bcnt, o.bstart, o.bcur);
  k_bucket_scatter<<<(int)blocks, 256, 0, HY_S(s)>>>(N, o.bkt, o.bcur, o.ord);
  const int C = (int)(N < kCompact ? N : kCompact);
  if (m <= 64) {
    k_gather_rows<T><<<152 * 8, 256, 0, HY_S(s)>>>(phi, N, m, o.ord, C, o.rows);
  }
  const int probe = (int)(N < kProbe ? N : kProbe);
  M_(-13);
  // DEIM.  The kernels of both greedy loops start with pdl_enter() and are
  // launched with programmatic stream serialization (pdl()): each is
  // scheduled while its predecessor runs and waits for it on the device.
  // A step is two passes; the second pass's last CTA picks the point and
  // forms the next step's coefficients.
  auto deim_loop = [&]() {
    cudaMemsetAsync(o.Li, 0, (size_t)64 * 64 * sizeof(double), s);
    cudaMemsetAsync(o.Ui, 0, (size_t)64 * 64 * sizeof(double), s);
    for (int l = 0; l < m; ++l) {
      pdl(k_deim_probe<T>, (probe + 15) / 16, 64, 0, s, phi, N, l, o.cvec, o.ord, o.picked,
          probe, o.bmax, o.bstart, tie_tol, o.ctl, o.scores, o.cand, o.rows, C);
      pdl(k_deim_rest<T>, 152 * 8, 256, 0, s, phi, N, l, m, o.cvec, o.ord, o.picked, probe,
          tie_tol, o.ctl, o.scores, o.cand, o.rows, C, pts, o.Li, o.Ui, o.yv, o.cvec);
    }
  };
  if (graphs)
    run_graphed(&graphs->deim, s, deim_loop);
  else
    deim_loop();
  if (mark) {  // DEIM ends, oversampling begins
    mark(mark_arg, -12);
    mark(mark_arg, 9);
  }
  if (np <= m) return 0;
  // ODEIM oversampling
  const int n = m % 2 ? m + 1 : m;  // Jacobi wants an even order
  k_odeim_gram<T><<<(m + 3) / 4, 256, 0, HY_S(s)>>>(phi, N, m, pts, m, o.M);
  const size_t smem_ex = sizeof(double) * ((size_t)64 * kLdw + 64 + 4 * 64 + 2 * 64 + 4 * 64);
  M_(12);
  // eigensystem of M: pivoted Cholesky + one-sided Jacobi (FP32 sweeps
  // first, then FP64 sweeps to full accuracy); two-sided Jacobi if M is
  // numerically rank deficient (its null space is needed)
  int rank_m = 0;
  if (run_psd_eig(o.M, m, o.V, o.lam, o.jbuf, o.jflag, (int*)host_pinned, 60, s,
                  (int*)host_pinned + 2, true) < 0)
    return -1;
  rank_m = ((int*)host_pinned)[2];
  cudaMemcpyAsync(&o.ctl->eig_sweeps, o.jflag + 4, sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (rank_m == m) {
    k_odeim_sort<<<1, 256, 0, HY_S(s)>>>(o.lam, o.V, m, m, o.lam_s, o.W_s, o.ctl, o.wt32);
  } else {
    k_pad_sym2<<<1, 256, 0, HY_S(s)>>>(o.M, m, n, o.Mp);
    if (run_jacobi_multi(o.Mp, n, o.V, o.lam, o.jbuf, o.jflag, (int*)host_pinned, o.jscale,
                         (double*)host_pinned + 1, 60, s) < 0)
      return -1;
    k_odeim_sort<<<1, 256, 0, HY_S(s)>>>(o.lam, o.V, n, m, o.lam_s, o.W_s, o.ctl, o.wt32);
  }
  M_(-13);
  // sub-stage marks only where the loop is not replayed from a graph (no
  // slot, or the legacy default stream, which cannot be captured)
  auto ML_ = [&](int id) {
    if (mark && (!graphs || s == 0)) mark(mark_arg, id);
  };
  if (over) {  // the loop is left to a multi-instance launch
    OdeimOver& v = *over;
    v.phi = phi;
    v.N = N;
    v.m = m;
    v.np = np;
    v.probe = probe;
    v.C = C;
    v.tie_tol = tie_tol;
    v.wt32 = o.wt32;
    v.nrm = o.nrm;
    v.ord = o.ord;
    v.picked = o.picked;
    v.bmax = o.bmax;
    v.bstart = o.bstart;
    v.ctl = o.ctl;
    v.scores = o.scores;
    v.list = o.list;
    v.xlist = o.xlist;
    v.R = o.rows;
    v.lam[0] = o.lam_s;
    v.lam[1] = o.lam_s2;
    v.W[0] = o.W_s;
    v.W[1] = o.W_s2;
    v.cand = o.cand;
    v.pts = pts;
    v.r1 = o.r1;
    v.Wrot = o.Wrot;
    v.Delta = o.Delta;
    if (v.m_cap < m) v.m_cap = m;
    v.active = 1;
    return 0;
  }
  smem_at_least((const void*)k_odeim_exact<T>, smem_ex);
  smem_at_least((const void*)k_r1_prepare<T>, smem_ex);
  // A pass is four scoring launches (the last picks the pass's points and
  // prepares the update for the first) and the three launches of each
  // eigensystem update (one point per pass in the paper's ODEIM; with
  // several, the updates of the later points each start with a preparation).
  auto over_loop = [&]() {
    for (int l = m; l < np;) {
      const int nbp = np - l < bs ? np - l : bs;
      ML_(13);
      pdl(k_odeim_probe<T>, (probe + kTile - 1) / kTile, kTileThreads, sizeof(TileSm), s, phi,
          N, m, o.wt32, o.nrm, o.ord, o.picked, probe, o.bmax, o.bstart, tie_tol, o.ctl,
          o.scores, o.rows, C, bs, o.Lbuf);
      ML_(-14);
      ML_(14);
      pdl(k_odeim_z1<T>, 152 * 8, 256, 0, s, phi, N, m, o.wt32, o.nrm, o.ord, o.picked, probe,
          tie_tol, o.ctl, o.scores, o.list, o.rows, C);
      ML_(-15);
      ML_(17);
      pdl(k_odeim_screen<T>, 152 * 4, kTileThreads, sizeof(TileSm), s, phi, N, m, o.wt32,
          o.nrm, o.ord, o.list, probe, tie_tol, o.ctl, o.scores, o.xlist, o.rows, C, bs);
      ML_(-18);
      ML_(15);
      pdl(k_odeim_exact<T>, 152, kExactThreads, smem_ex, s, phi, N, m, o.lam_s, o.W_s, o.ord,
          o.xlist, tie_tol, o.ctl, o.scores, o.cand, l, np, pts, o.picked, o.rows, C, o.r1,
          o.Wrot, bs, o.pick_pos);
      ML_(-16);
      for (int i = 0; i < nbp && l + i + 1 < np; ++i) {
        ML_(16);
        if (i > 0)
          pdl(k_r1_prepare<T>, 1, kExactThreads, smem_ex, s, phi, N, m, o.lam_s, o.W_s, pts,
              l + i, o.pick_pos, i, o.rows, C, o.r1, o.Wrot);
        pdl(k_r1_roots, m, 32, 0, s, o.r1, o.Delta);
        pdl(k_r1_loewner, (m + 3) / 4, 128, 0, s, o.r1, o.Delta);
        pdl(k_r1_vectors, m, 256, 0, s, o.r1, o.Delta, o.Wrot, m, o.lam_s2, o.W_s2, o.ctl,
            o.wt32);
        std::swap(o.lam_s, o.lam_s2);
        std::swap(o.W_s, o.W_s2);
        ML_(-17);
      }
      l += nbp;
    }
  };
  if (graphs)
    run_graphed(&graphs->over, s, over_loop);
  else
    over_loop();
  return 0;
}

template int launch_odeim<float>(const float*, int64_t, int, int, double, int*, void*, void*,
                                 cudaStream_t, void (*)(void*, int), void*, bool, OdeimGraphs*,
                                 OdeimOver*, int);
template int launch_odeim<double>(const double*, int64_t, int, int, double, int*, void*, void*,
                                  cudaStream_t, void (*)(void*, int), void*, bool, OdeimGraphs*,
                                  OdeimOver*, int);


// ---- several instances' oversampling loops, one launch per pass ------------
//
// The loops of n instances advance together: greedy step t of every
// instance (its point l = m + t) runs in one launch of each of the seven
// passes, instead of seven launches per instance and step.  An instance whose
// loop has ended (l >= np) leaves its CTAs idle.  The grid of a pass is the
// concatenation of the instances' own grids: work list `start` (n + 1 entries
// per pass) gives instance i the CTAs [start[i], start[i + 1]), and each
// CTA runs the single-instance pass body with its index and count within its
// instance, so the result is that of the instance's loop run alone (the
// picked point depends only on the exact scores, not on the CTA that scored
// a row).  The scoring passes' CTA counts follow the instance's row count
// (rows per CTA: the autotuned knob); the update's follow its m.

constexpr int kMultiPasses = 7;
constexpr int kTuneCands = 4;
constexpr int kRowsPerCta[kTuneCands] = {1024, 2048, 4096, 8192};
constexpr int kTuneReps = 2;

// the instance of CTA b: start[i] <= b < start[i + 1] (start ascending)
HY_DEV int multi_inst(const int* __restrict__ start, int n, int b) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= b)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_multi_probe(const OdeimOver* __restrict__ d,
                                                              const int* __restrict__ start,
                                                              int n, int t) {
  const int i = multi_inst(start, n, blockIdx.x);
  const OdeimOver& o = d[i];
  if (!o.active || o.m + t >= o.np) return;
  odeim_probe_body<T>(blockIdx.x - start[i], start[i + 1] - start[i], (const T*)o.phi, o.N, o.m,
                      o.wt32, o.nrm, o.ord, o.picked, o.probe, o.bmax, o.bstart, o.tie_tol,
                      (OdCtl*)o.ctl, o.scores, o.R, o.C, 1, (double*)nullptr);
}

template <typename T>
__global__ void __launch_bounds__(256) k_multi_z1(const OdeimOver* __restrict__ d,
                                                  const int* __restrict__ start, int n, int t) {
  start += n + 1;
  const int i = multi_inst(start, n, blockIdx.x);
  const OdeimOver& o = d[i];
  if (!o.active || o.m + t >= o.np) return;
  odeim_z1_body<T>(blockIdx.x - start[i], start[i + 1] - start[i], (const T*)o.phi, o.N, o.m,
                   o.wt32, o.nrm, o.ord, o.picked, o.probe, o.tie_tol, (OdCtl*)o.ctl, o.scores,
                   o.list, o.R, o.C);
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_multi_screen(const OdeimOver* __restrict__ d,
                                                               const int* __restrict__ start,
                                                               int n, int t) {
  start += 2 * (n + 1);
  const int i = multi_inst(start, n, blockIdx.x);
  const OdeimOver& o = d[i];
  if (!o.active || o.m + t >= o.np) return;
  odeim_screen_body<T>(blockIdx.x - start[i], start[i + 1] - start[i], (const T*)o.phi, o.N,
                       o.m, o.wt32, o.nrm, o.ord, o.list, o.probe, o.tie_tol, (OdCtl*)o.ctl,
                       o.scores, o.xlist, o.R, o.C, 1);
}

template <typename T>
__global__ void __launch_bounds__(kExactThreads) k_multi_exact(const OdeimOver* __restrict__ d,
                                                               const int* __restrict__ start,
                                                               int n, int t) {
  start += 3 * (n + 1);
  const int i = multi_inst(start, n, blockIdx.x);
  const OdeimOver& o = d[i];
  const int l = o.m + t;
  if (!o.active || l >= o.np) return;
  odeim_exact_body<T>(blockIdx.x - start[i], start[i + 1] - start[i], (const T*)o.phi, o.N, o.m,
                      o.lam[t & 1], o.W[t & 1], o.ord, o.xlist, o.tie_tol, (OdCtl*)o.ctl,
                      o.scores, o.cand, l, o.np, o.pts, o.picked, o.R, o.C, (R1Work*)o.r1,
                      o.Wrot, 1, (int*)nullptr);
}

__global__ void k_multi_roots(const OdeimOver* __restrict__ d, const int* __restrict__ start,
                              int n, int t) {
  start += 4 * (n + 1);
  const int i = multi_inst(start, n, blockIdx.x);
  const OdeimOver& o = d[i];
  if (!o.active || o.m + t + 1 >= o.np) return;
  r1_roots_body(blockIdx.x - start[i], (R1Work*)o.r1, o.Delta);
}

__global__ void __launch_bounds__(128) k_multi_loewner(const OdeimOver* __restrict__ d,
                                                       const int* __restrict__ start, int n,
                                                       int t) {
  start += 5 * (n + 1);
  const int i = multi_inst(start, n, blockIdx.x);
  const OdeimOver& o = d[i];
  if (!o.active || o.m + t + 1 >= o.np) return;
  r1_loewner_body(blockIdx.x - start[i], (R1Work*)o.r1, o.Delta);
}

__global__ void __launch_bounds__(256) k_multi_vectors(const OdeimOver* __restrict__ d,
                                                       const int* __restrict__ start, int n,
                                                       int t) {
  start += 6 * (n + 1);
  const int i = multi_inst(start, n, blockIdx.x);
  const OdeimOver& o = d[i];
  const int j = blockIdx.x - start[i];
  if (!o.active || o.m + t + 1 >= o.np || j >= o.m) return;
  r1_vectors_body(j, (const R1Work*)o.r1, o.Delta, o.Wrot, o.m, o.lam[(t + 1) & 1],
                  o.W[(t + 1) & 1], (OdCtl*)o.ctl, o.wt32);
}

struct OdeimMulti {
  int cap = 0;                     // instances the buffers hold
  OdeimOver* ddesc = nullptr;      // device: descriptors
  int* dstart = nullptr;           // device: kMultiPasses work lists of n + 1 entries
  OdeimOver* hdesc = nullptr;      // pinned staging of both
  int* hstart = nullptr;
  std::vector<long long> key;      // layout the graphs were captured for
  std::vector<std::pair<int, GraphSlot>> graphs;  // by step count
  // the autotuner: candidate c is timed kTuneReps times (ms per greedy step,
  // the least kept), then the fastest is used from then on
  int choice = -1;
  int calls = 0;
  float best[kTuneCands] = {-1.f, -1.f, -1.f, -1.f};
  int timed_cand = -1, timed_steps = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

OdeimMulti* odeim_multi_create() {
  OdeimMulti* mu = new (std::nothrow) OdeimMulti;
  if (!mu) return nullptr;
  if (cudaEventCreate(&mu->e0) != cudaSuccess || cudaEventCreate(&mu->e1) != cudaSuccess) {
    cudaGetLastError();
    odeim_multi_free(mu);
    return nullptr;
  }
  return mu;
}

void odeim_multi_free(OdeimMulti* mu) {
  if (!mu) return;
  for (auto& g : mu->graphs) graph_slot_free(&g.second);
  cudaFree(mu->ddesc);
  cudaFree(mu->dstart);
  cudaFreeHost(mu->hdesc);
  cudaFreeHost(mu->hstart);
  if (mu->e0) cudaEventDestroy(mu->e0);
  if (mu->e1) cudaEventDestroy(mu->e1);
  delete mu;
}

int odeim_multi_tuning(const OdeimMulti* mu, int* rows_per_cta, float* ms, int nc) {
  if (!mu) return -1;
  if (rows_per_cta) *rows_per_cta = mu->choice >= 0 ? kRowsPerCta[mu->choice] : 0;
  for (int c = 0; c < nc && c < kTuneCands; ++c) ms[c] = mu->best[c];
  return kTuneCands;
}

namespace {
template <typename... KArgs, typename... Args>
void pdl_multi(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
               Args&&... args) {
  if (grid > 0) pdl(kern, grid, block, smem, s, std::forward<Args>(args)...);
}

int clampi(long long v, int lo, int hi) { return (int)(v < lo ? lo : v > hi ? hi : v); }
}  // namespace

template <typename T>
int launch_odeim_multi(OdeimMulti* mu, const OdeimOver* const* inst, int n, cudaStream_t s) {
  if (!mu || n <= 0) return 0;
  // the timing of the previous call, if it was a tuning call
  if (mu->timed_cand >= 0) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, mu->e0, mu->e1) == cudaSuccess && mu->timed_steps > 0) {
      const float per = ms / mu->timed_steps;
      float& b = mu->best[mu->timed_cand];
      b = b < 0.f || per < b ? per : b;
    }
    cudaGetLastError();
    mu->timed_cand = -1;
  }
  int cand = mu->choice;
  if (cand < 0) {
    if (mu->calls >= kTuneCands * kTuneReps) {
      int c0 = 0;
      for (int c = 1; c < kTuneCands; ++c)
        if (mu->best[c] >= 0.f && (mu->best[c0] < 0.f || mu->best[c] < mu->best[c0])) c0 = c;
      mu->choice = cand = c0;
    } else {
      cand = mu->calls / kTuneReps;
    }
  }
  ++mu->calls;
  if (n > mu->cap) {
    cudaFree(mu->ddesc);
    cudaFree(mu->dstart);
    cudaFreeHost(mu->hdesc);
    cudaFreeHost(mu->hstart);
    mu->ddesc = nullptr;
    mu->dstart = nullptr;
    mu->hdesc = nullptr;
    mu->hstart = nullptr;
    mu->cap = 0;
    const size_t sb = (size_t)kMultiPasses * (n + 1) * sizeof(int);
    if (cudaMalloc((void**)&mu->ddesc, n * sizeof(OdeimOver)) != cudaSuccess ||
        cudaMalloc((void**)&mu->dstart, sb) != cudaSuccess ||
        cudaMallocHost((void**)&mu->hdesc, n * sizeof(OdeimOver)) != cudaSuccess ||
        cudaMallocHost((void**)&mu->hstart, sb) != cudaSuccess)
      return -1;
    mu->cap = n;
  }
  // work lists and the graph key
  const int rows = kRowsPerCta[cand];
  std::vector<long long> key;
  key.push_back(cand);
  key.push_back(n);
  int steps = 0;
  int* st = mu->hstart;
  for (int p = 0; p < kMultiPasses; ++p) st[p * (n + 1)] = 0;
  for (int i = 0; i < n; ++i) {
    const OdeimOver& v = *inst[i];
    mu->hdesc[i] = v;
    if (v.active && v.np - v.m > steps) steps = v.np - v.m;
    const int mc = v.m_cap > 0 ? v.m_cap : 1;
    const int cnt[kMultiPasses] = {
        (v.probe + kTile - 1) / kTile,
        clampi((v.N + rows - 1) / rows, 1, 152 * 16),
        clampi((v.N + 2ll * rows - 1) / (2ll * rows), 1, 152 * 8),
        clampi((v.N + 8ll * rows - 1) / (8ll * rows), 1, 152 * 2),
        mc,
        (mc + 3) / 4,
        mc};
    for (int p = 0; p < kMultiPasses; ++p) st[p * (n + 1) + i + 1] = st[p * (n + 1) + i] + cnt[p];
    key.push_back(v.N);
    key.push_back(v.probe);
    key.push_back(mc);
  }
  if (steps == 0) return 0;
  if (key != mu->key) {
    for (auto& g : mu->graphs) graph_slot_free(&g.second);
    mu->graphs.clear();
    mu->key = key;
  }
  if (cudaMemcpyAsync(mu->ddesc, mu->hdesc, n * sizeof(OdeimOver), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(mu->dstart, mu->hstart, (size_t)kMultiPasses * (n + 1) * sizeof(int),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return -1;
  int grid[kMultiPasses];
  for (int p = 0; p < kMultiPasses; ++p) grid[p] = st[p * (n + 1) + n];
  const size_t smem_ex = sizeof(double) * ((size_t)64 * kLdw + 64 + 4 * 64 + 2 * 64 + 4 * 64);
  smem_at_least((const void*)k_multi_exact<T>, smem_ex);
  const OdeimOver* dd = mu->ddesc;
  const int* ds = mu->dstart;
  auto loop = [&]() {
    for (int t = 0; t < steps; ++t) {
      pdl_multi(k_multi_probe<T>, grid[0], kTileThreads, sizeof(TileSm), s, dd, ds, n, t);
      pdl_multi(k_multi_z1<T>, grid[1], 256, 0, s, dd, ds, n, t);
      pdl_multi(k_multi_screen<T>, grid[2], kTileThreads, sizeof(TileSm), s, dd, ds, n, t);
      pdl_multi(k_multi_exact<T>, grid[3], kExactThreads, smem_ex, s, dd, ds, n, t);
      if (t + 1 < steps) {
        pdl_multi(k_multi_roots, grid[4], 32, 0, s, dd, ds, n, t);
        pdl_multi(k_multi_loewner, grid[5], 128, 0, s, dd, ds, n, t);
        pdl_multi(k_multi_vectors, grid[6], 256, 0, s, dd, ds, n, t);
      }
    }
  };
  GraphSlot* g = nullptr;
  for (auto& e : mu->graphs)
    if (e.first == steps) g = &e.second;
  if (!g) {
    mu->graphs.emplace_back(steps, GraphSlot{});
    g = &mu->graphs.back().second;
  }
  const bool timing = mu->choice < 0;
  if (timing) cudaEventRecord(mu->e0, s);
  run_graphed(g, s, loop);
  if (timing) {
    cudaEventRecord(mu->e1, s);
    mu->timed_cand = cand;
    mu->timed_steps = steps;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template int launch_odeim_multi<float>(OdeimMulti*, const OdeimOver* const*, int, cudaStream_t);
template int launch_odeim_multi<double>(OdeimMulti*, const OdeimOver* const*, int,
                                        cudaStream_t);

}  // namespace hy
