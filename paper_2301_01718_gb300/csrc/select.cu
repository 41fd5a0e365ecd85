// Error-indicator selection and sampling sets: Sec. 2.3.3 (RRE ordering,
// Eq. rre, S-hat = G union P) and the sampling-set steps of Algorithm 1 (union, setdiff,
// Neighbors; Fig. 1).
//
// Exact selection: each cell's error eps maps to an integer key
// floor(eps * 2^s), s = 63 - ceil(log2 Nc) - e where eps_max = f 2^e
// (f in [0.5, 1)), so sums of keys never overflow 63 bits and the RRE test
// sum_{top n} key >= delta * S is exact 128-bit integer arithmetic.  The
// order is (descending key, ascending cell id).  A most-significant-digit
// radix select (8 passes of 8-bit digits with per-digit counts and key sums)
// finds the threshold key K* and how many cells equal to K* are taken; an
// ordered scan takes those with the lowest ids.  Integer atomics make every
// count exact, so the result does not depend on scheduling.
#include "common.cuh"
#include "internal.h"

namespace hy {

struct SelState {
  unsigned long long prefix;  // high bits of K* found so far
  unsigned long long acc_gt;  // sum of keys above the current range
  long long cnt_gt;           // number of keys above the current range
  long long n_target;         // top-fraction: cells wanted
  long long n_g;              // result
  long long take_eq;          // cells with key == K* to take (lowest ids)
  int shift;                  // s
  int mode;                   // HYROM_SEL_*
  unsigned long long S;       // total of keys
  unsigned long long a;       // delta = a 2^(E-53)
  int sh;                     // 53 - E
  int empty;                  // 1: select nothing
};

__global__ void k_eps_max(const void* __restrict__ eps, int is_f32, int64_t nc,
                          unsigned long long* out_bits) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double e = is_f32 ? (double)((const float*)eps)[i] : ((const double*)eps)[i];
    m = e > m ? e : m;
  }
  m = block_max(m);
  if (threadIdx.x == 0) atomicMax(out_bits, dbits(m));
}

HY_DEV int ceil_log2_ll(long long n) {
  int b = 0;
  while ((1LL << b) < n) ++b;
  return b;
}

__global__ void k_sel_setup(const unsigned long long* emax_bits, int64_t nc, SelState* st) {
  const double emax = bitsd(*emax_bits);
  int e = 0;
  frexp(emax, &e);
  st->shift = emax > 0.0 ? 63 - ceil_log2_ll(nc) - e : 0;
  st->prefix = 0;
  st->acc_gt = 0;
  st->cnt_gt = 0;
  st->empty = emax > 0.0 ? 0 : 1;
}

__global__ void k_keys(const void* __restrict__ eps, int is_f32, int64_t nc,
                       const SelState* __restrict__ st, unsigned long long* __restrict__ keys,
                       unsigned long long* total) {
  const int s = st->shift;
  const bool empty = st->empty;
  unsigned long long sum = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double e = is_f32 ? (double)((const float*)eps)[i] : ((const double*)eps)[i];
    unsigned long long k = 0;
    if (!empty && e > 0.0) k = (unsigned long long)floor(ldexp(e, s));
    keys[i] = k;
    sum += k;
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(total, sum);
}

__global__ void k_sel_mode(SelState* st, const unsigned long long* total, int mode, double delta,
                           double top_frac, int64_t nc) {
  st->mode = mode;
  st->S = *total;
  if (mode == HYROM_SEL_TOPFRAC) {
    long long n = (long long)ceil(top_frac * (double)nc);
    if (n > nc) n = nc;
    if (n < 0) n = 0;
    st->n_target = n;
    st->empty = n == 0 ? 1 : 0;  // all-zero errors still give ids by order
  } else {
    int E = 0;
    const double f = frexp(delta, &E);
    st->a = (unsigned long long)ldexp(f, 53);
    st->sh = 53 - E;
    st->n_target = 0;
    if (st->S == 0) st->empty = 1;
  }
}

// histogram of digit `d` (bits 8d..8d+7) over keys whose bits above match;
// counts are aggregated per warp over lanes with the same digit, and key
// sums are formed only for the RRE rule (the top fraction needs counts)
__global__ void k_sel_hist(const unsigned long long* __restrict__ keys, int64_t nc, int d,
                           const SelState* __restrict__ st, unsigned int* __restrict__ hcnt,
                           unsigned long long* __restrict__ hsum) {
  __shared__ unsigned int sc[256];
  __shared__ unsigned long long ss[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    sc[i] = 0;
    ss[i] = 0;
  }
  __syncthreads();
  if (!st->empty) {
    const bool sums = st->mode != HYROM_SEL_TOPFRAC;
    const int hi = 8 * (d + 1);
    const int lane = threadIdx.x & 31;
    const unsigned long long pre = st->prefix;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // i - lane is the same for the 32 lanes of a warp: uniform trip count
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - lane < nc; i += stride) {
      unsigned long long k = 0;
      bool valid = i < nc;
      if (valid) {
        k = keys[i];
        valid = hi >= 64 || (k >> hi) == (pre >> hi);
      }
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      if (valid) {
        const int dg = (int)((k >> (8 * d)) & 255ull);
        const unsigned peers = __match_any_sync(vm, dg);
        if (lane == __ffs(peers) - 1) atomicAdd(&sc[dg], (unsigned)__popc(peers));
        if (sums) atomicAdd(&ss[dg], k);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    if (sc[i]) {
      atomicAdd(&hcnt[i], sc[i]);
      if (ss[i]) atomicAdd(&hsum[i], ss[i]);
    }
  }
}

HY_DEV bool rre_met(const SelState* st, unsigned long long acc) {
  const unsigned __int128 lhs = (unsigned __int128)acc << st->sh;
  const unsigned __int128 rhs = (unsigned __int128)st->a * st->S;
  return lhs >= rhs;
}

// Choose digit d of K*: scanning the digits from 255 down, the first at
// which the rule is met (top fraction: the cells above plus this digit's
// reach n_target; RRE: a nonempty digit whose keys plus all above meet Eq.
// rre), else 0.  One block of 256 threads: thread t = digit t; suffix sums
// of counts and key sums give each digit what lies above it, and the
// largest digit meeting the rule is the first from the top.  Clears the
// histogram for the next digit.
__global__ void __launch_bounds__(256) k_sel_level(int d, SelState* st, unsigned int* hcnt,
                                                   unsigned long long* hsum) {
  __shared__ long long wc[8];
  __shared__ unsigned long long wsm[8];
  __shared__ int chosen_s;
  __shared__ long long above_c[256];
  __shared__ unsigned long long above_s[256];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (t == 0) chosen_s = 0;
  const bool empty = st->empty;
  // reversed order: r = 255 - digit, so an inclusive scan over r sums the
  // digits >= this one
  const int dg = 255 - t;
  const long long c = empty ? 0 : (long long)hcnt[dg];
  const unsigned long long sm = empty ? 0ull : hsum[dg];
  long long ic = c;
  unsigned long long is = sm;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long yc = __shfl_up_sync(0xffffffffu, ic, o);
    const unsigned long long ys = __shfl_up_sync(0xffffffffu, is, o);
    if (lane >= o) {
      ic += yc;
      is += ys;
    }
  }
  if (lane == 31) {
    wc[wid] = ic;
    wsm[wid] = is;
  }
  __syncthreads();
  long long bc = 0;
  unsigned long long bs = 0;
  for (int w = 0; w < wid; ++w) {
    bc += wc[w];
    bs += wsm[w];
  }
  above_c[dg] = bc + ic - c;  // cells with a larger digit
  above_s[dg] = bs + is - sm;
  if (!empty) {
    bool stop;
    if (st->mode == HYROM_SEL_TOPFRAC)
      stop = st->cnt_gt + above_c[dg] + c >= st->n_target;
    else
      stop = c > 0 && rre_met(st, st->acc_gt + above_s[dg] + sm);
    if (stop) atomicMax(&chosen_s, dg);
  }
  hcnt[dg] = 0;
  hsum[dg] = 0;
  __syncthreads();
  if (t != 0 || empty) return;
  const int chosen = chosen_s;
  st->cnt_gt += above_c[chosen];
  st->acc_gt += above_s[chosen];
  st->prefix |= ((unsigned long long)chosen) << (8 * d);
  if (d == 0) {
    const unsigned long long K = st->prefix;
    long long r;
    if (st->mode == HYROM_SEL_TOPFRAC) {
      r = st->n_target - st->cnt_gt;
    } else {
      // smallest r with (acc_gt + r K) 2^sh >= a S
      const unsigned __int128 need = (unsigned __int128)st->a * st->S;
      const unsigned __int128 have = (unsigned __int128)st->acc_gt << st->sh;
      const unsigned __int128 step = (unsigned __int128)K << st->sh;
      r = 0;
      if (need > have && step > 0) r = (long long)((need - have + step - 1) / step);
    }
    st->take_eq = r;
    st->n_g = st->cnt_gt + r;
  }
}

// Mark G: keys > K*, plus the take_eq lowest-id cells with key == K*.
// Grid of CTAs over contiguous chunks of whole 32-cell words; ranks of the
// equal keys come from per-chunk counts (pass 1) and an exclusive scan.
__global__ void k_sel_count_eq(const unsigned long long* __restrict__ keys, int64_t nc,
                               int64_t chunk, const SelState* __restrict__ st,
                               long long* __restrict__ cnt) {
  const int64_t c0 = blockIdx.x * chunk;
  int64_t c1 = c0 + chunk;
  if (c1 > nc) c1 = nc;
  long long n = 0;
  if (!st->empty) {
    const unsigned long long K = st->prefix;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) n += keys[i] == K;
  }
  n = block_sum(n);
  if (threadIdx.x == 0) cnt[blockIdx.x] = n;
}

// In-place exclusive prefix sum of n <= 1024 counts by one block of 1024
// threads (warp shuffle scans, then a scan of the 32 warp totals).
__global__ void __launch_bounds__(1024) k_exclusive_scan_ll(long long* v, int n) {
  __shared__ long long wsum[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const long long x = t < n ? v[t] : 0;
  long long incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long w = wsum[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  if (t < n) v[t] = (wid > 0 ? wsum[wid - 1] : 0) + incl - x;
}

__global__ void k_sel_mark(const unsigned long long* __restrict__ keys, int64_t nc, int64_t chunk,
                           const SelState* __restrict__ st, const long long* __restrict__ off,
                           uint32_t* __restrict__ bm) {
  // one warp-synchronous pass in order; chunk is a multiple of 32
  __shared__ long long base;
  __shared__ int wcnt[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t c0 = blockIdx.x * chunk;
  int64_t c1 = c0 + chunk;
  if (c1 > nc) c1 = nc;
  const bool empty = st->empty;
  const unsigned long long K = st->prefix;
  const long long take = st->take_eq;
  if (threadIdx.x == 0) base = off[blockIdx.x];
  __syncthreads();
  for (int64_t w0 = c0; w0 < c1; w0 += 32 * (int64_t)nw) {
    const int64_t i = w0 + 32 * wid + lane;
    bool valid = i < c1;
    const unsigned long long k = valid ? keys[i] : 0;
    const bool gt = valid && !empty && k > K;
    const bool eq = valid && !empty && k == K;
    const unsigned eqm = __ballot_sync(0xffffffffu, eq);
    if (lane == 0) wcnt[wid] = __popc(eqm);
    __syncthreads();
    long long before = base;
    for (int x = 0; x < wid; ++x) before += wcnt[x];
    const long long rank = before + __popc(eqm & ((1u << lane) - 1u));
    const bool sel = gt || (eq && rank < take);
    const unsigned word = __ballot_sync(0xffffffffu, sel);
    const int64_t wbase = w0 + 32 * wid;
    if (lane == 0 && wbase < c1) bm[wbase >> 5] = word;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long add = 0;
      for (int x = 0; x < nw; ++x) add += wcnt[x];
      base += add;
    }
    __syncthreads();
  }
}

void launch_select(const void* eps, int is_f32, int64_t nc, int mode, double delta,
                   double top_frac, unsigned long long* keys, void* scratch, uint32_t* g_bitmap,
                   long long* n_g_dev, cudaStream_t s) {
  // scratch layout
  char* p = (char*)scratch;
  SelState* st = (SelState*)p;
  p += 256;
  unsigned long long* emax = (unsigned long long*)p;
  p += 64;
  unsigned long long* total = (unsigned long long*)p;
  p += 64;
  unsigned int* hcnt = (unsigned int*)p;
  p += 256 * sizeof(unsigned int);
  unsigned long long* hsum = (unsigned long long*)p;
  p += 256 * sizeof(unsigned long long);
  long long* cnt = (long long*)p;  // sel_chunks entries
  const int nchunk_max = 1024;
  int64_t chunk = (nc + nchunk_max - 1) / nchunk_max;
  chunk = ((chunk + 1023) / 1024) * 1024;
  const int nchunk = (int)((nc + chunk - 1) / chunk);
  cudaMemsetAsync(scratch, 0, 256 + 64 + 64 + 256 * (sizeof(unsigned int) + 8), s);
  int64_t blocks = (nc + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_eps_max<<<(int)blocks, 256, 0, HY_S(s)>>>(eps, is_f32, nc, emax);
  k_sel_setup<<<1, 1, 0, HY_S(s)>>>(emax, nc, st);
  k_keys<<<(int)blocks, 256, 0, HY_S(s)>>>(eps, is_f32, nc, st, keys, total);
  k_sel_mode<<<1, 1, 0, HY_S(s)>>>(st, total, mode, delta, top_frac, nc);
  // keys are below 2^(63 - ceil(log2 nc)): the digits above are zero and
  // their passes would choose digit 0 with nothing above it
  int lg = 0;
  while ((1LL << lg) < nc) ++lg;
  const int top = (63 - lg - 1) / 8;
  for (int d = top; d >= 0; --d) {
    k_sel_hist<<<(int)blocks, 256, 0, HY_S(s)>>>(keys, nc, d, st, hcnt, hsum);
    k_sel_level<<<1, 256, 0, HY_S(s)>>>(d, st, hcnt, hsum);
  }
  k_sel_count_eq<<<nchunk, 256, 0, HY_S(s)>>>(keys, nc, chunk, st, cnt);
  k_exclusive_scan_ll<<<1, 1024, 0, HY_S(s)>>>(cnt, nchunk);
  const int64_t nwords = (nc + 31) / 32;
  cudaMemsetAsync(g_bitmap, 0, nwords * sizeof(uint32_t), s);
  k_sel_mark<<<nchunk, 256, 0, HY_S(s)>>>(keys, nc, chunk, st, cnt, g_bitmap);
  cudaMemcpyAsync(n_g_dev, &st->n_g, sizeof(long long), cudaMemcpyDeviceToDevice, s);
}

size_t select_scratch_bytes() { return 256 + 64 + 64 + 256 * (4 + 8) + 1024 * 8 + 256; }

// ---------------------------------------------------------------------------
// sampling sets
// ---------------------------------------------------------------------------

__global__ void k_points_to_cells(const int* __restrict__ pts, int np, int64_t nc,
                                  uint32_t* __restrict__ bm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const int64_t c = pts[i] % nc;
    atomicOr(&bm[c >> 5], 1u << (c & 31));
  }
}

// dst = cells within diamond distance `radius` of a set cell of src;
// `exclude` (may be NULL) is removed from the result.  One thread per cell,
// one ballot per word.
__global__ void k_dilate(DevCfg c, const uint32_t* __restrict__ src, int radius,
                         const uint32_t* __restrict__ exclude, uint32_t* __restrict__ dst) {
  const bool twoD = c.ny > 1;
  const bool px = c.bc[0] == HYROM_BC_PERIODIC, py = c.bc[2] == HYROM_BC_PERIODIC;
  const int64_t nwords = (c.nc + 31) / 32;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll;
       base < nwords * 32; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = base + (threadIdx.x & 31);
    bool on = false;
    if (cell < c.nc) {
      const int gi = (int)(cell % c.nx), gj = (int)(cell / c.nx);
      const int ry = twoD ? radius : 0;
      for (int dj = -ry; dj <= ry && !on; ++dj) {
        const int rem = radius - (dj < 0 ? -dj : dj);
        for (int di = -rem; di <= rem && !on; ++di) {
          int ii = gi + di, jj = gj + dj;
          if (px)
            ii = imod(ii, c.nx);
          else if (ii < 0 || ii >= c.nx)
            continue;
          if (twoD) {
            if (py)
              jj = imod(jj, c.ny);
            else if (jj < 0 || jj >= c.ny)
              continue;
          }
          on = bit_get(src, (int64_t)jj * c.nx + ii);
        }
      }
      if (on && exclude && bit_get(exclude, cell)) on = false;
    }
    const unsigned word = __ballot_sync(0xffffffffu, on);
    if ((threadIdx.x & 31) == 0 && base < c.nc) dst[base >> 5] = word;
  }
}

__global__ void k_popcount(const uint32_t* __restrict__ bm, int64_t nwords, long long* out) {
  long long n = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords;
       i += (int64_t)gridDim.x * blockDim.x)
    n += __popc(bm[i]);
  n = block_sum(n);
  if (threadIdx.x == 0) atomicAdd((unsigned long long*)out, (unsigned long long)n);
}

// Tiles (TX x TY cells) that contain a set cell, as an unordered list.
__global__ void k_active_tiles(DevCfg c, const uint32_t* __restrict__ bm, int TX, int TY,
                               int* __restrict__ tiles, int* __restrict__ ntiles) {
  const int tx = (c.nx + TX - 1) / TX, ty = (c.ny + TY - 1) / TY;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tx * ty; t += gridDim.x * blockDim.x) {
    const int x0 = (t % tx) * TX, y0 = (t / tx) * TY;
    bool any = false;
    for (int j = y0; j < y0 + TY && j < c.ny && !any; ++j)
      for (int i = x0; i < x0 + TX && i < c.nx && !any; ++i)
        any = bit_get(bm, (int64_t)j * c.nx + i);
    if (any) tiles[atomicAdd(ntiles, 1)] = t;
  }
}

// Ascending list of the set cells (single pass per chunk with an offset
// from an exclusive scan of per-chunk counts).
__global__ void k_bits_count(const uint32_t* __restrict__ bm, int64_t nwords, int64_t wchunk,
                             long long* __restrict__ cnt) {
  const int64_t w0 = blockIdx.x * wchunk;
  int64_t w1 = w0 + wchunk;
  if (w1 > nwords) w1 = nwords;
  long long n = 0;
  for (int64_t i = w0 + threadIdx.x; i < w1; i += blockDim.x) n += __popc(bm[i]);
  n = block_sum(n);
  if (threadIdx.x == 0) cnt[blockIdx.x] = n;
}

// one warp per chunk: lane l takes word w0 + 32 i + l; a warp scan of the
// words' popcounts gives each lane its output offset
__global__ void k_bits_list(const uint32_t* __restrict__ bm, int64_t nwords, int64_t wchunk,
                            const long long* __restrict__ off, int* __restrict__ out, int64_t cap) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = blockIdx.x * wchunk;
  int64_t w1 = w0 + wchunk;
  if (w1 > nwords) w1 = nwords;
  long long o = off[blockIdx.x];
  for (int64_t wb = w0; wb < w1; wb += 32) {
    const int64_t w = wb + lane;
    uint32_t b = w < w1 ? bm[w] : 0u;
    const int c = __popc(b);
    int incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    long long my = o + incl - c;
    while (b) {
      const int t = __ffs(b) - 1;
      b &= b - 1;
      if (my < cap) out[my] = (int)(w * 32 + t);
      ++my;
    }
    o += __shfl_sync(0xffffffffu, incl, 31);
  }
}

void launch_bits_to_list(const uint32_t* bm, int64_t nc, long long* cnt_scratch, int* out,
                         int64_t cap, cudaStream_t s) {
  const int64_t nwords = (nc + 31) / 32;
  const int nchunk_max = 1024;
  int64_t wchunk = (nwords + nchunk_max - 1) / nchunk_max;
  if (wchunk < 1) wchunk = 1;
  const int nchunk = (int)((nwords + wchunk - 1) / wchunk);
  k_bits_count<<<nchunk, 256, 0, HY_S(s)>>>(bm, nwords, wchunk, cnt_scratch);
  k_exclusive_scan_ll<<<1, 1024, 0, HY_S(s)>>>(cnt_scratch, nchunk);
  k_bits_list<<<nchunk, 32, 0, HY_S(s)>>>(bm, nwords, wchunk, cnt_scratch, out, cap);
}

void launch_masks(const DevCfg& c, const uint32_t* g_bitmap, const int* pts, int np, int halo,
                  int stencil_r, uint32_t* base, uint32_t* s_hat, uint32_t* s_tilde,
                  long long* n_s_dev, cudaStream_t s) {
  const int64_t nwords = (c.nc + 31) / 32;
  if (g_bitmap)
    cudaMemcpyAsync(base, g_bitmap, nwords * 4, cudaMemcpyDeviceToDevice, s);
  else
    cudaMemsetAsync(base, 0, nwords * 4, s);
  if (np > 0) k_points_to_cells<<<(np + 255) / 256, 256, 0, HY_S(s)>>>(pts, np, c.nc, base);
  int64_t blocks = (nwords * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (halo > 0)
    k_dilate<<<(int)blocks, 256, 0, HY_S(s)>>>(c, base, halo, nullptr, s_hat);
  else
    cudaMemcpyAsync(s_hat, base, nwords * 4, cudaMemcpyDeviceToDevice, s);
  k_dilate<<<(int)blocks, 256, 0, HY_S(s)>>>(c, s_hat, stencil_r, s_hat, s_tilde);
  cudaMemsetAsync(n_s_dev, 0, sizeof(long long), s);
  k_popcount<<<152, 256, 0, HY_S(s)>>>(s_hat, nwords, n_s_dev);
}

void launch_popcount(const uint32_t* bm, int64_t nwords, long long* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(long long), s);
  k_popcount<<<152, 256, 0, HY_S(s)>>>(bm, nwords, out);
}

void launch_active_tiles(const DevCfg& c, const uint32_t* bm, int TX, int TY, int* tiles,
                         int* ntiles, cudaStream_t s) {
  cudaMemsetAsync(ntiles, 0, sizeof(int), s);
  const int nt = ((c.nx + TX - 1) / TX) * ((c.ny + TY - 1) / TY);
  k_active_tiles<<<(nt + 255) / 256, 256, 0, HY_S(s)>>>(c, bm, TX, TY, tiles, ntiles);
}

}  // namespace hy
