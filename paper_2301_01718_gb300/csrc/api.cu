// C ABI of libhyrom (include/hyrom.h): the context, Algorithm 1 of the paper
// (hybrid snapshot AROM) driven on one GPU stream, and the stage entry
// points.  All arithmetic runs in the kernels of hdm.cu, filter.cu, rom.cu,
// select.cu and odeim.cu; this file allocates, validates, enqueues and
// reads back the few counts the host needs (basis rank, sample sizes,
// subiteration convergence).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hyrom.h"
#include "common.cuh"
#include "internal.h"

using hy::DevCfg;

// The forward record of a run that hyrom_adjoint sweeps backwards: every
// state, and for each hybrid step the predictor (the partial step before the
// reconstruction), the reduced coordinates, the sampled set and ODEIM points
// in effect, and each filter pass's keep bitmap and order; for each rebuild
// the window and the reference-state versions it read and made.  Bases are
// not kept: the reverse sweep recomputes each from its window.
struct AdjStep {
  bool full = false, rebuild = false, psi_init = false;
  int phi_ver = -1, psi_ver = -1, m_eff = 0, n_p = 0;
  int psi_cur = -1, new_phi = -1, new_psi = -1, init_psi = -1;
};
struct AdjTape {
  int steps = 0, passmax = 0, box[4] = {0, 0, 0, 0};
  double wgt = 0.0;
  double* states = nullptr;   // (steps + 1) x N
  double* vpred = nullptr;    // (steps + 1) x N
  double* ys = nullptr;       // (steps + 1) x 64
  uint32_t* shats = nullptr;  // (steps + 1) x nwords
  int* rows = nullptr;        // (steps + 1) x n_p
  uint32_t* keeps = nullptr;  // (steps + 1) x passmax x nwords
  int* orders = nullptr;      // (steps + 1) x passmax
  int* npass = nullptr;       // steps + 1
  double* Jpart = nullptr;    // 1216 partial sums
  double* J = nullptr;        // the output
  std::vector<double*> psis;  // reference-state versions (N each)
  std::vector<AdjStep> rec;   // index = step
  int cur_phi = -1, cur_psi = -1, nphi = 0;
};

struct hyrom_ctx {
  hyrom_config cfg;
  AdjTape* tape = nullptr;  // set while hyrom_adjoint records its forward run
  DevCfg dc;
  cudaStream_t st = nullptr;
  // the selection of G_{k+1} runs on st2 beside the basis rebuild's
  // eigensolve (it reads the old basis; the new one is written after the
  // join); sel_pending: a selection forked and not yet joined
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool sel_pending = false;
  int f32 = 0;
  size_t esz = 8;
  int64_t N = 0, nc = 0, nwords = 0;
  int w = 0, m = 0, np = 0, nslot = 0, wp = 0, ntiles_max = 0;
  int64_t k = 0;
  int sticky = 0;
  std::string err;
  std::vector<void*> allocs;
  size_t bytes = 0;

  // snapshots and the basis in effect
  void* ring = nullptr;
  void* psi = nullptr;
  void* psi_next = nullptr;
  void* phi = nullptr;
  int m_eff = 0;
  int np_eff = 0;
  int has_basis = 0;
  int psi_set = 0;
  std::vector<int64_t> psi_steps;  // psi = mean of these snapshots
  int* pts = nullptr;
  double* pinv = nullptr;
  double* y = nullptr;
  double* y2 = nullptr;
  double* dy = nullptr;
  int* status = nullptr;
  // sampling sets
  uint32_t *g_bm = nullptr, *base_bm = nullptr, *shat = nullptr, *stilde = nullptr;
  uint32_t* tmp_bm = nullptr;
  int* tiles = nullptr;
  int* ntiles = nullptr;
  int* seg = nullptr;
  int* nseg = nullptr;
  long long* n_s_dev = nullptr;
  long long* n_g_dev = nullptr;
  long long* list_cnt = nullptr;
  int64_t n_s = 0;
  // filter
  void *fg = nullptr, *ftmp = nullptr, *rho_old = nullptr, *rho_new = nullptr;
  double* fpart = nullptr;
  int* fctl = nullptr;
  uint32_t* kbits = nullptr;
  int* ftiles_a = nullptr;
  int* ftiles_b = nullptr;
  int* fcounts = nullptr;
  int* forders = nullptr;
  // selection
  void* eps = nullptr;
  unsigned long long* keys = nullptr;
  void* sel_scratch = nullptr;
  // POD
  double* H = nullptr;
  double* Hpart = nullptr;
  int gram_chunks = 0;
  // a step whose state hyrom_set_state replaced and whose Gram row is still
  // to form (-1: none); the next Gram update forms it in the same pass
  int64_t gram_dirty = -1;
  double* hp = nullptr;
  double* pp = nullptr;
  double* Gc = nullptr;
  double* V = nullptr;
  double* lam = nullptr;
  double* sig = nullptr;
  double* xraw2 = nullptr;
  int* m_eff_dev = nullptr;
  void* C = nullptr;
  double* Cd = nullptr;
  int* win_dev = nullptr;
  int* ps_dev = nullptr;
  double* X = nullptr;
  double* rawpart = nullptr;
  int* rotated = nullptr;
  double* ident = nullptr;
  double* jbuf = nullptr;
  // ODEIM
  void* od_ws = nullptr;
  // Newton
  double* tol_dev = nullptr;
  double* newton_ws = nullptr;
  int* fail_dev = nullptr;
  // sample-row reduced solve: S-hat cells (ascending), normal-matrix partials,
  // the normal matrix, its Cholesky factor and inverse diagonal, right-hand
  // side; sample_ok = the factor of the current basis and S-hat is valid
  int* s_cells = nullptr;
  double* s_part = nullptr;
  double* s_G = nullptr;
  double* s_L = nullptr;
  double* s_dinv = nullptr;
  double* s_b = nullptr;
  bool sample_ok = false;
  // the basis product formed ODEIM's row-norm data for the current basis
  bool norms_ready = false;
  // the rebuild's DEIM and oversampling loops as CUDA graphs
  hy::OdeimGraphs od_graphs;
  // batching: a rebuild leaves its oversampling loop (described in `over`)
  // to a multi-instance launch and stops before the loop's consumers; the
  // rest of the rebuild runs in finish_rebuild
  bool defer_over = false;
  hy::OdeimOver over{};
  struct {
    bool on = false;
    hyrom_step_info inf{};
    const uint32_t* gbm = nullptr;
    int me = 0, np = 0;
  } pend;
  // the paper's HDM (MUSCL-Roe-BDF2): Newton-GMRES solver and the S-hat cell
  // list its partial solves run over
  hy::MusclSolver* mus = nullptr;
  int* mus_cells = nullptr;
  int muscl_fail = 0;    // Newton solves of the current call that hit newton_max
  int muscl_passes = 0;  // filter passes of the last hybrid step
  // the filter's passes as a CUDA graph, and their per-call arguments
  hy::GraphSlot filt_graph;
  void* fargs = nullptr;
  // pinned host mirror for read-backs
  void* host = nullptr;
  // optional per-stage CUDA-event timers (hyrom_profile): up to kEvPairs
  // intervals per stage between two synchronisations
  static constexpr int kEvPairs = 160;
  int profile = 0;
  cudaEvent_t* ev_a[HYROM_NSTAGE] = {};
  cudaEvent_t* ev_b[HYROM_NSTAGE] = {};
  int ev_used[HYROM_NSTAGE] = {};
  int ev_open[HYROM_NSTAGE] = {};
  double stage_ms[HYROM_NSTAGE] = {};
  int64_t stage_n[HYROM_NSTAGE] = {};
};

namespace hy {
// process total (any thread) and this thread's own count (graph capture
// attributes the launches it made to the graph it captured)
static std::atomic<unsigned long long> g_launches{0};
static thread_local unsigned long long t_launches = 0;
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void add_launches(unsigned long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
unsigned long long thread_launch_count() { return t_launches; }

void smem_at_least(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{dev, func}];
  if (bytes <= cur) return;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
      cudaSuccess)
    cur = bytes;
}
}  // namespace hy

static __global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

static void convert_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  k_f64_to_f32<<<152 * 8, 256, 0, HY_S(s)>>>(a, b, n);
}

namespace {

hyrom_status fail(hyrom_ctx* c, hyrom_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (s == HYROM_ECUDA) c->sticky = 1;
  }
  return s;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, HYROM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

#define CKL()                                                                           \
  do {                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, HYROM_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
  } while (0)

bool dalloc(hyrom_ctx* ctx, void** p, size_t n) {
  if (n == 0) n = 16;
  n = (n + 255) & ~(size_t)255;
  if (cudaMalloc(p, n) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ctx->allocs.push_back(*p);
  ctx->bytes += n;
  return true;
}

template <typename P>
bool dal(hyrom_ctx* ctx, P** p, size_t n) {
  return dalloc(ctx, (void**)p, n);
}

hyrom_status validate(const hyrom_config* c, char* why, size_t nwhy) {
  auto bad = [&](const char* m) {
    snprintf(why, nwhy, "%s", m);
    return HYROM_EINVAL;
  };
  if (c->pde != HYROM_PDE_BURGERS && c->pde != HYROM_PDE_EULER) return bad("pde");
  if (c->scheme != HYROM_SCHEME_BE && c->scheme != HYROM_SCHEME_RK2 &&
      c->scheme != HYROM_SCHEME_BDF2_MUSCL)
    return bad("scheme");
  if (c->scheme == HYROM_SCHEME_BDF2_MUSCL) {
    if (c->pde != HYROM_PDE_EULER) return bad("the MUSCL-Roe-BDF2 HDM is for the Euler equations");
    if (c->precision != HYROM_PREC_F64) return bad("the MUSCL-Roe-BDF2 HDM runs in FP64");
    if (c->nx < 4 || (c->ny > 1 && c->ny < 4)) return bad("MUSCL needs 4 cells per axis");
    if (!(c->newton_tol > 0.0)) return bad("newton_tol > 0");
  }
  if (c->precision != HYROM_PREC_F64 && c->precision != HYROM_PREC_F32) return bad("precision");
  if (c->nx < 4 || c->ny < 1) return bad("grid: nx >= 4, ny >= 1");
  if ((int64_t)c->nx * c->ny * (c->pde == HYROM_PDE_BURGERS ? 1 : 4) > (int64_t)1 << 30)
    return bad("grid too large (ndof > 2^30)");
  if (c->pde == HYROM_PDE_BURGERS && c->ny != 1) return bad("Burgers is 1D (ny = 1)");
  for (int i = 0; i < 4; ++i)
    if (c->bc[i] < 0 || c->bc[i] > 2) return bad("bc");
  if ((c->bc[0] == HYROM_BC_PERIODIC) != (c->bc[1] == HYROM_BC_PERIODIC))
    return bad("x sides must both be periodic or both not");
  if ((c->bc[2] == HYROM_BC_PERIODIC) != (c->bc[3] == HYROM_BC_PERIODIC))
    return bad("y sides must both be periodic or both not");
  if (c->pde == HYROM_PDE_BURGERS && (c->bc[0] == HYROM_BC_SHOCK))
    return bad("shock sides need the Euler equations");
  if (c->scheme == HYROM_SCHEME_BE) {
    if (c->pde != HYROM_PDE_BURGERS) return bad("BDF1 is implemented for Burgers");
    if (c->precision != HYROM_PREC_F64) return bad("BDF1 Newton runs in FP64");
    if (c->bc[0] != HYROM_BC_PERIODIC) return bad("BDF1 Burgers is periodic");
  }
  if (!(c->dx > 0 && c->dy > 0 && c->dt > 0)) return bad("dx, dy, dt > 0");
  if (c->m < 1 || c->m > 64) return bad("1 <= m <= 64");
  if (c->w < c->m || c->w > 128) return bad("m <= w <= 128");
  if (c->n_p < c->m || c->n_p > 1024) return bad("m <= n_p <= 1024");
  if (hy::gappy_pinv_smem(c->m, c->n_p) > 227 * 1024) return bad("n_p * m too large");
  if (c->sel_mode != HYROM_SEL_RRE && c->sel_mode != HYROM_SEL_TOPFRAC) return bad("sel_mode");
  if (c->sel_mode == HYROM_SEL_RRE && !(c->delta >= 1.0 / 1024 && c->delta <= 1.0))
    return bad("delta in [2^-10, 1]");
  if (c->sel_mode == HYROM_SEL_TOPFRAC && !(c->top_frac >= 0.0 && c->top_frac <= 1.0))
    return bad("top_frac in [0, 1]");
  if (c->halo < 0 || c->halo > 8) return bad("0 <= halo <= 8");
  if (c->regress_rows != HYROM_ROWS_ODEIM && c->regress_rows != HYROM_ROWS_SAMPLE)
    return bad("regress_rows");
  if (c->reduced_prec < HYROM_RED_F32 || c->reduced_prec > HYROM_RED_TF32_SPLIT)
    return bad("reduced_prec");
  if (c->reduced_prec != HYROM_RED_F32 && c->precision != HYROM_PREC_F32)
    return bad("tensor-core normal matrices need FP32 states");
  if (c->odeim_batch < 0 || c->odeim_batch > 16) return bad("odeim_batch must be in [0, 16]");
  if (c->jmax < 1 || c->jmax_f < 1 || c->newton_max < 1) return bad("iteration limits >= 1");
  if (c->n_filt < 0 || c->n_filt > 3) return bad("n_filt");
  for (int i = 0; i < c->n_filt; ++i)
    if (c->filt_orders[i] < 1 || c->filt_orders[i] > 3) return bad("filt_orders in {1,2,3}");
  if (!(c->tie_tol >= 0 && c->tie_tol < 1e-3)) return bad("tie_tol");
  return HYROM_OK;
}

// ---- stage timers: events on the context stream around each stage ----------
void t_begin(hyrom_ctx* c, int id, cudaStream_t s) {
  if (!c->profile || c->ev_used[id] >= hyrom_ctx::kEvPairs) return;
  cudaEventRecord(c->ev_a[id][c->ev_used[id]], s);
  c->ev_open[id] = 1;
}
void t_end(hyrom_ctx* c, int id, cudaStream_t s) {
  if (!c->profile || !c->ev_open[id]) return;
  cudaEventRecord(c->ev_b[id][c->ev_used[id]], s);
  c->ev_used[id] += 1;
  c->ev_open[id] = 0;
}
void t_begin(hyrom_ctx* c, int id) { t_begin(c, id, c->st); }
void t_end(hyrom_ctx* c, int id) { t_end(c, id, c->st); }

// the rebuild's stream waits for a forked selection
void join_select(hyrom_ctx* c) {
  if (!c->sel_pending) return;
  cudaStreamWaitEvent(c->st, c->ev_join, 0);
  c->sel_pending = false;
}
// after a stream synchronisation: fold finished intervals into the totals
void t_collect(hyrom_ctx* c) {
  if (!c->profile) return;
  for (int i = 0; i < HYROM_NSTAGE; ++i) {
    for (int j = 0; j < c->ev_used[i]; ++j) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->ev_a[i][j], c->ev_b[i][j]) == cudaSuccess) {
        c->stage_ms[i] += ms;
        c->stage_n[i] += 1;
      }
    }
    c->ev_used[i] = 0;
  }
}

// sub-stage marks from inside the ODEIM launcher: id >= 0 begins stage id,
// id < 0 ends stage -id - 1
void odeim_mark(void* p, int id) {
  hyrom_ctx* c = (hyrom_ctx*)p;
  if (id >= 0)
    t_begin(c, id);
  else
    t_end(c, -id - 1);
}

// ring slot of snapshot step j
inline int slot_of(const hyrom_ctx* c, int64_t j) { return (int)(j % c->nslot); }

hyrom_status sync(hyrom_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->st));
  CKL();
  t_collect(ctx);
  return HYROM_OK;
}

template <typename T>
T* ring_at(hyrom_ctx* c, int64_t step) {
  return (T*)c->ring + (int64_t)slot_of(c, step) * c->N;
}

// rows of the raw ring Gram for a freshly written slot (FP32 path)
template <typename T>
void gram_update(hyrom_ctx* c, int64_t step) {
  if (!c->f32) return;
  t_begin(c, HYROM_T_GRAM);
  const int64_t d = c->gram_dirty;
  c->gram_dirty = -1;
  if (d >= 0 && d != step && slot_of(c, d) != slot_of(c, step))
    hy::launch_gram_rows2<T>((const T*)c->ring, c->N, c->nslot, slot_of(c, d), slot_of(c, step),
                             c->Hpart, c->gram_chunks, c->H, c->st);
  else
    hy::launch_gram_row<T>((const T*)c->ring, c->N, c->nslot, slot_of(c, step), c->Hpart,
                           c->gram_chunks, c->H, c->st);
  t_end(c, HYROM_T_GRAM);
}

// Form a Gram row left pending by hyrom_set_state (before H is read).
void gram_flush(hyrom_ctx* c) {
  if (c->gram_dirty < 0) return;
  gram_update<float>(c, c->gram_dirty);
}

// ---------------------------------------------------------------------------
// Reduced coordinates of v (Sec. 2.2): on the ODEIM rows P through the
// stored pseudo-inverse, or on every dof row of S-hat through the stored
// Cholesky factor of the sample-row normal matrix.
template <typename T>
void gappy_y(hyrom_ctx* ctx, const T* v, const T* psi, double* y, const double* y_prev,
             double* dy, cudaStream_t s) {
  if (ctx->sample_ok)
    hy::launch_sample_solve<T>((const T*)ctx->phi, ctx->N, ctx->m_eff, ctx->s_cells,
                               (int)ctx->n_s, ctx->dc.nvar, ctx->nc, v, psi, ctx->s_part,
                               ctx->s_b, ctx->s_L, ctx->s_dinv, y, y_prev, dy, s);
  else
    hy::launch_gappy_apply<T>(ctx->pinv, ctx->m_eff, ctx->np_eff, ctx->pts, v, psi, y, y_prev,
                              dy, s);
}
template <typename T>
void gappy_y(hyrom_ctx* ctx, const T* v, const T* psi, double* y, const double* y_prev,
             double* dy) {
  gappy_y<T>(ctx, v, psi, y, y_prev, dy, ctx->st);
}

// The paper's HDM: R_k(q) = 0 by Newton-GMRES on the listed cells (all when
// cells is null), q holding the start and the frozen values; the tolerance
// is newton_tol * max(1, max |q_{k-1}|), as for the BDF1 HDM.
hyrom_status muscl_solve(hyrom_ctx* ctx, double* q, const double* qp, const double* qp2,
                         int64_t k, const int* cells, int64_t n) {
  hy::launch_newton_tol(ctx->dc, qp, ctx->cfg.newton_tol, ctx->tol_dev, ctx->st);
  double* hd = (double*)ctx->host + 24;
  CK(cudaMemcpyAsync(hd, ctx->tol_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  int its = 0, arn = 0;
  const int r = hy::muscl_newton(ctx->mus, ctx->dc, q, qp, qp2, k, cells, n, hd[0],
                                 ctx->cfg.newton_max, 1e-6, ctx->st, &its, &arn);
  if (r < 0) return fail(ctx, HYROM_ECUDA, "Newton-GMRES: %s", cudaGetErrorString(cudaGetLastError()));
  if (r > 0) ctx->muscl_fail += 1;
  return HYROM_OK;
}

// Algorithm 1, advance part: full-step test, full HDM step or hybrid step
// ---------------------------------------------------------------------------

template <typename T>
hyrom_status newton_full(hyrom_ctx* ctx, const T* qp, T* q) {
  hy::launch_newton_tol(ctx->dc, (const double*)qp, ctx->cfg.newton_tol, ctx->tol_dev, ctx->st);
  hy::launch_burgers_newton_full(ctx->dc, (const double*)qp, (double*)q, ctx->tol_dev,
                                 ctx->cfg.newton_max, ctx->newton_ws, ctx->fail_dev, ctx->st);
  CKL();
  return HYROM_OK;
}

template <typename T>
hyrom_status newton_partial(hyrom_ctx* ctx, const T* qp, T* q, const uint32_t* shat,
                            int64_t n_s) {
  if (n_s >= ctx->nc) return newton_full<T>(ctx, qp, q);
  hy::launch_newton_tol(ctx->dc, (const double*)qp, ctx->cfg.newton_tol, ctx->tol_dev, ctx->st);
  hy::launch_burgers_newton_partial(ctx->dc, (const double*)qp, (double*)q, shat, ctx->seg,
                                    ctx->nseg, ctx->tol_dev, ctx->cfg.newton_max,
                                    ctx->newton_ws, ctx->fail_dev, ctx->st);
  CKL();
  return HYROM_OK;
}

template <typename T>
hyrom_status advance_t(hyrom_ctx* ctx, hyrom_step_info* info) {
  const hyrom_config& cf = ctx->cfg;
  const int64_t k = ctx->k + 1;
  const bool full = (k + 1 <= cf.w) || (cf.z > 0 && k % cf.z == 0);
  const T* qp = ring_at<T>(ctx, k - 1);
  T* q = ring_at<T>(ctx, k);
  hyrom_step_info inf;
  memset(&inf, 0, sizeof inf);
  inf.k = k;
  inf.was_full = full;
  CK(cudaMemsetAsync(ctx->fail_dev, 0, sizeof(int), ctx->st));
  CK(cudaMemsetAsync(ctx->fail_dev + 12, 0, sizeof(int), ctx->st));
  ctx->muscl_fail = 0;
  const bool muscl = cf.scheme == HYROM_SCHEME_BDF2_MUSCL;
  const T* qp2 = (muscl && k >= 2) ? ring_at<T>(ctx, k - 2) : nullptr;
  if (full) {
    t_begin(ctx, HYROM_T_FULL);
    if (muscl) {
      if constexpr (sizeof(T) == 8) {
        CK(cudaMemcpyAsync(q, qp, ctx->N * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
        if (hyrom_status s = muscl_solve(ctx, q, qp, qp2, k, nullptr, ctx->nc)) return s;
      }
    } else if (cf.scheme == HYROM_SCHEME_RK2) {
      hy::launch_rk2<T>(ctx->dc, qp, q, k, nullptr, nullptr, nullptr, ctx->st);
    } else {
      CK(cudaMemcpyAsync(q, qp, ctx->N * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
      hyrom_status s = newton_full<T>(ctx, qp, q);
      if (s) return s;
    }
    t_end(ctx, HYROM_T_FULL);
    inf.n_s = (int32_t)ctx->nc;
  } else {
    if (!ctx->has_basis) return fail(ctx, HYROM_ESTATE, "hybrid step %lld without a basis", (long long)k);
    inf.n_s = (int32_t)ctx->n_s;
    const T* psi = (const T*)ctx->psi;
    const T* phi = (const T*)ctx->phi;
    if (cf.scheme == HYROM_SCHEME_RK2) {
      t_begin(ctx, HYROM_T_PARTIAL);
      hy::launch_rk2<T>(ctx->dc, qp, q, k, ctx->shat, ctx->tiles, ctx->ntiles, ctx->st);
      t_end(ctx, HYROM_T_PARTIAL);
      t_begin(ctx, HYROM_T_GAPPY);
      if (ctx->m_eff > 0)
        gappy_y<T>(ctx, q, psi, ctx->y, nullptr, nullptr);
      t_end(ctx, HYROM_T_GAPPY);
      inf.J = 1;
      if (AdjTape* tp = ctx->tape) {  // the adjoint's record of this hybrid step
        const size_t N = (size_t)ctx->N, nw = (size_t)ctx->nwords;
        CK(cudaMemcpyAsync(tp->vpred + k * N, q, N * 8, cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaMemcpyAsync(tp->ys + k * 64, ctx->y, 64 * 8, cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaMemcpyAsync(tp->shats + k * nw, ctx->shat, nw * 4, cudaMemcpyDeviceToDevice,
                           ctx->st));
        CK(cudaMemcpyAsync(tp->rows + k * (size_t)cf.n_p, ctx->pts, (size_t)ctx->np_eff * 4,
                           cudaMemcpyDeviceToDevice, ctx->st));
        AdjStep& r = tp->rec[k];
        r.phi_ver = tp->cur_phi;
        r.psi_ver = tp->cur_psi;
        r.m_eff = ctx->m_eff;
        r.n_p = ctx->np_eff;
      }
    } else {
      CK(cudaMemcpyAsync(q, qp, ctx->N * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
      if (muscl)  // the cells of S-hat, ascending: the partial solve's unknowns
        hy::launch_bits_to_list(ctx->shat, ctx->nc, ctx->list_cnt, ctx->mus_cells, ctx->nc,
                                ctx->st);
      double* yv = ctx->y;
      double* yo = ctx->y2;
      double* hd = (double*)ctx->host;
      for (int j = 1; j <= cf.jmax; ++j) {
        t_begin(ctx, HYROM_T_PARTIAL);
        hyrom_status s = HYROM_OK;
        if (muscl) {
          if constexpr (sizeof(T) == 8)
            s = muscl_solve(ctx, q, qp, qp2, k, ctx->mus_cells, ctx->n_s);
        } else {
          s = newton_partial<T>(ctx, qp, q, ctx->shat, ctx->n_s);
        }
        t_end(ctx, HYROM_T_PARTIAL);
        if (s) return s;
        inf.J = j;
        if (ctx->m_eff == 0) {
          std::swap(yv, yo);
          break;
        }
        gappy_y<T>(ctx, q, psi, yv, j > 1 ? yo : nullptr, ctx->dy);
        CK(cudaMemcpyAsync(hd, ctx->dy, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        if (hyrom_status s2 = sync(ctx)) return s2;
        inf.dy_last = hd[0];
        std::swap(yv, yo);  // yo now holds y^(j)
        if (j > 1 && hd[0] < cf.eps_y) break;
        hy::launch_reconstruct<T>(phi, ctx->N, ctx->nc, ctx->m_eff, yo, psi, ctx->stilde, 1, q,
                                  ctx->st);
      }
      if (yo != ctx->y)
        CK(cudaMemcpyAsync(ctx->y, yo, ctx->m * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    }
    // reconstruction on S-breve
    t_begin(ctx, HYROM_T_RECON);
    hy::launch_reconstruct<T>(phi, ctx->N, ctx->nc, ctx->m_eff, ctx->y, psi, ctx->shat, 0, q,
                              ctx->st);
    t_end(ctx, HYROM_T_RECON);
    // SpatialFilter
    t_begin(ctx, HYROM_T_FILTER);
    if (cf.n_filt > 0 && muscl) {
      if constexpr (sizeof(T) == 8) {
        const int np = hy::muscl_filter(ctx->mus, ctx->dc, q, qp, qp2, k, cf.filt_orders, cf.n_filt,
                                        cf.jmax_f, cf.eps_f, (double*)ctx->fg,
                                        (double*)ctx->ftmp, (double*)ctx->rho_old,
                                        (double*)ctx->rho_new, ctx->fpart, ctx->dy + 2,
                                        (double*)ctx->host + 28, ctx->st);
        if (np < 0) return fail(ctx, HYROM_ECUDA, "filter: %s", cudaGetErrorString(cudaGetLastError()));
        ctx->muscl_passes = np;
      }
    } else if (cf.n_filt > 0) {
      AdjTape* tp = ctx->tape;
      const size_t nw = (size_t)ctx->nwords;
      hy::launch_filter_sparse<T>(ctx->dc, cf.filt_orders, cf.n_filt, cf.jmax_f, cf.eps_f, q, qp,
                                  k, (T*)ctx->fg, ctx->kbits, ctx->ftiles_a, ctx->ftiles_b,
                                  ctx->fcounts, ctx->fpart, ctx->fctl, ctx->fargs,
                                  &ctx->filt_graph, ctx->st,
                                  tp ? tp->keeps + (size_t)k * tp->passmax * nw : nullptr,
                                  tp ? tp->orders + (size_t)k * tp->passmax : nullptr,
                                  tp ? tp->npass + k : nullptr);
    }
    t_end(ctx, HYROM_T_FILTER);
  }
  // physical-state check of the new snapshot (Euler): rho > 0 and p > 0
  if (ctx->dc.nvar == 4) hy::launch_count_nonphys<T>(ctx->dc, q, ctx->fail_dev + 12, ctx->st);
  if (AdjTape* tp = ctx->tape) {  // the state and the output term of this step
    if constexpr (sizeof(T) == 8) {
      CK(cudaMemcpyAsync(tp->states + k * (size_t)ctx->N, q, (size_t)ctx->N * 8,
                         cudaMemcpyDeviceToDevice, ctx->st));
      hy::launch_box_pressure(ctx->dc, q, tp->box, tp->wgt, tp->Jpart, tp->J, ctx->st);
    }
    tp->rec[k].full = full;
  }
  CKL();
  ctx->k = k;
  gram_update<T>(ctx, k);
  int* hi = (int*)ctx->host;
  CK(cudaMemcpyAsync(hi, ctx->fail_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (!full && cf.n_filt > 0 && !muscl)
    CK(cudaMemcpyAsync(hi + 1, ctx->fctl + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(hi + 2, ctx->fail_dev + 12, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  inf.newton_fail = muscl ? ctx->muscl_fail : hi[0];
  inf.filt_passes = (!full && cf.n_filt > 0) ? (muscl ? ctx->muscl_passes : hi[1]) : 0;
  inf.n_p = ctx->np_eff;
  inf.m_eff = ctx->m_eff;
  if (info) *info = inf;
  if (hi[2])
    return fail(ctx, HYROM_ENONPHYS, "step %lld: %d cell(s) with rho <= 0 or p <= 0 or not finite",
                (long long)k, hi[2]);
  if (inf.newton_fail) return fail(ctx, HYROM_ENOTCONV, "Newton hit newton_max in %d solve(s)", inf.newton_fail);
  return HYROM_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 1, basis-update part: psi initialisation, rebuild test, selection,
// POD, ODEIM, sampling sets, psi update
// ---------------------------------------------------------------------------

constexpr bool kUseTensorBasisProduct = true;

// n ints from host memory to dev on the context stream, staged through the
// context's pinned scratch at byte offset off (bytes [1024, 4096) are kept for
// this): a copy from pageable memory would first wait for the stream to drain.
cudaError_t h2d_ints(hyrom_ctx* ctx, int* dev, const int* src, size_t n, size_t off) {
  if (off < 1024 || off + n * sizeof(int) > 4096)
    return cudaMemcpyAsync(dev, src, n * sizeof(int), cudaMemcpyHostToDevice, ctx->st);
  int* stage = (int*)((char*)ctx->host + off);
  memcpy(stage, src, n * sizeof(int));
  return cudaMemcpyAsync(dev, stage, n * sizeof(int), cudaMemcpyHostToDevice, ctx->st);
}

template <typename T>
hyrom_status pod_t(hyrom_ctx* ctx, const T* ring, int nslot, const std::vector<int>& win,
                   const T* psi, const std::vector<int>* psi_slots, T* phi_out, T* psi_next,
                   int* m_eff_host) {
  if (ctx->f32 && (const void*)ring == ctx->ring) gram_flush(ctx);
  const int w = (int)win.size();
  const int wp = w % 2 ? w + 1 : w;
  bool tc_used = false;
  CK(h2d_ints(ctx, ctx->win_dev, win.data(), (size_t)w, 1024));
  const hyrom_config& cf = ctx->cfg;
  if (!ctx->f32) {
    // FP64: one-sided Jacobi SVD of the centred window
    join_select(ctx);
    t_begin(ctx, HYROM_T_EIG);
    hy::launch_center_window<T>(ring, ctx->N, ctx->win_dev, w, wp, psi, ctx->X, ctx->rawpart,
                                ctx->xraw2, ctx->st);
    hy::launch_identity(ctx->V, wp, ctx->st);
    int* hi = (int*)ctx->host;
    for (int sweep = 0; sweep < 60; ++sweep) {
      CK(cudaMemsetAsync(ctx->rotated, 0, sizeof(int), ctx->st));
      for (int r = 0; r < wp - 1; ++r)
        hy::launch_hestenes_round(ctx->X, ctx->N, wp, ctx->V, r, 1e-15, ctx->rotated, ctx->jbuf,
                                  ctx->st);
      CK(cudaMemcpyAsync(hi, ctx->rotated, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
      if (hyrom_status s = sync(ctx)) return s;
      if (!hi[0]) break;
    }
    t_end(ctx, HYROM_T_EIG);
    t_begin(ctx, HYROM_T_FORMPHI);
    hy::launch_colnorm2(ctx->X, ctx->N, wp, ctx->lam, ctx->st);
    hy::launch_pod_coeffs<double>(ctx->lam, nullptr, wp, wp, cf.m, cf.pod_tol, cf.pod_abs,
                                  ctx->xraw2, ctx->sig, ctx->m_eff_dev, ctx->Cd, ctx->st);
    hy::launch_phi_from_columns<T>(ctx->X, ctx->N, wp, ctx->Cd, ctx->m_eff_dev, cf.m, phi_out,
                                   ctx->st);
    if (psi_next) hy::launch_window_mean<T>(ring, ctx->N, ctx->win_dev, w, psi_next, ctx->st);
    t_end(ctx, HYROM_T_FORMPHI);
  } else {
    // FP32: raw ring Gram, centred by the identity, FP64 Jacobi
    t_begin(ctx, HYROM_T_EIG);
    bool ident_ok = psi_slots != nullptr;
    if (ident_ok) {
      CK(h2d_ints(ctx, ctx->ps_dev, psi_slots->data(), psi_slots->size(), 2048));
      hy::launch_gram_center(ctx->H, nslot, ctx->win_dev, w, ctx->ps_dev, (int)psi_slots->size(),
                             ctx->Gc, wp, ctx->xraw2, ctx->st);
    } else {
      hy::launch_dots<T>(psi, ring, ctx->N, nslot, ctx->Hpart, ctx->gram_chunks, ctx->hp, ctx->st);
      hy::launch_dots<T>(psi, psi, ctx->N, 1, ctx->Hpart, ctx->gram_chunks, ctx->pp, ctx->st);
      hy::launch_gram_center_explicit(ctx->H, nslot, ctx->win_dev, w, ctx->hp, ctx->pp, ctx->Gc,
                                      wp, ctx->xraw2, ctx->st);
    }
    if (hy::run_psd_eig(ctx->Gc, wp, ctx->V, ctx->lam, ctx->jbuf, ctx->rotated,
                        (int*)ctx->host + 8, 60, ctx->st, nullptr, true) < 0)
      return fail(ctx, HYROM_ECUDA, "Jacobi eigensolver: %s", cudaGetErrorString(cudaGetLastError()));
    hy::launch_pod_coeffs<T>(ctx->lam, ctx->V, wp, w, cf.m, cf.pod_tol, cf.pod_abs, ctx->xraw2,
                             ctx->sig, ctx->m_eff_dev, (T*)ctx->C, ctx->st);
    t_end(ctx, HYROM_T_EIG);
    join_select(ctx);  // the selection has read the old basis
    t_begin(ctx, HYROM_T_FORMPHI);
    if constexpr (sizeof(T) == 4) {
      if (kUseTensorBasisProduct && hy::form_phi_tc_ok(ctx->N, w, cf.m)) {
        // tensor-core product; its bounded waits report through fail_dev[4].
        // For the context's own basis its epilogue also forms ODEIM's
        // row-norm data, so the rebuild's ODEIM skips that pass over Phi.
        CK(cudaMemsetAsync(ctx->fail_dev + 4, 0, sizeof(int), ctx->st));
        hy::OdeimNorms nout = {nullptr, nullptr, nullptr, nullptr};
        if (phi_out == (T*)ctx->phi) {
          nout = hy::odeim_norm_bufs(ctx->od_ws, ctx->N);
          CK(cudaMemsetAsync(nout.bcnt, 0, (hy::kNormBucketCount + 1) * sizeof(int), ctx->st));
          CK(cudaMemsetAsync(nout.bmax, 0, hy::kNormBucketCount * sizeof(int), ctx->st));
        }
        hy::launch_form_phi_tc(ring, ctx->N, nslot, ctx->win_dev, w, psi, (const float*)ctx->C,
                               cf.m, ctx->m_eff_dev, phi_out,
                               psi_next ? psi_next : (T*)ctx->fg, ctx->fail_dev + 4, nout,
                               ctx->st);
        ctx->norms_ready = nout.nrm != nullptr;
        tc_used = true;
      }
    }
    if (!tc_used)
      hy::launch_form_phi<T>(ring, ctx->N, ctx->win_dev, w, psi, (const T*)ctx->C, cf.m,
                             ctx->m_eff_dev, phi_out, psi_next ? psi_next : (T*)ctx->fg, ctx->st);
    t_end(ctx, HYROM_T_FORMPHI);
  }
  // column signs: normalised on the FP64 path (direct basis comparison);
  // the method is invariant to them, so the FP32 path skips the extra pass
  if (!ctx->f32) hy::launch_sign_fix<T>(phi_out, ctx->N, cf.m, ctx->m_eff_dev, ctx->st);
  CKL();
  int* hi = (int*)ctx->host;
  CK(cudaMemcpyAsync(hi, ctx->m_eff_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  hi[1] = 0;
  if (tc_used)
    CK(cudaMemcpyAsync(hi + 1, ctx->fail_dev + 4, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  if (hi[1]) return fail(ctx, HYROM_ETIMEOUT, "basis product: a pipeline wait timed out");
  *m_eff_host = hi[0];
  return HYROM_OK;
}

template <typename T>
hyrom_status masks_and_tiles(hyrom_ctx* ctx, const uint32_t* gbm, const int* pts, int np,
                             uint32_t* shat, uint32_t* stilde, int64_t* n_s) {
  // stencil reach: one cell for first-order BDF1, two for SSP-RK2 (two
  // stages) and for MUSCL (two neighbours per face)
  const int rs = ctx->cfg.scheme == HYROM_SCHEME_BE ? 1 : 2;
  t_begin(ctx, HYROM_T_MASKS);
  hy::launch_masks(ctx->dc, gbm, pts, np, ctx->cfg.halo, rs, ctx->base_bm, shat, stilde,
                   ctx->n_s_dev, ctx->st);
  t_end(ctx, HYROM_T_MASKS);
  CKL();
  long long* hl = (long long*)ctx->host;
  CK(cudaMemcpyAsync(hl, ctx->n_s_dev, sizeof(long long), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  *n_s = hl[0];
  return HYROM_OK;
}

template <typename T>
hyrom_status rebuild_tail_t(hyrom_ctx* ctx, hyrom_step_info inf, const uint32_t* gbm, int me,
                            int np, hyrom_step_info* info);

template <typename T>
hyrom_status update_basis_t(hyrom_ctx* ctx, hyrom_step_info* info) {
  const hyrom_config& cf = ctx->cfg;
  const int64_t k = ctx->k;
  const int w = cf.w;
  hyrom_step_info inf;
  if (info)
    inf = *info;
  else
    memset(&inf, 0, sizeof inf);
  inf.k = k;
  if (k == w - 1) {  // psi initialisation: psi_{w-1} = mean(gamma_0..gamma_{w-1})
    std::vector<int> win(w);
    ctx->psi_steps.clear();
    for (int i = 0; i < w; ++i) {
      win[i] = slot_of(ctx, i);
      ctx->psi_steps.push_back(i);
    }
    CK(cudaMemcpyAsync(ctx->win_dev, win.data(), w * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
    hy::launch_window_mean<T>((const T*)ctx->ring, ctx->N, ctx->win_dev, w, (T*)ctx->psi, ctx->st);
    ctx->psi_set = 1;
    if (AdjTape* tp = ctx->tape) {  // version: psi_{w-1}
      double* v = nullptr;
      CK(cudaMalloc((void**)&v, (size_t)ctx->N * 8));
      CK(cudaMemcpyAsync(v, ctx->psi, (size_t)ctx->N * 8, cudaMemcpyDeviceToDevice, ctx->st));
      tp->psis.push_back(v);
      tp->cur_psi = (int)tp->psis.size() - 1;
      tp->rec[k].psi_init = true;
      tp->rec[k].init_psi = tp->cur_psi;
    }
  }
  const bool due = k >= w - 1 && (cf.z <= 0 || (k + 1) % cf.z != 0);
  if (!due) {
    inf.n_p = ctx->np_eff;
    inf.m_eff = ctx->m_eff;
    if (info) *info = inf;
    return sync(ctx);
  }
  if (!ctx->psi_set) return fail(ctx, HYROM_ESTATE, "no reference state at step %lld", (long long)k);
  inf.rebuilt = 1;
  const T* gk = ring_at<T>(ctx, k);
  // selection: G_{k+1} from the reconstruction error of the final gamma_k
  const uint32_t* gbm = nullptr;
  int64_t n_g = 0;
  // (on st2, beside the eigensolve: it reads the old basis, which the
  // rebuild overwrites only after joining it)
  long long* hl = (long long*)((char*)ctx->host + 128);
  if (k >= w && ctx->has_basis) {
    cudaStream_t ss = ctx->st2;
    CK(cudaEventRecord(ctx->ev_fork, ctx->st));
    CK(cudaStreamWaitEvent(ss, ctx->ev_fork, 0));
    t_begin(ctx, HYROM_T_SELECT, ss);
    if (ctx->m_eff > 0)
      gappy_y<T>(ctx, gk, (const T*)ctx->psi, ctx->y2, nullptr, nullptr, ss);
    hy::launch_cell_error<T>(gk, (const T*)ctx->psi, (const T*)ctx->phi, ctx->nc, ctx->dc.nvar,
                             ctx->m_eff, ctx->y2, (T*)ctx->eps, ss);
    hy::launch_select(ctx->eps, ctx->f32, ctx->nc, cf.sel_mode, cf.delta, cf.top_frac, ctx->keys,
                      ctx->sel_scratch, ctx->g_bm, ctx->n_g_dev, ss);
    t_end(ctx, HYROM_T_SELECT, ss);
    CKL();
    CK(cudaMemcpyAsync(hl, ctx->n_g_dev, sizeof(long long), cudaMemcpyDeviceToHost, ss));
    CK(cudaEventRecord(ctx->ev_join, ss));
    ctx->sel_pending = true;
    gbm = ctx->g_bm;
  }
  inf.n_g = (int32_t)n_g;
  // POD of the window centred at the psi in effect
  std::vector<int> win(w);
  for (int i = 0; i < w; ++i) win[i] = slot_of(ctx, k - w + 1 + i);
  std::vector<int> ps;
  bool ps_ok = true;
  for (int64_t j : ctx->psi_steps) {
    if (j < k - w) ps_ok = false;
    ps.push_back(slot_of(ctx, j));
  }
  int me = 0;
  hyrom_status s = pod_t<T>(ctx, (const T*)ctx->ring, ctx->nslot, win, (const T*)ctx->psi,
                            ps_ok ? &ps : nullptr, (T*)ctx->phi, (T*)ctx->psi_next, &me);
  join_select(ctx);
  if (s) return s;
  if (gbm) {  // pod_t synchronised ctx->st after joining the selection
    n_g = hl[0];
    inf.n_g = (int32_t)n_g;
  }
  ctx->m_eff = me;
  // ODEIM points
  ctx->np_eff = 0;
  int np = 0;
  if (me > 0) {
    np = cf.n_p;
    if (np > ctx->N) np = (int)ctx->N;
    t_begin(ctx, HYROM_T_DEIM);
    const bool nr = ctx->norms_ready;
    ctx->norms_ready = false;
    hy::OdeimOver* ov = ctx->defer_over ? &ctx->over : nullptr;
    if (ov && ov->m_cap < cf.m) ov->m_cap = cf.m < 64 ? cf.m : 64;
    if (hy::launch_odeim<T>((const T*)ctx->phi, ctx->N, me, np, cf.tie_tol, ctx->pts,
                            ctx->od_ws, (char*)ctx->host + 256, ctx->st, &odeim_mark, ctx,
                            nr, &ctx->od_graphs, ov, cf.odeim_batch) < 0)
      return fail(ctx, HYROM_ECUDA, "ODEIM: %s", cudaGetErrorString(cudaGetLastError()));
    if (ov && ov->active) {  // finish_rebuild completes the step
      ctx->pend.on = true;
      ctx->pend.inf = inf;
      ctx->pend.gbm = gbm;
      ctx->pend.me = me;
      ctx->pend.np = np;
      if (info) *info = inf;
      return HYROM_OK;
    }
  }
  return rebuild_tail_t<T>(ctx, inf, gbm, me, np, info);
}

// The rebuild after its ODEIM points: the sampled pseudo-inverse, the
// sampling sets, the sample-row normal matrix, the tiles and the psi
// update (Algorithm 1, after the greedy selection of the points).
template <typename T>
hyrom_status rebuild_tail_t(hyrom_ctx* ctx, hyrom_step_info inf, const uint32_t* gbm, int me,
                            int np, hyrom_step_info* info) {
  const hyrom_config& cf = ctx->cfg;
  const int64_t k = ctx->k;
  const int w = cf.w;
  hyrom_status s;
  if (me > 0) {
    ctx->np_eff = np;
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->st));
    hy::launch_gappy_pinv<T>((const T*)ctx->phi, ctx->N, me, ctx->pts, np, ctx->pinv,
                             ctx->status, ctx->st);
    t_end(ctx, HYROM_T_ODEIM);
  }
  // sampling sets
  if ((s = masks_and_tiles<T>(ctx, gbm, ctx->pts, ctx->np_eff, ctx->shat, ctx->stilde, &ctx->n_s)))
    return s;
  // sample-row form: normal matrix of the new basis on the new S-hat
  ctx->sample_ok = false;
  if (cf.regress_rows == HYROM_ROWS_SAMPLE && me > 0 && ctx->n_s > 0) {
    t_begin(ctx, HYROM_T_SNORMAL);
    hy::launch_bits_to_list(ctx->shat, ctx->nc, ctx->list_cnt, ctx->s_cells, ctx->nc, ctx->st);
    CK(cudaMemsetAsync(ctx->fail_dev + 8, 0, 2 * sizeof(int), ctx->st));
    hy::launch_sample_normal<T>((const T*)ctx->phi, ctx->N, me, ctx->s_cells, (int)ctx->n_s,
                                ctx->dc.nvar, ctx->nc, cf.reduced_prec, ctx->s_part, ctx->s_G,
                                ctx->s_L, ctx->s_dinv, ctx->fail_dev + 8, ctx->st);
    t_end(ctx, HYROM_T_SNORMAL);
    int* hf = (int*)ctx->host + 12;
    CK(cudaMemcpyAsync(hf, ctx->fail_dev + 8, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    if ((s = sync(ctx))) return s;
    if (hf[1]) return fail(ctx, HYROM_ETIMEOUT, "sample-row normal matrix: a device wait gave up");
    // a sample set that does not determine y falls back to the ODEIM rows
    ctx->sample_ok = hf[0] == 0;
  }
  if (cf.scheme == HYROM_SCHEME_RK2)
    hy::launch_active_tiles(ctx->dc, ctx->shat, hy::rk2_tile_width(ctx->dc),
                            hy::rk2_tile_height(ctx->dc), ctx->tiles, ctx->ntiles, ctx->st);
  // psi update: psi_{k+1} = mean of the window
  std::swap(ctx->psi, ctx->psi_next);
  if (AdjTape* tp = ctx->tape) {  // this rebuild: its window and versions
    AdjStep& r = tp->rec[k];
    r.rebuild = true;
    r.psi_cur = tp->cur_psi;
    double* v = nullptr;
    CK(cudaMalloc((void**)&v, (size_t)ctx->N * 8));
    CK(cudaMemcpyAsync(v, ctx->psi, (size_t)ctx->N * 8, cudaMemcpyDeviceToDevice, ctx->st));
    tp->psis.push_back(v);
    r.new_psi = tp->cur_psi = (int)tp->psis.size() - 1;
    r.new_phi = tp->cur_phi = tp->nphi++;
    r.m_eff = me;
  }
  ctx->psi_steps.clear();
  for (int i = 0; i < w; ++i) ctx->psi_steps.push_back(k - w + 1 + i);
  ctx->has_basis = 1;
  CKL();
  int* hq = (int*)ctx->host + 16;
  hq[0] = 0;
  if (me > 0) CK(cudaMemcpyAsync(hq, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if ((s = sync(ctx))) return s;
  inf.n_p = ctx->np_eff;
  inf.m_eff = ctx->m_eff;
  if (info) *info = inf;
  // information: the step is complete, with fewer modes than asked for or
  // a rank-deficient P^T Phi (its solve is truncated)
  if (me < cf.m)
    return fail(ctx, HYROM_ERANK, "step %lld: the window has rank %d < m = %d (POD kept %d modes)",
                (long long)k, me, cf.m, me);
  if (hq[0]) return fail(ctx, HYROM_ERANK, "step %lld: P^T Phi is rank-deficient", (long long)k);
  return HYROM_OK;
}

template <typename T>
hyrom_status init_state(hyrom_ctx* ctx, const double* q0, int on_host) {
  T* g0 = ring_at<T>(ctx, 0);
  if (!ctx->f32) {
    CK(cudaMemcpyAsync(g0, q0, ctx->N * sizeof(double),
                       on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->st));
  } else {
    // convert through the filter scratch (device) buffer
    double* tmp = (double*)ctx->X;
    CK(cudaMemcpyAsync(tmp, q0, ctx->N * sizeof(double),
                       on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->st));
    convert_f64_to_f32(tmp, (float*)g0, ctx->N, ctx->st);
  }
  gram_update<T>(ctx, 0);
  CKL();
  return sync(ctx);
}

}  // namespace

// ---------------------------------------------------------------------------
// public entry points
// ---------------------------------------------------------------------------

namespace hy {
void* ctx_stream(const hyrom_ctx* ctx) { return ctx ? (void*)ctx->st : nullptr; }
void ctx_set_defer(hyrom_ctx* ctx, bool on) {
  if (ctx) ctx->defer_over = on;
}
const OdeimOver* ctx_pending_over(const hyrom_ctx* ctx) {
  return ctx && ctx->pend.on ? &ctx->over : nullptr;
}
bool ctx_is_f32(const hyrom_ctx* ctx) { return ctx && ctx->f32; }
void ctx_drop_pending(hyrom_ctx* ctx) {
  if (ctx) ctx->pend.on = false;
}
hyrom_status ctx_finish_rebuild(hyrom_ctx* ctx, hyrom_step_info* info) {
  if (!ctx || !ctx->pend.on) return HYROM_OK;
  ctx->pend.on = false;
  if (ctx->sticky) return HYROM_ECUDA;
  const auto& p = ctx->pend;
  return ctx->f32 ? rebuild_tail_t<float>(ctx, p.inf, p.gbm, p.me, p.np, info)
                  : rebuild_tail_t<double>(ctx, p.inf, p.gbm, p.me, p.np, info);
}
}  // namespace hy

extern "C" {

hyrom_status hyrom_init(const hyrom_config* cfg, const double* q0, int q0_on_host, void* stream,
                        hyrom_ctx** out) {
  if (!cfg || !q0 || !out) return HYROM_EINVAL;
  char why[256];
  if (validate(cfg, why, sizeof why) != HYROM_OK) {
    fprintf(stderr, "hyrom_init: invalid configuration: %s\n", why);
    return HYROM_EINVAL;
  }
  hyrom_ctx* ctx = new hyrom_ctx();
  ctx->cfg = *cfg;
  ctx->dc = hy::make_devcfg(*cfg);
  ctx->st = (cudaStream_t)stream;
  ctx->f32 = cfg->precision == HYROM_PREC_F32;
  ctx->esz = ctx->f32 ? 4 : 8;
  ctx->N = ctx->dc.ndof;
  ctx->nc = ctx->dc.nc;
  ctx->nwords = (ctx->nc + 31) / 32;
  ctx->w = cfg->w;
  ctx->m = cfg->m;
  ctx->np = cfg->n_p;
  ctx->nslot = cfg->w + 1;
  ctx->wp = (cfg->w + 1) % 2 ? cfg->w + 2 : cfg->w + 1;  // even, >= w + 1
  const int64_t N = ctx->N, nc = ctx->nc, nw = ctx->nwords;
  const size_t es = ctx->esz;
  const int wp = ctx->wp, m = ctx->m;
  ctx->gram_chunks = 1024;
  const int ntiles_max = (int)(((cfg->nx + 31) / 32 + 1) * ((cfg->ny + 7) / 8 + 1) + (cfg->nx + 255) / 256 + 1);
  ctx->ntiles_max = ntiles_max;
  bool ok = true;
  ok &= dalloc(ctx, &ctx->ring, (size_t)ctx->nslot * N * es);
  ok &= dalloc(ctx, &ctx->psi, N * es);
  ok &= dalloc(ctx, &ctx->psi_next, N * es);
  ok &= dalloc(ctx, &ctx->phi, (size_t)N * m * es);
  ok &= dal(ctx, &ctx->pts, 1024 * sizeof(int));
  ok &= dal(ctx, &ctx->pinv, (size_t)m * cfg->n_p * sizeof(double));
  if (cfg->regress_rows == HYROM_ROWS_SAMPLE) {
    ok &= dal(ctx, &ctx->s_cells, (size_t)nc * sizeof(int));
    ok &= dal(ctx, &ctx->s_part, hy::sample_part_doubles() * sizeof(double));
    ok &= dal(ctx, &ctx->s_G, 4096 * sizeof(double));
    ok &= dal(ctx, &ctx->s_L, 4096 * sizeof(double));
    ok &= dal(ctx, &ctx->s_dinv, 64 * sizeof(double));
    ok &= dal(ctx, &ctx->s_b, 64 * sizeof(double));
  }
  ok &= dal(ctx, &ctx->y, 256 * sizeof(double));
  ok &= dal(ctx, &ctx->y2, 256 * sizeof(double));
  ok &= dal(ctx, &ctx->dy, 64);
  ok &= dal(ctx, &ctx->status, 64);
  ok &= dal(ctx, &ctx->g_bm, nw * 4);
  ok &= dal(ctx, &ctx->base_bm, nw * 4);
  ok &= dal(ctx, &ctx->shat, nw * 4);
  ok &= dal(ctx, &ctx->stilde, nw * 4);
  ok &= dal(ctx, &ctx->tmp_bm, nw * 4);
  ok &= dal(ctx, &ctx->tiles, (size_t)ntiles_max * sizeof(int));
  ok &= dal(ctx, &ctx->ntiles, 64);
  ok &= dal(ctx, &ctx->seg, (size_t)cfg->nx * sizeof(int));
  ok &= dal(ctx, &ctx->nseg, 64);
  ok &= dal(ctx, &ctx->n_s_dev, 64);
  ok &= dal(ctx, &ctx->n_g_dev, 64);
  ok &= dal(ctx, &ctx->list_cnt, 1024 * sizeof(long long));
  ok &= dalloc(ctx, &ctx->fg, N * es);
  ok &= dalloc(ctx, &ctx->ftmp, N * es);
  ok &= dalloc(ctx, &ctx->rho_old, nc * es);
  ok &= dalloc(ctx, &ctx->rho_new, nc * es);
  ok &= dal(ctx, &ctx->fpart, 3 * 152 * 8 * sizeof(double));
  ok &= dal(ctx, &ctx->kbits, nw * 4);
  ok &= dal(ctx, &ctx->ftiles_a, (size_t)ntiles_max * sizeof(int));
  // the second tile list, then the filter's per-tile claim stamps
  ok &= dal(ctx, &ctx->ftiles_b, (size_t)2 * ntiles_max * sizeof(int));
  ok &= dal(ctx, &ctx->fcounts, 64);
  ok &= dal(ctx, &ctx->fctl, 64);
  ok &= dalloc(ctx, &ctx->eps, nc * es);
  ok &= dal(ctx, &ctx->keys, nc * sizeof(unsigned long long));
  ok &= dalloc(ctx, &ctx->sel_scratch, hy::select_scratch_bytes());
  ok &= dal(ctx, &ctx->H, (size_t)ctx->nslot * ctx->nslot * sizeof(double));
  ok &= dal(ctx, &ctx->Hpart, (size_t)(2 * ctx->nslot + 1) * ctx->gram_chunks * sizeof(double));
  ok &= dal(ctx, &ctx->hp, (size_t)(ctx->nslot + 1) * sizeof(double));
  ok &= dal(ctx, &ctx->pp, 64);
  ok &= dal(ctx, &ctx->Gc, (size_t)wp * wp * sizeof(double));
  ok &= dal(ctx, &ctx->V, (size_t)wp * wp * sizeof(double));
  ok &= dal(ctx, &ctx->lam, (size_t)wp * sizeof(double));
  ok &= dal(ctx, &ctx->sig, (size_t)wp * sizeof(double));
  ok &= dal(ctx, &ctx->xraw2, 64);
  {
    // the eigensolver's work array (FP32 POD), or the FP64 Jacobi rounds'
    // partial sums and rotations
    size_t a = (size_t)2 * wp * wp + 512;
    const size_t b = hy::hestenes_scratch_doubles(wp), c2 = hy::psd_eig_scratch_doubles(wp);
    if (c2 > a) a = c2;
    ok &= dal(ctx, &ctx->jbuf, (a > b ? a : b) * sizeof(double));
  }
  ok &= dal(ctx, &ctx->m_eff_dev, 64);
  ok &= dalloc(ctx, &ctx->C, (size_t)wp * m * es);
  ok &= dal(ctx, &ctx->Cd, (size_t)wp * m * sizeof(double));
  ok &= dal(ctx, &ctx->win_dev, 256 * sizeof(int));
  ok &= dal(ctx, &ctx->ps_dev, 256 * sizeof(int));
  // FP64 path: centred window for the one-sided Jacobi; FP32 path: q0 staging
  ok &= dal(ctx, &ctx->X, ctx->f32 ? (size_t)N * sizeof(double) : (size_t)N * wp * sizeof(double));
  ok &= dal(ctx, &ctx->rawpart, 152 * 4 * sizeof(double));
  ok &= dal(ctx, &ctx->rotated, 64);
  ok &= dalloc(ctx, &ctx->fargs, 64);
  if (ok) ok &= cudaMemsetAsync(ctx->rotated, 0, 64, ctx->st) == cudaSuccess;
  ok &= dal(ctx, &ctx->ident, (size_t)wp * wp * sizeof(double));
  ok &= dalloc(ctx, &ctx->od_ws, hy::odeim_ws_bytes(N, m));
  if (ok) ok &= cudaMemsetAsync(ctx->od_ws, 0, 256, ctx->st) == cudaSuccess;  // control block
  ok &= dal(ctx, &ctx->tol_dev, 64);
  ok &= dal(ctx, &ctx->newton_ws, (size_t)6 * cfg->nx * sizeof(double));
  ok &= dal(ctx, &ctx->fail_dev, 64);
  if (ok && cfg->scheme == HYROM_SCHEME_BDF2_MUSCL) {
    ok &= dal(ctx, &ctx->mus_cells, (size_t)nc * sizeof(int));
    ctx->mus = hy::muscl_create(nc, nc);
    ok &= ctx->mus != nullptr;
    ctx->bytes += hy::muscl_bytes(ctx->mus);
  }
  if (!ok) {
    hyrom_destroy(ctx);
    fprintf(stderr, "hyrom_init: device allocation failed\n");
    return HYROM_ENOMEM;
  }
  if (cudaMallocHost(&ctx->host, 4096) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->st2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    hyrom_destroy(ctx);
    return HYROM_ENOMEM;
  }
  std::vector<double> id((size_t)wp * wp, 0.0);
  for (int i = 0; i < wp; ++i) id[(size_t)i * wp + i] = 1.0;
  hyrom_status s = HYROM_OK;
  if (cudaMemcpy(ctx->ident, id.data(), id.size() * sizeof(double), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(ctx->H, 0, (size_t)ctx->nslot * ctx->nslot * sizeof(double)) != cudaSuccess ||
      cudaMemset(ctx->ftiles_b, 0, (size_t)2 * ntiles_max * sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->fctl, 0, 64) != cudaSuccess) {
    s = HYROM_ECUDA;
  }
  if (s == HYROM_OK) s = ctx->f32 ? init_state<float>(ctx, q0, q0_on_host)
                                  : init_state<double>(ctx, q0, q0_on_host);
  if (s != HYROM_OK) {
    fprintf(stderr, "hyrom_init: %s\n", ctx->err.c_str());
    hyrom_destroy(ctx);
    return s;
  }
  *out = ctx;
  return HYROM_OK;
}

void hyrom_destroy(hyrom_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  if (ctx->st2) {
    cudaStreamSynchronize(ctx->st2);
    cudaStreamDestroy(ctx->st2);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  hy::odeim_graphs_free(&ctx->od_graphs);
  hy::graph_slot_free(&ctx->filt_graph);
  hy::muscl_destroy(ctx->mus);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->host) cudaFreeHost(ctx->host);
  for (int i = 0; i < HYROM_NSTAGE; ++i) {
    if (!ctx->ev_a[i]) continue;
    for (int j = 0; j < hyrom_ctx::kEvPairs; ++j) {
      cudaEventDestroy(ctx->ev_a[i][j]);
      cudaEventDestroy(ctx->ev_b[i][j]);
    }
    delete[] ctx->ev_a[i];
    delete[] ctx->ev_b[i];
  }
  delete ctx;
}

const char* hyrom_last_error(const hyrom_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t hyrom_device_bytes(const hyrom_ctx* ctx) { return ctx ? ctx->bytes : 0; }

uint64_t hyrom_kernel_launches(void) { return hy::launch_count(); }

hyrom_status hyrom_profile(hyrom_ctx* ctx, int on) {
  if (!ctx) return HYROM_EINVAL;
  if (on && !ctx->ev_a[0]) {
    for (int i = 0; i < HYROM_NSTAGE; ++i) {
      ctx->ev_a[i] = new cudaEvent_t[hyrom_ctx::kEvPairs];
      ctx->ev_b[i] = new cudaEvent_t[hyrom_ctx::kEvPairs];
      for (int j = 0; j < hyrom_ctx::kEvPairs; ++j) {
        CK(cudaEventCreate(&ctx->ev_a[i][j]));
        CK(cudaEventCreate(&ctx->ev_b[i][j]));
      }
    }
  }
  ctx->profile = on ? 1 : 0;
  for (int i = 0; i < HYROM_NSTAGE; ++i) {
    ctx->stage_ms[i] = 0.0;
    ctx->stage_n[i] = 0;
    ctx->ev_used[i] = 0;
    ctx->ev_open[i] = 0;
  }
  return HYROM_OK;
}

hyrom_status hyrom_odeim_counters(hyrom_ctx* ctx, int64_t* out4) {
  if (!ctx || !out4) return HYROM_EINVAL;
  if (ctx->sticky) return HYROM_ECUDA;
  unsigned long long* h = (unsigned long long*)ctx->host;
  hy::odeim_stats(ctx->od_ws, h, ctx->st);
  if (hyrom_status s = sync(ctx)) return s;
  for (int i = 0; i < 4; ++i) out4[i] = (int64_t)h[i];
  return HYROM_OK;
}

hyrom_status hyrom_eig_sweeps(hyrom_ctx* ctx, int32_t* out2) {
  if (!ctx || !out2) return HYROM_EINVAL;
  if (ctx->sticky) return HYROM_ECUDA;
  int* h = (int*)ctx->host;
  CK(cudaMemcpyAsync(h, ctx->rotated + 4, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  hy::odeim_eig_sweeps(ctx->od_ws, h + 1, ctx->st);
  if (hyrom_status s = sync(ctx)) return s;
  out2[0] = h[0];
  out2[1] = h[1];
  return HYROM_OK;
}

hyrom_status hyrom_stage_times(const hyrom_ctx* ctx, double* ms, int64_t* count) {
  if (!ctx || !ms) return HYROM_EINVAL;
  for (int i = 0; i < HYROM_NSTAGE; ++i) {
    ms[i] = ctx->stage_ms[i];
    if (count) count[i] = ctx->stage_n[i];
  }
  return HYROM_OK;
}

#define GUARD()                                                              \
  do {                                                                       \
    if (!ctx) return HYROM_EINVAL;                                           \
    if (ctx->sticky) return HYROM_ECUDA;                                     \
  } while (0)

hyrom_status hyrom_advance(hyrom_ctx* ctx, hyrom_step_info* info) {
  GUARD();
  return ctx->f32 ? advance_t<float>(ctx, info) : advance_t<double>(ctx, info);
}

hyrom_status hyrom_update_basis(hyrom_ctx* ctx, hyrom_step_info* info) {
  GUARD();
  return ctx->f32 ? update_basis_t<float>(ctx, info) : update_basis_t<double>(ctx, info);
}

hyrom_status hyrom_step(hyrom_ctx* ctx, hyrom_step_info* info) {
  GUARD();
  hyrom_step_info inf;
  memset(&inf, 0, sizeof inf);
  hyrom_status s = hyrom_advance(ctx, &inf);
  if (s != HYROM_OK && s != HYROM_ENOTCONV && s != HYROM_ENONPHYS) return s;
  hyrom_status s2 = hyrom_update_basis(ctx, &inf);
  if (info) *info = inf;
  // a failure of the rebuild first, then the advance's own condition, then
  // the rebuild's rank information
  if (s2 != HYROM_OK && s2 != HYROM_ERANK) return s2;
  if (s != HYROM_OK) return s;
  return s2;
}

// ---- the reverse sweep (hyrom_adjoint) -------------------------------------------
namespace {

__global__ void k_add_into(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

void add_into(const double* x, double* y, int64_t n, cudaStream_t s) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  k_add_into<<<(int)(b < 1 ? 1 : b), 256, 0, HY_S(s)>>>(x, y, n);
}

void free_tape(AdjTape* tp) {
  if (!tp) return;
  cudaFree(tp->states);
  cudaFree(tp->vpred);
  cudaFree(tp->ys);
  cudaFree(tp->shats);
  cudaFree(tp->rows);
  cudaFree(tp->keeps);
  cudaFree(tp->orders);
  cudaFree(tp->npass);
  cudaFree(tp->Jpart);
  cudaFree(tp->J);
  for (double* v : tp->psis) cudaFree(v);
  delete tp;
}

// The POD of version v recomputed from its window (the same kernels on the
// same inputs as the forward rebuild, so the same bits): phi_out gets Phi,
// ctx->X the rotated window columns (U Sigma, unsorted), ctx->V their right
// vectors, ctx->lam the squared column norms.
hyrom_status recompute_pod(hyrom_ctx* ctx, AdjTape* tp, int k_rebuild, int psi_cur, double* phi_out,
                           int* me) {
  const int w = ctx->cfg.w;
  const size_t N = (size_t)ctx->N;
  std::vector<int> win(w);
  for (int c = 0; c < w; ++c) {
    win[c] = c;
    CK(cudaMemcpyAsync((double*)ctx->ring + (size_t)c * N, tp->states + (size_t)(k_rebuild - w + 1 + c) * N,
                       N * 8, cudaMemcpyDeviceToDevice, ctx->st));
  }
  return pod_t<double>(ctx, (const double*)ctx->ring, ctx->nslot, win, tp->psis[psi_cur], nullptr,
                       phi_out, nullptr, me);
}

// The thin-SVD adjoint of a rebuild (Sec. 2.3.1, Eq. pod; distinct singular
// values): with the POD's window columns X = U Sigma V^T (ctx->X, ->V, ->lam
// after recompute_pod) and the cotangent L of Phi's m kept columns (Phi_j =
// g_j U_j, g_j the sign that makes Phi's largest entry positive),
//   lam_X = sum_j [(l_j - U U^T l_j) / s_j] V_j^T
//         + sum_j sum_{i != j} c_ij (s_j U_i V_j^T + s_i U_j V_i^T),
//   c_ij = (U_i . l_j) / (s_j^2 - s_i^2),
// written as lam_X = L B1 + X B2 with small B1 (m x w), B2 (wp x w) formed on
// the host; then lam_{window} += lam_X + lpsi_new / w, lpsi_cur -= sum_c lam_X.
hyrom_status pod_vjp(hyrom_ctx* ctx, AdjTape* tp, int k_rebuild, const double* phi, int m,
                     const double* lphi, const double* lpsi_new, double* lpsi_cur, double* lam,
                     double* part) {
  // the POD's own column count: the window padded to an even width
  const int w = ctx->cfg.w, wp = w % 2 ? w + 1 : w;
  const int64_t N = ctx->N;
  std::vector<double> lam2(wp), V((size_t)wp * wp), D1((size_t)wp * std::max(m, 1)),
      D2((size_t)wp * std::max(m, 1));
  CK(cudaMemcpyAsync(lam2.data(), ctx->lam, wp * 8, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(V.data(), ctx->V, (size_t)wp * wp * 8, cudaMemcpyDeviceToHost, ctx->st));
  double* dev_small = part + hy::tsdots_part_doubles(wp, m);
  if (m > 0) {
    hy::launch_tsdots(ctx->X, wp, lphi, m, N, part, dev_small, ctx->st);
    CK(cudaMemcpyAsync(D1.data(), dev_small, (size_t)wp * m * 8, cudaMemcpyDeviceToHost, ctx->st));
    hy::launch_tsdots(ctx->X, wp, phi, m, N, part, dev_small, ctx->st);
    CK(cudaMemcpyAsync(D2.data(), dev_small, (size_t)wp * m * 8, cudaMemcpyDeviceToHost, ctx->st));
  }
  if (hyrom_status s = sync(ctx)) return s;
  // singular values in descending order (ties: lower column first), nonzero ones
  std::vector<int> perm;
  for (int c = 0; c < wp; ++c)
    if (lam2[c] > 0.0) perm.push_back(c);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return lam2[a] > lam2[b]; });
  const int r = (int)perm.size();
  if (m > r) return fail(ctx, HYROM_ESTATE, "adjoint: the window has rank %d < %d", r, m);
  std::vector<double> sg(r), gsign(r, 1.0);
  for (int i = 0; i < r; ++i) sg[i] = std::sqrt(lam2[perm[i]]);
  for (int j = 0; j < m; ++j) gsign[j] = D2[(size_t)perm[j] * m + j] >= 0.0 ? 1.0 : -1.0;
  auto Vv = [&](int i, int c) { return gsign[i] * V[(size_t)perm[i] * wp + c]; };  // V_i[c]
  // A[i][j] = U_i . l_j
  std::vector<double> A((size_t)r * m);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = gsign[i] * D1[(size_t)perm[i] * m + j] / sg[i];
  std::vector<double> B1((size_t)std::max(m, 1) * w, 0.0), M((size_t)r * w, 0.0),
      B2((size_t)wp * w, 0.0);
  for (int j = 0; j < m; ++j)
    for (int c = 0; c < w; ++c) B1[(size_t)j * w + c] = Vv(j, c) / sg[j];
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < m; ++j) {
      double coef = -A[(size_t)i * m + j] / sg[j];
      if (i != j) coef += A[(size_t)i * m + j] / (sg[j] * sg[j] - sg[i] * sg[i]) * sg[j];
      for (int c = 0; c < w; ++c) M[(size_t)i * w + c] += coef * Vv(j, c);
    }
  for (int j = 0; j < m; ++j)  // term 3 on U_j: sum_{i != j} c_ij s_i V_i
    for (int i = 0; i < r; ++i) {
      if (i == j) continue;
      const double cij = A[(size_t)i * m + j] / (sg[j] * sg[j] - sg[i] * sg[i]);
      for (int c = 0; c < w; ++c) M[(size_t)j * w + c] += cij * sg[i] * Vv(i, c);
    }
  for (int i = 0; i < r; ++i)  // U_i = g_i X[:, perm_i] / s_i
    for (int c = 0; c < w; ++c) B2[(size_t)perm[i] * w + c] = gsign[i] * M[(size_t)i * w + c] / sg[i];
  double* dB1 = dev_small;
  double* dB2 = dev_small + (size_t)std::max(m, 1) * w;
  int* dwin = (int*)(dB2 + (size_t)wp * w);
  std::vector<int> win(w);
  for (int c = 0; c < w; ++c) win[c] = k_rebuild - w + 1 + c;
  CK(cudaMemcpyAsync(dB1, B1.data(), B1.size() * 8, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(dB2, B2.data(), B2.size() * 8, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(dwin, win.data(), w * 4, cudaMemcpyHostToDevice, ctx->st));
  hy::launch_pod_vjp_apply(N, m, wp, w, lphi, ctx->X, dB1, dB2, dwin, lpsi_new, lam, lpsi_cur,
                           ctx->st);
  CKL();
  return sync(ctx);
}

}  // namespace

hyrom_status hyrom_stage_pod_vjp(hyrom_ctx* ctx, const double* window, int32_t w,
                                 const double* psi, const double* lphi, int32_t m,
                                 double* lam_window, double* lpsi_out) {
  GUARD();
  if (!window || !psi || !lphi || !lam_window || !lpsi_out || w != ctx->cfg.w || m < 1)
    return HYROM_EINVAL;
  if (ctx->f32) return fail(ctx, HYROM_EINVAL, "hyrom_stage_pod_vjp: FP64 contexts");
  const size_t N = (size_t)ctx->N;
  std::vector<int> win(w);
  for (int c = 0; c < w; ++c) {
    win[c] = c;
    CK(cudaMemcpyAsync((double*)ctx->ring + c * N, window + c * N, N * 8, cudaMemcpyDeviceToDevice,
                       ctx->st));
  }
  double* phi = nullptr;
  double* part = nullptr;
  const size_t pwork = hy::tsdots_part_doubles(ctx->wp, m) + (size_t)m * w + (size_t)ctx->wp * w +
                       w + 64;
  if (cudaMalloc((void**)&phi, N * m * 8) != cudaSuccess ||
      cudaMalloc((void**)&part, pwork * 8) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(phi);
    return fail(ctx, HYROM_ENOMEM, "hyrom_stage_pod_vjp: scratch");
  }
  int me = 0;
  hyrom_status s = pod_t<double>(ctx, (const double*)ctx->ring, ctx->nslot, win, psi, nullptr, phi,
                                 nullptr, &me);
  if (s == HYROM_OK && me != m)
    s = fail(ctx, HYROM_EINVAL, "hyrom_stage_pod_vjp: the POD keeps %d modes, not %d", me, m);
  if (s == HYROM_OK && (cudaMemsetAsync(lam_window, 0, N * w * 8, ctx->st) != cudaSuccess ||
                        cudaMemsetAsync(lpsi_out, 0, N * 8, ctx->st) != cudaSuccess))
    s = fail(ctx, HYROM_ECUDA, "hyrom_stage_pod_vjp: clear");
  if (s == HYROM_OK) {
    AdjTape tp;  // window c = step c: the window lands on lam_window's columns
    s = pod_vjp(ctx, &tp, w - 1, phi, m, lphi, nullptr, lpsi_out, lam_window, part);
  }
  cudaFree(phi);
  cudaFree(part);
  return s;
}

hyrom_status hyrom_stage_filter_vjp(hyrom_ctx* ctx, const double* q, const double* q_prev,
                                    int64_t k, double* lam_io) {
  GUARD();
  if (!q || !q_prev || !lam_io) return HYROM_EINVAL;
  if (ctx->f32 || ctx->cfg.scheme != HYROM_SCHEME_RK2 || ctx->cfg.pde != HYROM_PDE_EULER)
    return fail(ctx, HYROM_EINVAL, "hyrom_stage_filter_vjp: FP64 Euler SSP-RK2 contexts");
  const hyrom_config& cf = ctx->cfg;
  const size_t N = (size_t)ctx->N, nw = (size_t)ctx->nwords;
  const int passmax = std::max(1, cf.n_filt * cf.jmax_f);
  double *qf = nullptr, *t1 = nullptr, *t2 = nullptr;
  uint32_t* keeps = nullptr;
  int *orders = nullptr, *count = nullptr;
  bool ok = cudaMalloc((void**)&qf, N * 8) == cudaSuccess &&
            cudaMalloc((void**)&t1, N * 8) == cudaSuccess &&
            cudaMalloc((void**)&t2, N * 8) == cudaSuccess &&
            cudaMalloc((void**)&keeps, (size_t)passmax * nw * 4) == cudaSuccess &&
            cudaMalloc((void**)&orders, (size_t)passmax * 4) == cudaSuccess &&
            cudaMalloc((void**)&count, 4) == cudaSuccess;
  hyrom_status s = HYROM_OK;
  if (!ok) {
    cudaGetLastError();
    s = fail(ctx, HYROM_ENOMEM, "hyrom_stage_filter_vjp: scratch");
  }
  std::vector<int> ord(passmax);
  int npass = 0;
  if (s == HYROM_OK) {
    CK(cudaMemcpyAsync(qf, q, N * 8, cudaMemcpyDeviceToDevice, ctx->st));
    hy::launch_filter_sparse<double>(ctx->dc, cf.filt_orders, cf.n_filt, cf.jmax_f, cf.eps_f, qf,
                                     q_prev, k, (double*)ctx->fg, ctx->kbits, ctx->ftiles_a,
                                     ctx->ftiles_b, ctx->fcounts, ctx->fpart, ctx->fctl,
                                     ctx->fargs, nullptr, ctx->st, keeps, orders, count);
    CK(cudaMemcpyAsync(&npass, count, 4, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ord.data(), orders, passmax * 4, cudaMemcpyDeviceToHost, ctx->st));
    s = sync(ctx);
  }
  if (s == HYROM_OK) {
    hy::launch_filter_vjp(ctx->dc, keeps, ord.data(), npass, lam_io, t1, t2, ctx->st);
    s = sync(ctx);
  }
  cudaFree(qf);
  cudaFree(t1);
  cudaFree(t2);
  cudaFree(keeps);
  cudaFree(orders);
  cudaFree(count);
  return s;
}

hyrom_status hyrom_adjoint(hyrom_ctx* ctx, int32_t steps, const int32_t* box, double* J_out,
                           double* dJdq0) {
  GUARD();
  const hyrom_config& cf = ctx->cfg;
  if (steps < 1 || !box || !dJdq0) return HYROM_EINVAL;
  if (ctx->f32 || cf.pde != HYROM_PDE_EULER || cf.scheme != HYROM_SCHEME_RK2 ||
      cf.regress_rows != HYROM_ROWS_ODEIM)
    return fail(ctx, HYROM_EINVAL, "hyrom_adjoint: FP64 Euler SSP-RK2 contexts on ODEIM rows");
  if (ctx->k != 0) return fail(ctx, HYROM_ESTATE, "hyrom_adjoint: the context must be at k = 0");
  if (!(box[0] >= 0 && box[0] < box[1] && box[1] <= cf.nx && box[2] >= 0 && box[2] < box[3] &&
        box[3] <= cf.ny))
    return fail(ctx, HYROM_EINVAL, "hyrom_adjoint: box outside the grid");
  const size_t N = (size_t)ctx->N, nw = (size_t)ctx->nwords;
  AdjTape* tp = new AdjTape;
  tp->steps = steps;
  for (int i = 0; i < 4; ++i) tp->box[i] = box[i];
  tp->wgt = cf.dt * cf.dx * cf.dy;
  tp->passmax = std::max(1, cf.n_filt * cf.jmax_f);
  tp->rec.assign(steps + 1, AdjStep());
  const size_t S = (size_t)steps + 1;
  bool ok = true;
  auto al = [&](void** p, size_t b) {
    if (ok && cudaMalloc(p, b) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  };
  al((void**)&tp->states, S * N * 8);
  al((void**)&tp->vpred, S * N * 8);
  al((void**)&tp->ys, S * 64 * 8);
  al((void**)&tp->shats, S * nw * 4);
  al((void**)&tp->rows, S * (size_t)cf.n_p * 4);
  al((void**)&tp->keeps, S * tp->passmax * nw * 4);
  al((void**)&tp->orders, S * tp->passmax * 4);
  al((void**)&tp->npass, S * 4);
  al((void**)&tp->Jpart, 152 * 8 * 8);
  al((void**)&tp->J, 8);
  if (!ok) {
    free_tape(tp);
    return fail(ctx, HYROM_ENOMEM, "hyrom_adjoint: tape allocation");
  }
  hyrom_status st = HYROM_OK;
  auto done = [&](hyrom_status s) {
    ctx->tape = nullptr;
    free_tape(tp);
    return s;
  };
  if (cudaMemsetAsync(tp->J, 0, 8, ctx->st) != cudaSuccess ||
      cudaMemsetAsync(tp->npass, 0, S * 4, ctx->st) != cudaSuccess ||
      cudaMemcpyAsync(tp->states, ring_at<double>(ctx, 0), N * 8, cudaMemcpyDeviceToDevice,
                      ctx->st) != cudaSuccess)
    return done(fail(ctx, HYROM_ECUDA, "hyrom_adjoint: tape set-up"));
  // ---- forward run, recorded
  ctx->tape = tp;
  for (int k = 1; k <= steps; ++k) {
    hyrom_step_info inf;
    st = hyrom_step(ctx, &inf);
    if (st != HYROM_OK && st != HYROM_ERANK) return done(st);
  }
  ctx->tape = nullptr;
  std::vector<int> npass(S);
  std::vector<int> orders(S * tp->passmax);
  double Jh = 0.0;
  if (cudaMemcpyAsync(npass.data(), tp->npass, S * 4, cudaMemcpyDeviceToHost, ctx->st) !=
          cudaSuccess ||
      cudaMemcpyAsync(orders.data(), tp->orders, S * tp->passmax * 4, cudaMemcpyDeviceToHost,
                      ctx->st) != cudaSuccess ||
      cudaMemcpyAsync(&Jh, tp->J, 8, cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess)
    return done(fail(ctx, HYROM_ECUDA, "hyrom_adjoint: tape read-back"));
  if ((st = sync(ctx))) return done(st);
  if (J_out) *J_out = Jh;
  // ---- reverse sweep
  const int m = cf.m;
  double *lam = nullptr, *lphi = nullptr, *phi = nullptr, *lk = nullptr, *lv = nullptr,
         *lpsi_t = nullptr, *lphi_t = nullptr, *lin = nullptr, *t1 = nullptr, *t2 = nullptr,
         *work = nullptr, *part = nullptr;
  std::vector<double*> lpsi(tp->psis.size(), nullptr);
  const size_t rwork = hy::reduced_vjp_work_doubles(m, cf.n_p);
  const size_t pwork = hy::tsdots_part_doubles(ctx->wp, m) + (size_t)m * cf.w +
                       (size_t)ctx->wp * cf.w + cf.w + 64;
  al((void**)&lam, S * N * 8);
  al((void**)&lphi, N * m * 8);
  al((void**)&phi, N * m * 8);
  al((void**)&lk, N * 8);
  al((void**)&lv, N * 8);
  al((void**)&lpsi_t, N * 8);
  al((void**)&lphi_t, N * m * 8);
  al((void**)&lin, N * 8);
  al((void**)&t1, N * 8);
  al((void**)&t2, N * 8);
  al((void**)&work, std::max(rwork, 3 * N) * 8);
  al((void**)&part, pwork * 8);
  for (auto& p : lpsi) al((void**)&p, N * 8);
  auto release = [&](hyrom_status s) {
    for (double* p : {lam, lphi, phi, lk, lv, lpsi_t, lphi_t, lin, t1, t2, work, part}) cudaFree(p);
    for (double* p : lpsi) cudaFree(p);
    return done(s);
  };
  if (!ok) return release(fail(ctx, HYROM_ENOMEM, "hyrom_adjoint: sweep allocation"));
  if (cudaMemsetAsync(lam, 0, S * N * 8, ctx->st) != cudaSuccess ||
      cudaMemsetAsync(lphi, 0, N * m * 8, ctx->st) != cudaSuccess)
    return release(fail(ctx, HYROM_ECUDA, "hyrom_adjoint: sweep set-up"));
  for (double* p : lpsi)
    if (cudaMemsetAsync(p, 0, N * 8, ctx->st) != cudaSuccess)
      return release(fail(ctx, HYROM_ECUDA, "hyrom_adjoint: sweep set-up"));
  // rebuild step of each basis version, and the version whose POD is in phi
  std::vector<int> made_at(tp->nphi, -1), made_psi(tp->nphi, -1);
  for (int k = 0; k <= steps; ++k)
    if (tp->rec[k].rebuild) {
      made_at[tp->rec[k].new_phi] = k;
      made_psi[tp->rec[k].new_phi] = tp->rec[k].psi_cur;
    }
  int cached = -1, cached_me = 0;
  auto ensure_pod = [&](int v) -> hyrom_status {
    if (cached == v) return HYROM_OK;
    int me = 0;
    if (hyrom_status s = recompute_pod(ctx, tp, made_at[v], made_psi[v], phi, &me)) return s;
    cached = v;
    cached_me = me;
    return HYROM_OK;
  };
  for (int k = steps; k >= 1; --k) {
    const AdjStep& r = tp->rec[k];
    if (r.rebuild) {  // the rebuild after step k: its POD and its psi
      if ((st = ensure_pod(r.new_phi))) return release(st);
      if (cached_me != r.m_eff) return release(fail(ctx, HYROM_ECUDA, "adjoint: POD rank differs"));
      if ((st = pod_vjp(ctx, tp, k, phi, r.m_eff, lphi, lpsi[r.new_psi], lpsi[r.psi_cur], lam, part)))
        return release(st);
      if (cudaMemsetAsync(lphi, 0, N * m * 8, ctx->st) != cudaSuccess)
        return release(fail(ctx, HYROM_ECUDA, "adjoint"));
    }
    if (r.psi_init) {  // psi_{w-1} = mean(gamma_0 .. gamma_{w-1})
      std::vector<int> win(cf.w);
      for (int c = 0; c < cf.w; ++c) win[c] = c;
      int* dwin = (int*)part;
      CK(cudaMemcpyAsync(dwin, win.data(), cf.w * 4, cudaMemcpyHostToDevice, ctx->st));
      hy::launch_mean_vjp(ctx->N, dwin, cf.w, lpsi[r.init_psi], lam, ctx->st);
      if ((st = sync(ctx))) return release(st);
    }
    // lk = lambda_k + the output term of step k
    CK(cudaMemcpyAsync(lk, lam + (size_t)k * N, N * 8, cudaMemcpyDeviceToDevice, ctx->st));
    hy::launch_pressure_vjp(ctx->dc, tp->states + (size_t)k * N, tp->box, tp->wgt, lk, ctx->st);
    const double* prev = tp->states + (size_t)(k - 1) * N;
    double* lprev = lam + (size_t)(k - 1) * N;
    if (r.full) {
      hy::launch_rk2_vjp(ctx->dc, prev, lk, lin, nullptr, k, work, ctx->st);
      add_into(lin, lprev, (int64_t)N, ctx->st);
    } else {
      const uint32_t* shat = tp->shats + (size_t)k * nw;
      hy::launch_filter_vjp(ctx->dc, tp->keeps + (size_t)k * tp->passmax * nw,
                            orders.data() + (size_t)k * tp->passmax, npass[k], lk, t1, t2,
                            ctx->st);
      if ((st = ensure_pod(r.phi_ver))) return release(st);
      hy::launch_reduced_vjp(ctx->N, ctx->nc, r.m_eff, phi, tp->rows + (size_t)k * cf.n_p, r.n_p,
                             tp->vpred + (size_t)k * N, tp->psis[r.psi_ver],
                             tp->ys + (size_t)k * 64, shat, lk, lv, lpsi_t, lphi_t, work,
                             ctx->st);
      add_into(lpsi_t, lpsi[r.psi_ver], (int64_t)N, ctx->st);
      add_into(lphi_t, lphi, (int64_t)N * r.m_eff, ctx->st);
      hy::launch_rk2_vjp(ctx->dc, prev, lv, lin, shat, k, work, ctx->st);
      add_into(lin, lprev, (int64_t)N, ctx->st);
    }
    CKL();
    if ((st = sync(ctx))) return release(st);
  }
  CK(cudaMemcpyAsync(dJdq0, lam, N * 8, cudaMemcpyDeviceToDevice, ctx->st));
  st = sync(ctx);
  return release(st);
}

// ---- checkpoint / resume ------------------------------------------------------
namespace {

struct CkRec {
  uint32_t tag;
  void* p;
  size_t bytes;
};

// The device state that carries from one step to the next.
std::vector<CkRec> ck_records(hyrom_ctx* c) {
  const size_t es = c->esz, N = (size_t)c->N, nw = (size_t)c->nwords;
  std::vector<CkRec> r = {
      {1, c->ring, (size_t)c->nslot * N * es},
      {2, c->psi, N * es},
      {3, c->phi, N * (size_t)c->m * es},
      {4, c->pts, 1024 * sizeof(int)},
      {5, c->pinv, (size_t)c->m * c->cfg.n_p * sizeof(double)},
      {6, c->y, 256 * sizeof(double)},
      {7, c->shat, nw * 4},
      {8, c->stilde, nw * 4},
      {9, c->g_bm, nw * 4},
      {10, c->tiles, (size_t)c->ntiles_max * sizeof(int)},
      {11, c->ntiles, 64},
      {12, c->H, (size_t)c->nslot * c->nslot * sizeof(double)},
      {13, c->m_eff_dev, 64},
  };
  if (c->cfg.regress_rows == HYROM_ROWS_SAMPLE) {
    r.push_back({14, c->s_cells, (size_t)c->nc * sizeof(int)});
    r.push_back({15, c->s_L, 4096 * sizeof(double)});
    r.push_back({16, c->s_dinv, 64 * sizeof(double)});
  }
  return r;
}

const char kCkMagic[8] = {'H', 'Y', 'R', 'O', 'M', 'C', 'K', 1};

bool same_layout(const hyrom_config& a, const hyrom_config& b) {
  bool ok = a.pde == b.pde && a.scheme == b.scheme && a.precision == b.precision &&
            a.nx == b.nx && a.ny == b.ny && a.w == b.w && a.m == b.m && a.n_p == b.n_p &&
            a.regress_rows == b.regress_rows;
  for (int i = 0; i < 4; ++i) ok = ok && a.bc[i] == b.bc[i];
  return ok;
}

}  // namespace

hyrom_status hyrom_save(hyrom_ctx* ctx, const char* path) {
  GUARD();
  if (!path) return HYROM_EINVAL;
  if (ctx->f32) gram_flush(ctx);
  if (hyrom_status s = sync(ctx)) return s;
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, HYROM_EINVAL, "hyrom_save: cannot open %s", path);
  const std::vector<CkRec> recs = ck_records(ctx);
  const size_t chunk = (size_t)64 << 20;
  void* stage = nullptr;
  if (cudaMallocHost(&stage, chunk) != cudaSuccess) {
    cudaGetLastError();
    fclose(f);
    return fail(ctx, HYROM_ENOMEM, "hyrom_save: pinned staging buffer");
  }
  bool ok = true;
  auto put = [&](const void* p, size_t n) { ok = ok && fwrite(p, 1, n, f) == n; };
  const uint32_t version = 1, cfg_bytes = (uint32_t)sizeof(hyrom_config);
  put(kCkMagic, 8);
  put(&version, 4);
  put(&cfg_bytes, 4);
  put(&ctx->cfg, sizeof(hyrom_config));
  const int64_t k = ctx->k, n_s = ctx->n_s;
  const int32_t sc[6] = {ctx->m_eff, ctx->np_eff, ctx->has_basis, ctx->psi_set,
                         ctx->sample_ok ? 1 : 0, 0};
  put(&k, 8);
  put(&n_s, 8);
  put(sc, sizeof sc);
  const uint32_t npsi = (uint32_t)ctx->psi_steps.size();
  put(&npsi, 4);
  if (npsi) put(ctx->psi_steps.data(), npsi * sizeof(int64_t));
  const uint32_t nrec = (uint32_t)recs.size();
  put(&nrec, 4);
  hyrom_status st = HYROM_OK;
  for (const CkRec& r : recs) {
    const uint64_t bytes = r.bytes;
    put(&r.tag, 4);
    put(&bytes, 8);
    for (size_t off = 0; ok && off < r.bytes; off += chunk) {
      const size_t n = r.bytes - off < chunk ? r.bytes - off : chunk;
      if (cudaMemcpyAsync(stage, (const char*)r.p + off, n, cudaMemcpyDeviceToHost, ctx->st) !=
              cudaSuccess ||
          cudaStreamSynchronize(ctx->st) != cudaSuccess) {
        st = HYROM_ECUDA;
        ok = false;
        break;
      }
      put(stage, n);
    }
  }
  cudaFreeHost(stage);
  if (fclose(f) != 0) ok = false;
  if (st == HYROM_ECUDA) return fail(ctx, HYROM_ECUDA, "hyrom_save: device read failed");
  if (!ok) return fail(ctx, HYROM_EINVAL, "hyrom_save: write to %s failed", path);
  return HYROM_OK;
}

hyrom_status hyrom_load(hyrom_ctx* ctx, const char* path) {
  GUARD();
  if (!path) return HYROM_EINVAL;
  ctx->gram_dirty = -1;  // the file holds a complete H
  FILE* f = fopen(path, "rb");
  if (!f) return fail(ctx, HYROM_EINVAL, "hyrom_load: cannot open %s", path);
  bool ok = true;
  auto get = [&](void* p, size_t n) { ok = ok && fread(p, 1, n, f) == n; };
  char magic[8];
  uint32_t version = 0, cfg_bytes = 0;
  get(magic, 8);
  get(&version, 4);
  get(&cfg_bytes, 4);
  if (!ok || memcmp(magic, kCkMagic, 8) != 0 || version != 1 ||
      cfg_bytes != sizeof(hyrom_config)) {
    fclose(f);
    return fail(ctx, HYROM_EINVAL, "hyrom_load: %s is not a checkpoint of this library", path);
  }
  hyrom_config saved;
  get(&saved, sizeof saved);
  if (!ok || !same_layout(saved, ctx->cfg)) {
    fclose(f);
    return fail(ctx, HYROM_EINVAL,
                "hyrom_load: the checkpoint's grid, scheme, precision, sides, w, m, n_p or "
                "regression rows differ from this context's");
  }
  int64_t k = 0, n_s = 0;
  int32_t sc[6];
  uint32_t npsi = 0;
  get(&k, 8);
  get(&n_s, 8);
  get(sc, sizeof sc);
  get(&npsi, 4);
  std::vector<int64_t> psi_steps(npsi);
  if (npsi) get(psi_steps.data(), npsi * sizeof(int64_t));
  uint32_t nrec = 0;
  get(&nrec, 4);
  const std::vector<CkRec> recs = ck_records(ctx);
  if (!ok || nrec != recs.size()) {
    fclose(f);
    return fail(ctx, HYROM_EINVAL, "hyrom_load: %s is truncated or of another layout", path);
  }
  const size_t chunk = (size_t)64 << 20;
  void* stage = nullptr;
  if (cudaMallocHost(&stage, chunk) != cudaSuccess) {
    cudaGetLastError();
    fclose(f);
    return fail(ctx, HYROM_ENOMEM, "hyrom_load: pinned staging buffer");
  }
  hyrom_status st = HYROM_OK;
  for (const CkRec& r : recs) {
    uint32_t tag = 0;
    uint64_t bytes = 0;
    get(&tag, 4);
    get(&bytes, 8);
    if (!ok || tag != r.tag || bytes != r.bytes) {
      ok = false;
      break;
    }
    for (size_t off = 0; ok && off < r.bytes; off += chunk) {
      const size_t n = r.bytes - off < chunk ? r.bytes - off : chunk;
      get(stage, n);
      if (!ok) break;
      if (cudaMemcpyAsync((char*)r.p + off, stage, n, cudaMemcpyHostToDevice, ctx->st) !=
              cudaSuccess ||
          cudaStreamSynchronize(ctx->st) != cudaSuccess) {
        st = HYROM_ECUDA;
        ok = false;
      }
    }
  }
  cudaFreeHost(stage);
  fclose(f);
  if (st == HYROM_ECUDA) return fail(ctx, HYROM_ECUDA, "hyrom_load: device write failed");
  if (!ok) return fail(ctx, HYROM_EINVAL, "hyrom_load: %s is truncated or of another layout", path);
  ctx->k = k;
  ctx->n_s = n_s;
  ctx->m_eff = sc[0];
  ctx->np_eff = sc[1];
  ctx->has_basis = sc[2];
  ctx->psi_set = sc[3];
  ctx->sample_ok = sc[4] != 0;
  ctx->norms_ready = false;
  ctx->psi_steps = psi_steps;
  return HYROM_OK;
}

hyrom_status hyrom_sample(hyrom_ctx* ctx, int32_t* idx_dev, int64_t cap, int64_t* n_out,
                          uint32_t* bitmap_dev) {
  GUARD();
  if (!ctx->has_basis) return fail(ctx, HYROM_ESTATE, "no sampled set before the first rebuild");
  if (n_out) *n_out = ctx->n_s;
  if (bitmap_dev)
    CK(cudaMemcpyAsync(bitmap_dev, ctx->shat, ctx->nwords * 4, cudaMemcpyDeviceToDevice, ctx->st));
  if (idx_dev) {
    if (cap < ctx->n_s) return fail(ctx, HYROM_ECAP, "capacity %lld < %lld", (long long)cap, (long long)ctx->n_s);
    hy::launch_bits_to_list(ctx->shat, ctx->nc, ctx->list_cnt, idx_dev, cap, ctx->st);
  }
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_get_state(hyrom_ctx* ctx, void* q, int q_on_host) {
  GUARD();
  if (!q) return HYROM_EINVAL;
  const void* src = (const char*)ctx->ring + (size_t)slot_of(ctx, ctx->k) * ctx->N * ctx->esz;
  CK(cudaMemcpyAsync(q, src, ctx->N * ctx->esz,
                     q_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->st));
  return sync(ctx);
}

hyrom_status hyrom_set_state(hyrom_ctx* ctx, const void* q, int q_on_host) {
  GUARD();
  if (!q) return HYROM_EINVAL;
  void* dst = (char*)ctx->ring + (size_t)slot_of(ctx, ctx->k) * ctx->N * ctx->esz;
  CK(cudaMemcpyAsync(dst, q, ctx->N * ctx->esz,
                     q_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->st));
  if (ctx->f32) {
    // the new state's Gram row is formed by the next Gram update (the next
    // step's, in the same pass over the window as its own row), or before H
    // is next read
    if (ctx->gram_dirty >= 0 && ctx->gram_dirty != ctx->k) gram_flush(ctx);
    ctx->gram_dirty = ctx->k;
  }
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_get_basis(hyrom_ctx* ctx, void* phi_dev, int32_t* m_eff, void* psi_dev,
                             int32_t* points_dev, int32_t* n_p) {
  GUARD();
  if (!ctx->has_basis) return fail(ctx, HYROM_ESTATE, "no basis before the first rebuild");
  if (m_eff) *m_eff = ctx->m_eff;
  if (n_p) *n_p = ctx->np_eff;
  if (phi_dev && ctx->m_eff)
    CK(cudaMemcpyAsync(phi_dev, ctx->phi, (size_t)ctx->N * ctx->m_eff * ctx->esz,
                       cudaMemcpyDeviceToDevice, ctx->st));
  if (psi_dev)
    CK(cudaMemcpyAsync(psi_dev, ctx->psi, ctx->N * ctx->esz, cudaMemcpyDeviceToDevice, ctx->st));
  if (points_dev && ctx->np_eff)
    CK(cudaMemcpyAsync(points_dev, ctx->pts, ctx->np_eff * sizeof(int), cudaMemcpyDeviceToDevice,
                       ctx->st));
  return sync(ctx);
}

// ---- stage entry points ------------------------------------------------------

hyrom_status hyrom_stage_full_step(hyrom_ctx* ctx, const void* q_prev, void* q_out, int64_t k) {
  GUARD();
  if (!q_prev || !q_out || q_prev == q_out) return HYROM_EINVAL;
  CK(cudaMemsetAsync(ctx->fail_dev, 0, sizeof(int), ctx->st));
  if (ctx->cfg.scheme == HYROM_SCHEME_RK2) {
    t_begin(ctx, HYROM_T_FULL);
    if (ctx->f32)
      hy::launch_rk2<float>(ctx->dc, (const float*)q_prev, (float*)q_out, k, nullptr, nullptr,
                            nullptr, ctx->st);
    else
      hy::launch_rk2<double>(ctx->dc, (const double*)q_prev, (double*)q_out, k, nullptr, nullptr,
                             nullptr, ctx->st);
    t_end(ctx, HYROM_T_FULL);
  } else {
    CK(cudaMemcpyAsync(q_out, q_prev, ctx->N * 8, cudaMemcpyDeviceToDevice, ctx->st));
    if (hyrom_status s = newton_full<double>(ctx, (const double*)q_prev, (double*)q_out)) return s;
  }
  CKL();
  int* hi = (int*)ctx->host;
  CK(cudaMemcpyAsync(hi, ctx->fail_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  return hi[0] ? fail(ctx, HYROM_ENOTCONV, "Newton did not converge") : HYROM_OK;
}

// ---- the paper's HDM (MUSCL-Roe-BDF2) --------------------------------------
#define MUSCL_ONLY()                                                          \
  do {                                                                        \
    if (ctx->cfg.scheme != HYROM_SCHEME_BDF2_MUSCL)                           \
      return fail(ctx, HYROM_EINVAL, "needs a MUSCL-Roe-BDF2 context");       \
  } while (0)

hyrom_status hyrom_stage_muscl_residual(hyrom_ctx* ctx, const double* q, const double* q_prev,
                                        const double* q_prev2, int64_t k, double* r_out) {
  GUARD();
  MUSCL_ONLY();
  if (!q || !q_prev || !r_out) return HYROM_EINVAL;
  hy::launch_muscl_residual(ctx->dc, q, q_prev, q_prev2, (double)k * ctx->cfg.dt, nullptr,
                            ctx->nc, r_out, ctx->st);
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_stage_muscl_jvp(hyrom_ctx* ctx, const double* q, const double* v, int64_t k,
                                   int32_t bdf2, double* jv_out) {
  GUARD();
  MUSCL_ONLY();
  if (!q || !v || !jv_out || v == jv_out) return HYROM_EINVAL;
  const double dtb = bdf2 ? ctx->cfg.dt * (2.0 / 3.0) : ctx->cfg.dt;
  hy::launch_muscl_jvp(ctx->dc, q, v, (double)k * ctx->cfg.dt, 1.0, dtb, nullptr, ctx->nc, jv_out,
                       ctx->st);
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_stage_muscl_step(hyrom_ctx* ctx, const double* q_prev2, const double* q_prev,
                                    double* q_io, const uint32_t* s_hat, int64_t k) {
  GUARD();
  MUSCL_ONLY();
  if (!q_prev || !q_io || q_prev == q_io || q_prev2 == q_io) return HYROM_EINVAL;
  ctx->muscl_fail = 0;
  if (!s_hat) {
    CK(cudaMemcpyAsync(q_io, q_prev, ctx->N * 8, cudaMemcpyDeviceToDevice, ctx->st));
    if (hyrom_status s = muscl_solve(ctx, q_io, q_prev, q_prev2, k, nullptr, ctx->nc)) return s;
  } else {
    long long* hl = (long long*)ctx->host;
    CK(cudaMemsetAsync(ctx->list_cnt, 0, sizeof(long long), ctx->st));
    hy::launch_bits_to_list(s_hat, ctx->nc, ctx->list_cnt, ctx->mus_cells, ctx->nc, ctx->st);
    hy::launch_popcount(s_hat, ctx->nwords, ctx->n_s_dev, ctx->st);
    CK(cudaMemcpyAsync(hl, ctx->n_s_dev, sizeof(long long), cudaMemcpyDeviceToHost, ctx->st));
    if (hyrom_status s = sync(ctx)) return s;
    const int64_t n = hl[0];
    if (n > 0)
      if (hyrom_status s = muscl_solve(ctx, q_io, q_prev, q_prev2, k, ctx->mus_cells, n)) return s;
  }
  if (hyrom_status s = sync(ctx)) return s;
  return ctx->muscl_fail ? fail(ctx, HYROM_ENOTCONV, "Newton-GMRES hit newton_max") : HYROM_OK;
}

hyrom_status hyrom_stage_muscl_filter(hyrom_ctx* ctx, double* q_io, const double* q_prev,
                                      const double* q_prev2, int64_t k, int32_t* passes) {
  GUARD();
  MUSCL_ONLY();
  if (!q_io || !q_prev || q_io == q_prev) return HYROM_EINVAL;
  const hyrom_config& cf = ctx->cfg;
  const int np = hy::muscl_filter(ctx->mus, ctx->dc, q_io, q_prev, q_prev2, k, cf.filt_orders, cf.n_filt,
                                  cf.jmax_f, cf.eps_f, (double*)ctx->fg, (double*)ctx->ftmp,
                                  (double*)ctx->rho_old, (double*)ctx->rho_new, ctx->fpart,
                                  ctx->dy + 2, (double*)ctx->host + 28, ctx->st);
  if (np < 0) return fail(ctx, HYROM_ECUDA, "filter: %s", cudaGetErrorString(cudaGetLastError()));
  if (passes) *passes = np;
  return sync(ctx);
}

hyrom_status hyrom_stage_partial_step(hyrom_ctx* ctx, const void* q_prev, void* q_io,
                                      const uint32_t* s_hat, int64_t k) {
  GUARD();
  if (!q_prev || !q_io || !s_hat || q_prev == q_io) return HYROM_EINVAL;
  CK(cudaMemsetAsync(ctx->fail_dev, 0, sizeof(int), ctx->st));
  if (ctx->cfg.scheme == HYROM_SCHEME_RK2) {
    hy::launch_active_tiles(ctx->dc, s_hat, hy::rk2_tile_width(ctx->dc),
                            hy::rk2_tile_height(ctx->dc), ctx->tiles, ctx->ntiles, ctx->st);
    if (ctx->f32)
      hy::launch_rk2<float>(ctx->dc, (const float*)q_prev, (float*)q_io, k, s_hat, ctx->tiles,
                            ctx->ntiles, ctx->st);
    else
      hy::launch_rk2<double>(ctx->dc, (const double*)q_prev, (double*)q_io, k, s_hat, ctx->tiles,
                             ctx->ntiles, ctx->st);
  } else {
    // count the sampled cells to detect the all-cells (cyclic) case
    CK(cudaMemsetAsync(ctx->n_s_dev, 0, sizeof(long long), ctx->st));
    long long* hl = (long long*)ctx->host;
    hy::launch_masks(ctx->dc, s_hat, nullptr, 0, 0, 1, ctx->base_bm, ctx->tmp_bm,
                     ctx->g_bm, ctx->n_s_dev, ctx->st);
    CK(cudaMemcpyAsync(hl, ctx->n_s_dev, sizeof(long long), cudaMemcpyDeviceToHost, ctx->st));
    if (hyrom_status s = sync(ctx)) return s;
    if (hyrom_status s = newton_partial<double>(ctx, (const double*)q_prev, (double*)q_io, s_hat, hl[0]))
      return s;
  }
  CKL();
  int* hi = (int*)ctx->host;
  CK(cudaMemcpyAsync(hi, ctx->fail_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  return hi[0] ? fail(ctx, HYROM_ENOTCONV, "Newton did not converge") : HYROM_OK;
}

hyrom_status hyrom_stage_gappy(hyrom_ctx* ctx, const void* phi, int32_t m, const int32_t* points,
                               int32_t n_p, const void* v, const void* psi, double* y_out) {
  GUARD();
  if (!phi || !points || !v || !psi || !y_out || m < 1 || m > 256 || n_p < m || n_p > 1024)
    return HYROM_EINVAL;
  if (hy::gappy_pinv_smem(m, n_p) > 227 * 1024) return HYROM_EINVAL;
  double* pinv = nullptr;
  if (cudaMallocAsync((void**)&pinv, (size_t)m * n_p * sizeof(double), ctx->st) != cudaSuccess)
    return fail(ctx, HYROM_ENOMEM, "pinv allocation");
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->st));
  if (ctx->f32) {
    hy::launch_gappy_pinv<float>((const float*)phi, ctx->N, m, points, n_p, pinv, ctx->status, ctx->st);
    hy::launch_gappy_apply<float>(pinv, m, n_p, points, (const float*)v, (const float*)psi, y_out,
                                  nullptr, nullptr, ctx->st, ctx->status);
  } else {
    hy::launch_gappy_pinv<double>((const double*)phi, ctx->N, m, points, n_p, pinv, ctx->status, ctx->st);
    hy::launch_gappy_apply<double>(pinv, m, n_p, points, (const double*)v, (const double*)psi,
                                   y_out, nullptr, nullptr, ctx->st, ctx->status);
  }
  CKL();
  CK(cudaFreeAsync(pinv, ctx->st));
  int* hi = (int*)ctx->host;
  CK(cudaMemcpyAsync(hi, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  if (hi[0]) return fail(ctx, HYROM_ERANK, "P^T Phi is rank-deficient (y set to NaN)");
  return HYROM_OK;
}

hyrom_status hyrom_stage_gappy_rows(hyrom_ctx* ctx, const void* phi, int32_t m,
                                    const int32_t* cells, int32_t n_cells, const void* v,
                                    const void* psi, double* y_out) {
  GUARD();
  if (!phi || !cells || !v || !psi || !y_out || m < 1 || m > 64 || n_cells < 1 ||
      n_cells > ctx->nc)
    return HYROM_EINVAL;
  if (ctx->cfg.regress_rows != HYROM_ROWS_SAMPLE)
    return fail(ctx, HYROM_ESTATE, "the context was not configured for sample rows");
  // the factor of the context's own basis is overwritten: fall back to the
  // ODEIM rows until the next rebuild
  ctx->sample_ok = false;
  CK(cudaMemsetAsync(ctx->fail_dev + 8, 0, 2 * sizeof(int), ctx->st));
  if (ctx->f32) {
    t_begin(ctx, HYROM_T_SNORMAL);
    hy::launch_sample_normal<float>((const float*)phi, ctx->N, m, cells, n_cells, ctx->dc.nvar,
                                    ctx->nc, ctx->cfg.reduced_prec, ctx->s_part, ctx->s_G,
                                    ctx->s_L, ctx->s_dinv, ctx->fail_dev + 8, ctx->st);
    t_end(ctx, HYROM_T_SNORMAL);
    t_begin(ctx, HYROM_T_GAPPY);
    hy::launch_sample_solve<float>((const float*)phi, ctx->N, m, cells, n_cells, ctx->dc.nvar,
                                   ctx->nc, (const float*)v, (const float*)psi, ctx->s_part,
                                   ctx->s_b, ctx->s_L, ctx->s_dinv, y_out, nullptr, nullptr,
                                   ctx->st);
    t_end(ctx, HYROM_T_GAPPY);
  } else {
    t_begin(ctx, HYROM_T_SNORMAL);
    hy::launch_sample_normal<double>((const double*)phi, ctx->N, m, cells, n_cells,
                                     ctx->dc.nvar, ctx->nc, ctx->cfg.reduced_prec, ctx->s_part,
                                     ctx->s_G, ctx->s_L, ctx->s_dinv, ctx->fail_dev + 8, ctx->st);
    t_end(ctx, HYROM_T_SNORMAL);
    t_begin(ctx, HYROM_T_GAPPY);
    hy::launch_sample_solve<double>((const double*)phi, ctx->N, m, cells, n_cells, ctx->dc.nvar,
                                    ctx->nc, (const double*)v, (const double*)psi, ctx->s_part,
                                    ctx->s_b, ctx->s_L, ctx->s_dinv, y_out, nullptr, nullptr,
                                    ctx->st);
    t_end(ctx, HYROM_T_GAPPY);
  }
  CKL();
  int* hf = (int*)ctx->host + 12;
  CK(cudaMemcpyAsync(hf, ctx->fail_dev + 8, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status st = sync(ctx)) return st;
  if (hf[1]) return fail(ctx, HYROM_ETIMEOUT, "sample-row normal matrix: a device wait gave up");
  if (hf[0]) return fail(ctx, HYROM_ENOTCONV, "sample-row normal matrix is not positive definite");
  return HYROM_OK;
}

hyrom_status hyrom_stage_reconstruct(hyrom_ctx* ctx, const void* phi, int32_t m, const double* y,
                                     const void* psi, const uint32_t* s_hat, void* q_io) {
  GUARD();
  if (!phi || !y || !psi || !q_io || m < 0 || m > 256) return HYROM_EINVAL;
  if (ctx->f32)
    hy::launch_reconstruct<float>((const float*)phi, ctx->N, ctx->nc, m, y, (const float*)psi,
                                  s_hat, 0, (float*)q_io, ctx->st);
  else
    hy::launch_reconstruct<double>((const double*)phi, ctx->N, ctx->nc, m, y, (const double*)psi,
                                   s_hat, 0, (double*)q_io, ctx->st);
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_stage_filter(hyrom_ctx* ctx, void* q_io, const void* q_prev, int64_t k,
                                int32_t* passes) {
  GUARD();
  if (!q_io || !q_prev) return HYROM_EINVAL;
  const hyrom_config& cf = ctx->cfg;
  if (cf.n_filt > 0) {
    if (ctx->f32)
      hy::launch_filter_sparse<float>(ctx->dc, cf.filt_orders, cf.n_filt, cf.jmax_f, cf.eps_f,
                                      (float*)q_io, (const float*)q_prev, k, (float*)ctx->fg,
                                      ctx->kbits, ctx->ftiles_a, ctx->ftiles_b, ctx->fcounts,
                                      ctx->fpart, ctx->fctl, ctx->fargs, &ctx->filt_graph,
                                      ctx->st);
    else
      hy::launch_filter_sparse<double>(ctx->dc, cf.filt_orders, cf.n_filt, cf.jmax_f, cf.eps_f,
                                       (double*)q_io, (const double*)q_prev, k, (double*)ctx->fg,
                                       ctx->kbits, ctx->ftiles_a, ctx->ftiles_b, ctx->fcounts,
                                       ctx->fpart, ctx->fctl, ctx->fargs, &ctx->filt_graph,
                                       ctx->st);
  }
  CKL();
  int* hi = (int*)ctx->host;
  hi[1] = 0;
  if (cf.n_filt > 0)
    CK(cudaMemcpyAsync(hi + 1, ctx->fctl + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  if (passes) *passes = hi[1];
  return HYROM_OK;
}

hyrom_status hyrom_stage_cell_error(hyrom_ctx* ctx, const void* g, const void* psi,
                                    const void* phi, int32_t m, const double* y, void* eps_out) {
  GUARD();
  if (!g || !psi || !eps_out || m < 0 || m > 256 || (m > 0 && (!phi || !y))) return HYROM_EINVAL;
  if (ctx->f32)
    hy::launch_cell_error<float>((const float*)g, (const float*)psi, (const float*)phi, ctx->nc,
                                 ctx->dc.nvar, m, y, (float*)eps_out, ctx->st);
  else
    hy::launch_cell_error<double>((const double*)g, (const double*)psi, (const double*)phi,
                                  ctx->nc, ctx->dc.nvar, m, y, (double*)eps_out, ctx->st);
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_stage_rk2_vjp(hyrom_ctx* ctx, const void* q_prev, const void* lam_out,
                                 void* lam_in, const uint32_t* s_hat, int64_t k, void* work) {
  GUARD();
  if (!q_prev || !lam_out || !lam_in || !work || lam_in == lam_out || lam_in == q_prev)
    return HYROM_EINVAL;
  if (ctx->f32 || ctx->cfg.scheme != HYROM_SCHEME_RK2 || ctx->cfg.pde != HYROM_PDE_EULER)
    return fail(ctx, HYROM_EINVAL, "the step adjoint is defined for FP64 Euler SSP-RK2 contexts");
  hy::launch_rk2_vjp(ctx->dc, (const double*)q_prev, (const double*)lam_out, (double*)lam_in,
                     s_hat, k, (double*)work, ctx->st);
  CKL();
  return sync(ctx);
}

size_t hyrom_reduced_vjp_work_doubles(int32_t m, int32_t n_rows) {
  if (m < 1 || m > 64 || n_rows < 0) return 0;
  return hy::reduced_vjp_work_doubles(m, n_rows);
}

hyrom_status hyrom_stage_reduced_vjp(hyrom_ctx* ctx, const void* phi, int32_t m,
                                     const int32_t* rows, int32_t n_rows, const void* v,
                                     const void* psi, const double* y, const uint32_t* s_hat,
                                     const void* lam, void* lam_v, void* lam_psi, void* lam_phi,
                                     void* work) {
  GUARD();
  if (!phi || !rows || !v || !psi || !y || !s_hat || !lam || !lam_v || !lam_psi || !lam_phi ||
      !work || m < 1 || m > 64 || n_rows < m || n_rows > 4096)
    return HYROM_EINVAL;
  if (ctx->f32) return fail(ctx, HYROM_EINVAL, "the reduced-step adjoint runs on FP64 contexts");
  hy::launch_reduced_vjp(ctx->N, ctx->nc, m, (const double*)phi, rows, n_rows, (const double*)v,
                         (const double*)psi, y, s_hat, (const double*)lam, (double*)lam_v,
                         (double*)lam_psi, (double*)lam_phi, (double*)work, ctx->st);
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_stage_select(hyrom_ctx* ctx, const void* eps, uint32_t* g_bitmap,
                                int32_t* n_g) {
  GUARD();
  if (!eps || !g_bitmap) return HYROM_EINVAL;
  const hyrom_config& cf = ctx->cfg;
  hy::launch_select(eps, ctx->f32, ctx->nc, cf.sel_mode, cf.delta, cf.top_frac, ctx->keys,
                    ctx->sel_scratch, g_bitmap, ctx->n_g_dev, ctx->st);
  CKL();
  long long* hl = (long long*)ctx->host;
  CK(cudaMemcpyAsync(hl, ctx->n_g_dev, sizeof(long long), cudaMemcpyDeviceToHost, ctx->st));
  if (hyrom_status s = sync(ctx)) return s;
  if (n_g) *n_g = (int32_t)hl[0];
  return HYROM_OK;
}

hyrom_status hyrom_stage_pod(hyrom_ctx* ctx, const void* window, int32_t w, const void* psi,
                             void* phi_out, double* sigma_out, int32_t* m_eff) {
  GUARD();
  if (!window || !psi || !phi_out || w < 1 || w > ctx->cfg.w) return HYROM_EINVAL;
  std::vector<int> win(w);
  for (int i = 0; i < w; ++i) win[i] = i;
  int me = 0;
  hyrom_status s;
  if (ctx->f32) {
    ctx->gram_dirty = -1;  // every live row is formed again below
    // raw Gram of the caller's window (all pairs), psi given explicitly
    for (int i = 0; i < w; ++i)
      hy::launch_gram_row<float>((const float*)window, ctx->N, w, i, ctx->Hpart, ctx->gram_chunks,
                                 ctx->H, ctx->st);
    s = pod_t<float>(ctx, (const float*)window, w, win, (const float*)psi, nullptr,
                     (float*)phi_out, (float*)ctx->ftmp, &me);
  } else {
    s = pod_t<double>(ctx, (const double*)window, w, win, (const double*)psi, nullptr,
                      (double*)phi_out, nullptr, &me);
  }
  if (s) return s;
  if (sigma_out)
    CK(cudaMemcpyAsync(sigma_out, ctx->sig, w * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  if (m_eff) *m_eff = me;
  if (ctx->f32 && ctx->k >= 0) {
    // the ring Gram rows were overwritten: rebuild them for the live ring
    CK(cudaMemsetAsync(ctx->H, 0, (size_t)ctx->nslot * ctx->nslot * sizeof(double), ctx->st));
    const int64_t lo = ctx->k - ctx->w > 0 ? ctx->k - ctx->w : 0;
    for (int64_t j = lo; j <= ctx->k; ++j) gram_update<float>(ctx, j);
  }
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_stage_odeim(hyrom_ctx* ctx, const void* phi, int32_t m, int32_t n_p,
                               int32_t* points_out) {
  GUARD();
  if (!phi || !points_out || m < 1 || m > ctx->cfg.m || n_p < m || n_p > 1024) return HYROM_EINVAL;
  int rc;
  const int bs = ctx->cfg.odeim_batch;
  if (ctx->f32)
    rc = hy::launch_odeim<float>((const float*)phi, ctx->N, m, n_p, ctx->cfg.tie_tol, points_out,
                                 ctx->od_ws, (char*)ctx->host + 256, ctx->st, nullptr, nullptr,
                                 false, nullptr, nullptr, bs);
  else
    rc = hy::launch_odeim<double>((const double*)phi, ctx->N, m, n_p, ctx->cfg.tie_tol,
                                  points_out, ctx->od_ws, (char*)ctx->host + 256, ctx->st, nullptr,
                                  nullptr, false, nullptr, nullptr, bs);
  if (rc < 0) return fail(ctx, HYROM_ECUDA, "ODEIM: %s", cudaGetErrorString(cudaGetLastError()));
  CKL();
  return sync(ctx);
}

hyrom_status hyrom_stage_masks(hyrom_ctx* ctx, const uint32_t* g_bitmap, const int32_t* points,
                               int32_t n_p, uint32_t* s_hat, uint32_t* s_tilde, int32_t* n_s) {
  GUARD();
  if (!s_hat || !s_tilde || n_p < 0 || (n_p > 0 && !points)) return HYROM_EINVAL;
  int64_t ns = 0;
  hyrom_status s = ctx->f32 ? masks_and_tiles<float>(ctx, g_bitmap, points, n_p, s_hat, s_tilde, &ns)
                            : masks_and_tiles<double>(ctx, g_bitmap, points, n_p, s_hat, s_tilde, &ns);
  if (s) return s;
  if (n_s) *n_s = (int32_t)ns;
  return HYROM_OK;
}

}  // extern "C"
