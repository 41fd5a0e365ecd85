// Host-side launchers shared between the translation units of libhyrom.
// Not part of the public ABI (include/hyrom.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hyrom.h"

namespace hy {

struct DevCfg;

// Kernel-launch counter (api.cu): kernels of a replayed graph are added.
// launch_count: all threads; thread_launch_count: the calling thread's.
unsigned long long launch_count();
unsigned long long thread_launch_count();
void add_launches(unsigned long long n);

// The stream a context was created with (api.cu).
void* ctx_stream(const hyrom_ctx* ctx);
// batching (api.cu): with defer on, a rebuild that has an oversampling loop
// describes it (ctx_pending_over) and returns before the loop's consumers;
// after the loop has run, ctx_finish_rebuild completes the rebuild (its
// status and step info are those hyrom_update_basis would have returned).
struct OdeimOver;
void ctx_set_defer(hyrom_ctx* ctx, bool on);
const OdeimOver* ctx_pending_over(const hyrom_ctx* ctx);
bool ctx_is_f32(const hyrom_ctx* ctx);
hyrom_status ctx_finish_rebuild(hyrom_ctx* ctx, hyrom_step_info* info);
void ctx_drop_pending(hyrom_ctx* ctx);  // the loop did not run: forget the rebuild's rest

// Raise the dynamic shared memory limit of kernel `func` on the current
// device to at least `bytes`.  The limit is a per-function global shared by
// all host threads; it is only ever raised (under a lock), so that a launch
// never meets a limit another thread lowered for a smaller instance between
// its own setting and its launch.
void smem_at_least(const void* func, size_t bytes);

// A stream's work kept as a CUDA graph: captured at the first run, replayed
// after.  Whatever the work bakes in (pointers, sizes) must be the same on
// every run.  Launch counts: the launches made while capturing stand for the
// first replay, later replays add `launches`.
struct GraphSlot {
  void* exec = nullptr;  // cudaGraphExec_t
  unsigned long long launches = 0;
};
inline void graph_slot_free(GraphSlot* g) {
  if (g->exec) cudaGraphExecDestroy((cudaGraphExec_t)g->exec);
  g->exec = nullptr;
  g->launches = 0;
}
// Run `body` (stream work only, no synchronisation) on s: replay the slot's
// graph, or capture body into it and launch that; if the stream cannot be
// captured (the legacy default stream), run body directly.
template <typename F>
void run_graphed(GraphSlot* g, cudaStream_t s, F body) {
  if (g->exec) {
    cudaGraphLaunch((cudaGraphExec_t)g->exec, s);
    add_launches(g->launches);
    return;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
      cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    body();
    return;
  }
  const unsigned long long before = thread_launch_count();
  body();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  const unsigned long long n = thread_launch_count() - before;
  cudaGraphExec_t ge = nullptr;
  if (e != cudaSuccess || !graph || cudaGraphInstantiate(&ge, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    body();  // the captured work did not run
    return;
  }
  cudaGraphDestroy(graph);
  g->exec = (void*)ge;
  g->launches = n;
  cudaGraphLaunch(ge, s);
}

// hdm.cu
template <typename T>
void launch_rk2(const DevCfg& c, const T* q, T* out, int64_t k, const uint32_t* mask,
                const int* tiles, const int* ntiles_dev, cudaStream_t s);
// Reverse-sweep pieces (adjoint.cu), FP64.  box: {i0, i1, j0, j1}.
void launch_pressure_vjp(const DevCfg& c, const double* q, const int* box, double w, double* lam,
                         cudaStream_t s);
void launch_box_pressure(const DevCfg& c, const double* q, const int* box, double w,
                         double* part, double* total, cudaStream_t s);
void launch_filter_vjp(const DevCfg& c, const uint32_t* keeps, const int* orders, int npass,
                       double* lam, double* tmp1, double* tmp2, cudaStream_t s);
void launch_center_states(const double* states, int64_t N, const int* win, int w, int wp,
                          const double* psi, double* X, cudaStream_t s);
void launch_tsdots(const double* A, int na, const double* B, int nb, int64_t N, double* part,
                   double* out, cudaStream_t s);
size_t tsdots_part_doubles(int na, int nb);
void launch_pod_vjp_apply(int64_t N, int m, int wp, int w, const double* L, const double* X,
                          const double* B1, const double* B2, const int* win,
                          const double* lpsi_new, double* lam, double* lpsi_cur, cudaStream_t s);
void launch_mean_vjp(int64_t N, const int* win, int w, const double* lpsi, double* lam,
                     cudaStream_t s);

// The paper's HDM (muscl.cu): MUSCL-minmod-Roe residual of BDF2 (BDF1 when
// qp2 is null) on listed cells (null = all; compact SoA output), its exact
// JVP, the filter's residual measure, and a Newton-GMRES solver with its
// own workspace for up to max_cells unknown cells.  FP64.
struct MusclSolver;
MusclSolver* muscl_create(int64_t nc, int64_t max_cells);
void muscl_destroy(MusclSolver* m);
size_t muscl_bytes(const MusclSolver* m);
void launch_muscl_residual(const DevCfg& c, const double* q, const double* qp, const double* qp2,
                           double t, const int* cells, int64_t n, double* out, cudaStream_t s);
void launch_muscl_jvp(const DevCfg& c, const double* q, const double* dv, double t, double a2,
                      double dtb, const int* cells, int64_t n, double* out, cudaStream_t s);
void launch_muscl_rho(const DevCfg& c, const double* q, const double* qp, const double* qp2,
                      double t, double* rho, cudaStream_t s);
int muscl_newton(MusclSolver* m, const DevCfg& c, double* q, const double* qp,
                 const double* qp2, int64_t k, const int* cells, int64_t n, double tol_abs,
                 int newton_max, double eta, cudaStream_t s, int* iters_out, int* arnoldi_out);
int muscl_filter(MusclSolver* m, const DevCfg& c, double* q, const double* qp, const double* qp2, int64_t k,
                 const int* orders, int n_filt, int jmax_f, double eps_f, double* g,
                 double* tmp, double* rho_old, double* rho_new, double* part, double* out3,
                 double* host3, cudaStream_t s);
// FP32 full SSP-RK2 step of the 2D Euler equations streamed by warp strips
// (hdm_f32.cu); rk2_euler_sweep_ok tells whether it takes the grid.
bool rk2_euler_sweep_ok(const DevCfg& c);
void launch_rk2_euler_sweep(const DevCfg& c, const float* q, float* out, int64_t k,
                            cudaStream_t s);
// Euler cells with rho <= 0 or p <= 0 or not finite, added to *count.
template <typename T>
void launch_count_nonphys(const DevCfg& c, const T* q, int* count, cudaStream_t s);
int rk2_tile_width(const DevCfg& c);
int rk2_tile_height(const DevCfg& c);
template <typename T>
void launch_cell_residual(const DevCfg& c, const T* q, const T* qp, int64_t k, T* rho,
                          const uint32_t* only, cudaStream_t s);
template <typename T>
void launch_cell_residual_skip(const DevCfg& c, const T* q, const T* qp, int64_t k, T* rho,
                               const int* skip, cudaStream_t s);
void launch_newton_tol(const DevCfg& c, const double* qp, double newton_tol, double* tol_dev,
                       cudaStream_t s);
void launch_burgers_newton_full(const DevCfg& c, const double* up, double* u,
                                const double* tol_dev, int newton_max, double* ws, int* fail,
                                cudaStream_t s);
void launch_burgers_newton_partial(const DevCfg& c, const double* up, double* u,
                                   const uint32_t* s_hat, int* starts, int* nstart,
                                   const double* tol_dev, int newton_max, double* ws, int* fail,
                                   cudaStream_t s);

// adjoint.cu: lam_in = (d q_k / d q_prev)^T lam_out for the SSP-RK2 Euler
// step k (FP64), restricted to the cells of mask (the partial step; the
// other cells pass lam_out through) or the full step (mask null); work
// holds 3 N doubles
void launch_rk2_vjp(const DevCfg& c, const double* q, const double* lam_out, double* lam_in,
                    const uint32_t* mask, int64_t k, double* work, cudaStream_t s);

// adjoint.cu: the reduced step's adjoint (reconstruction on the dofs
// outside S-hat and the gappy coordinates on `rows`), FP64, m <= 64,
// Phi column-major N x m; work: reduced_vjp_work_doubles(m, nr) doubles
void launch_reduced_vjp(int64_t N, int64_t nc, int m, const double* phi, const int* rows, int nr,
                        const double* v, const double* psi, const double* y,
                        const uint32_t* s_hat, const double* lam, double* lam_v, double* lam_psi,
                        double* lam_phi, double* work, cudaStream_t s);
size_t reduced_vjp_work_doubles(int m, int nr);

// filter.cu
// fargs: device memory (64 bytes) for the per-call arguments; graph
// (nullable): the passes kept as one CUDA graph (the other arguments must
// then be the same on every call).  tape_keeps (nullable): record each pass
// run (keep bitmap of ceil(Nc/32) words, Shapiro n in tape_orders, count in
// *tape_count); recording calls launch directly, outside the graph.
template <typename T>
void launch_filter_sparse(const DevCfg& c, const int* orders, int norders, int jmax_f,
                          double eps_f, T* q, const T* qp, int64_t k, T* gbuf, uint32_t* kbits,
                          int* tiles_a, int* tiles_b, int* counts, double* part, int* ctl,
                          void* fargs, GraphSlot* graph, cudaStream_t s,
                          uint32_t* tape_keeps = nullptr, int* tape_orders = nullptr,
                          int* tape_count = nullptr);

// rom.cu
template <typename T>
void launch_gappy_pinv(const T* phi, int64_t N, int m, const int* pts, int np, double* pinv,
                       int* status, cudaStream_t s);
size_t gappy_pinv_smem(int m, int np);
template <typename T>
void launch_gappy_apply(const double* pinv, int m, int np, const int* pts, const T* v,
                        const T* psi, double* y, const double* y_prev, double* dy,
                        cudaStream_t s, const int* rank_flag = nullptr);
template <typename T>
void launch_reconstruct(const T* phi, int64_t N, int64_t nc, int m, const double* y,
                        const T* psi, const uint32_t* s_hat, int only_set, T* q, cudaStream_t s);
template <typename T>
void launch_cell_error(const T* g, const T* psi, const T* phi, int64_t nc, int nvar, int m,
                       const double* y, T* eps, cudaStream_t s);
template <typename T>
void launch_gram_row(const T* ring, int64_t N, int nslot, int s, double* part, int max_chunks,
                     double* H, cudaStream_t st);
// rows s1 and s2 of H in one pass over the ring (the same bits as two
// launch_gram_row calls); part holds 2 * nslot * max_chunks doubles
template <typename T>
void launch_gram_rows2(const T* ring, int64_t N, int nslot, int s1, int s2, double* part,
                       int max_chunks, double* H, cudaStream_t st);
void launch_gram_center(const double* H, int nslot, const int* win, int w, const int* ps,
                        int npsi, double* G, int ldg, double* xraw2, cudaStream_t s);
void launch_gram_center_explicit(const double* H, int nslot, const int* win, int w,
                                 const double* hp, const double* pp, double* G, int ldg,
                                 double* xraw2, cudaStream_t s);
template <typename T>
void launch_dots(const T* a, const T* ring, int64_t N, int nslot, double* part, int max_chunks,
                 double* out, cudaStream_t st);
template <typename T>
void launch_pod_coeffs(const double* lam, const double* V, int n, int w, int m, double pod_tol,
                       double pod_abs, const double* xraw2, double* sig_out, int* m_eff_out,
                       T* C, cudaStream_t s);
template <typename T>
void launch_form_phi(const T* ring, int64_t N, const int* win, int w, const T* psi, const T* C,
                     int m, const int* m_eff_dev, T* phi, T* psi_next, cudaStream_t s);
template <typename T>
void launch_center_window(const T* ring, int64_t N, const int* win, int w, int wp, const T* psi,
                          double* X, double* raw_part, double* raw_out, cudaStream_t s);
size_t hestenes_scratch_doubles(int wp);
void launch_hestenes_round(double* X, int64_t N, int wp, double* V, int r, double tol,
                           int* rotated, double* scratch, cudaStream_t s);
void launch_identity(double* V, int n, cudaStream_t s);
int run_jacobi_multi(const double* A, int n, double* V, double* lam, double* buf, int* flag,
                     int* host_flag, double* scale_dev, double* host_scale, int max_sweeps,
                     cudaStream_t s);
// Row-norm data ODEIM orders its rows by (odeim.cu); the basis product can
// form it in its epilogue.
constexpr int kNormBucketCount = 256;
struct OdeimNorms {
  float* nrm;          // N upper bounds of the squared row norms
  unsigned char* bkt;  // N bucket ids
  int* bcnt;           // 257 bucket counts (zeroed before the producer runs)
  unsigned int* bmax;  // 256 bucket maxima (bits of the FP32 bounds; zeroed likewise)
};
// Phi = (X - psi 1^T) C and psi_next on the tensor cores (formphi_tc.cu):
// FP32 ring, N % 4 == 0, w <= 128, m <= 64.  *err is set if a pipeline wait
// timed out.  With norms.nrm != NULL the epilogue also forms ODEIM's
// row-norm data for the new Phi.
bool form_phi_tc_ok(int64_t N, int w, int m);
void launch_form_phi_tc(const float* ring, int64_t N, int nslot, const int* win, int w,
                        const float* psi, const float* C, int m, const int* m_eff_dev,
                        float* phi, float* psi_next, int* err, OdeimNorms norms,
                        cudaStream_t s);
// scratch (doubles) run_psd_eig needs at order n
size_t psd_eig_scratch_doubles(int n);
// fp32_pre: FP32 preconditioning sweeps first (the FP32 POD's window
// Gram, where eigenvalues accurate to eps times the largest suffice)
int run_psd_eig(const double* G, int n, double* V, double* lam, double* buf, int* flag,
                int* host_flag, int max_sweeps, cudaStream_t s, int* host_rank = nullptr,
                bool fp32_pre = false);
void launch_colnorm2(const double* X, int64_t N, int ncol, double* out, cudaStream_t s);
template <typename T>
void launch_phi_from_columns(const double* X, int64_t N, int wp, const double* C,
                             const int* m_eff, int m, T* phi, cudaStream_t s);
template <typename T>
void launch_window_mean(const T* ring, int64_t N, const int* win, int w, T* out, cudaStream_t s);
template <typename T>
void launch_sign_fix(T* phi, int64_t N, int m, const int* m_eff, cudaStream_t s);

// select.cu
void launch_select(const void* eps, int is_f32, int64_t nc, int mode, double delta,
                   double top_frac, unsigned long long* keys, void* scratch, uint32_t* g_bitmap,
                   long long* n_g_dev, cudaStream_t s);
size_t select_scratch_bytes();
void launch_masks(const DevCfg& c, const uint32_t* g_bitmap, const int* pts, int np, int halo,
                  int stencil_r, uint32_t* base, uint32_t* s_hat, uint32_t* s_tilde,
                  long long* n_s_dev, cudaStream_t s);
void launch_active_tiles(const DevCfg& c, const uint32_t* bm, int TX, int TY, int* tiles,
                         int* ntiles, cudaStream_t s);
void launch_bits_to_list(const uint32_t* bm, int64_t nc, long long* cnt_scratch, int* out,
                         int64_t cap, cudaStream_t s);
// *out = number of set bits of bm (nwords words)
void launch_popcount(const uint32_t* bm, int64_t nwords, long long* out, cudaStream_t s);

// reduced.cu: sample-row reduced solve (normal equations on all dof rows
// of the listed cells; red = HYROM_RED_* precision of the normal matrix;
// fail[0]: not positive definite, fail[1]: a device wait gave up)
size_t sample_part_doubles();
template <typename T>
void launch_sample_normal(const T* phi, int64_t N, int m, const int* cells, int ns, int nvar,
                          int64_t nc, int red, double* part, double* G, double* L, double* dinv,
                          int* fail, cudaStream_t s);
template <typename T>
void launch_sample_solve(const T* phi, int64_t N, int m, const int* cells, int ns, int nvar,
                         int64_t nc, const T* v, const T* psi, double* part, double* b,
                         const double* L, const double* dinv, double* y, const double* y_prev,
                         double* dy, cudaStream_t s);
// reduced_tc.cu: CTA partials of the normal matrix on the tensor cores
// (red = HYROM_RED_TF32, _BF16 or _TF32_SPLIT) to part[b * 4096 ...];
// returns the number of partials; *err = 1 if a wait gave up
int launch_sample_gram_tc(const float* phi, int64_t N, int m, const int* cells, int ns, int nvar,
                          int64_t nc, int red, double* part, int* err, cudaStream_t s);

// odeim.cu.  norms_ready: the row-norm bounds, bucket ids and bucket counts
// and maxima (OdeimNorms) were already formed for phi (by the basis product).
// graphs (nullable): the DEIM loop and the oversampling loop are captured as
// CUDA graphs at the first call with a given (N, m, n_p) and replayed after;
// the arguments baked into them (phi, pts, ws, tie_tol) must then be the
// same on every call.  Inside a replayed loop no sub-stage marks are made.
struct OdeimGraphs {
  GraphSlot deim, over;
  int64_t N = -1;
  int m = -1, np = -1, bs = -1;
};
void odeim_graphs_free(OdeimGraphs* g);
OdeimNorms odeim_norm_bufs(void* ws, int64_t N);
// One instance's oversampling loop, described for a launch that runs the
// loops of several instances together (launch_odeim_multi) instead of being
// run by launch_odeim.  Pointers are device pointers into the instance's
// ODEIM workspace; the struct is copied to the device as it is.
struct OdeimOver {
  int active;  // 1: the loop has steps (np > m) and was left to the caller
  int m_cap;   // upper bound of m over the instance's calls (sizes the update's grids)
  const void* phi;  // T*, N x m column-major
  int64_t N;
  int m, np, probe, C;
  double tie_tol;
  float* wt32;
  const float* nrm;
  const int* ord;
  unsigned char* picked;
  const unsigned* bmax;
  const int* bstart;
  void* ctl;  // the control block
  double* scores;
  int* list;
  int* xlist;
  const float* R;
  double* lam[2];  // eigenvalues of M, read at even / odd steps (the other is written)
  double* W[2];    // eigenvectors likewise
  int* cand;
  int* pts;
  void* r1;  // the rank-one update's work block
  double* Wrot;
  double* Delta;
};
// over (nullable): if given, launch_odeim runs DEIM and the first
// eigensystem, then describes the oversampling loop in *over instead of
// running it (over->active = 0 when there is none).  bsel > 1: the
// oversampling takes the bsel best rows per scoring pass (a cheaper variant,
// not the paper's greedy); its loop is then always run here.
template <typename T>
int launch_odeim(const T* phi, int64_t N, int m, int np, double tie_tol, int* pts, void* ws,
                 void* host_pinned, cudaStream_t s, void (*mark)(void*, int) = nullptr,
                 void* mark_arg = nullptr, bool norms_ready = false,
                 OdeimGraphs* graphs = nullptr, OdeimOver* over = nullptr, int bsel = 1);
// Several instances' oversampling loops (all of element type T) run
// together: one launch per pass over all instances, a CTA's instance found
// from a work list, replayed from a CUDA graph; the rows-per-CTA of the
// scoring passes picked by timing candidates on the first calls.  Results
// are those of each loop run alone.  Returns 0, or -1 on a CUDA error.
struct OdeimMulti;
OdeimMulti* odeim_multi_create();
void odeim_multi_free(OdeimMulti* mu);
template <typename T>
int launch_odeim_multi(OdeimMulti* mu, const OdeimOver* const* inst, int n, cudaStream_t s);
// the autotuner's state: the rows per CTA in use (0 while still timing) and
// the measured ms per greedy step of each candidate (nc entries, -1 untimed)
int odeim_multi_tuning(const OdeimMulti* mu, int* rows_per_cta, float* ms, int nc);
size_t odeim_ws_bytes(int64_t N, int m);
void odeim_stats(const void* ws, unsigned long long* out4, cudaStream_t s);
void odeim_eig_sweeps(const void* ws, int* out, cudaStream_t s);

}  // namespace hy
