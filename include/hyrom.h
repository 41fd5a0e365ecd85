/*
 * hyrom.h - C ABI of the GB300 (sm_103a) hybrid-snapshot adaptive ROM.
 *
 * The method is Algorithm 1 of Zucatti & Zahr, "An adaptive, training-free
 * reduced-order model for convection-dominated problems based on hybrid
 * snapshots": at each time step the high-dimensional model (HDM) is solved
 * only on a sampled set of cells (Sec. 2.3, Eq. partial_hdm2), the rest of
 * the state is rebuilt from an on-the-fly POD basis by gappy least squares
 * at ODEIM points (Sec. 2.3.1, Eqs. red_coord, pod, odeim, mean), the mixed
 * state is passed through residual-gated Shapiro filters (Sec. 2.3.4), and
 * the next sampled set is chosen from the pointwise reconstruction error
 * (Sec. 2.3.3, Eq. rre).
 *
 * Conventions (all entry points):
 *   - A state is an array of nvar*Nc values in structure-of-arrays layout,
 *     q[v*Nc + cell], cell = j*nx + i (x fastest).  Nc = nx*ny; nvar = 1
 *     (Burgers) or 4 (Euler: rho, rho u, rho v, rho E).
 *   - "dev" pointers are CUDA device pointers on the device current when the
 *     context was created; "host" pointers are ordinary host memory (pinned
 *     memory gives the fastest copies).  Arrays of the state type ("real")
 *     hold double when the context precision is HYROM_PREC_F64 and float
 *     when it is HYROM_PREC_F32.
 *   - The caller keeps ownership of every pointer it passes; the library
 *     never retains one past the call (q0 is copied).  The context owns all
 *     of its device workspaces (allocated by hyrom_init, freed by
 *     hyrom_destroy).
 *   - Work is enqueued on the stream given to hyrom_init (a cudaStream_t
 *     passed as void*; NULL = the legacy default stream).  Calls return
 *     after their work is enqueued unless they return host-side counts, in
 *     which case they synchronise that stream.
 *   - No entry point aborts or throws.  Each returns a hyrom_status; the
 *     message of the last failure is available from hyrom_last_error().  A
 *     CUDA error makes the context unusable (HYROM_ECUDA is sticky).
 *   - One context must not be used by two host threads at once.
 */
#ifndef HYROM_H
#define HYROM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HYROM_OK = 0,
  HYROM_EINVAL = 1,    /* bad argument or configuration                     */
  HYROM_ENOMEM = 2,    /* device allocation failed                          */
  HYROM_ECUDA = 3,     /* a CUDA call failed; the context is unusable      */
  HYROM_ENOTCONV = 4,  /* a Newton solve hit newton_max (result still set)  */
  HYROM_ESTATE = 5,    /* call out of order (e.g. no basis yet)             */
  HYROM_ECAP = 6,      /* output buffer too small                           */
  HYROM_ETIMEOUT = 7,  /* an iterative device solver hit its sweep limit    */
  HYROM_ERANK = 8,     /* information, the call completed: the window has
                          rank below m (POD kept m_eff < m modes, Sec.
                          2.3.1) or P^T Phi is rank-deficient             */
  HYROM_ENONPHYS = 9   /* the call completed but the Euler state has cells
                          with rho <= 0 or p <= 0 (or not finite)          */
} hyrom_status;

enum { HYROM_PDE_BURGERS = 0, HYROM_PDE_EULER = 1 };
/* Time schemes: BDF1 (backward Euler, Burgers, Godunov flux), SSP-RK2
 * (Rusanov flux), and the paper's own HDM (Sec. 3.1): MUSCL reconstruction of
 * the primitive variables with the minmod limiter and the Roe flux, BDF2 of
 * Eq. bdf (BDF1 for the first step), each step solved by Newton-GMRES with
 * exact Jacobian-vector products (Euler, FP64). */
enum { HYROM_SCHEME_BE = 0, HYROM_SCHEME_RK2 = 1, HYROM_SCHEME_BDF2_MUSCL = 2 };
enum { HYROM_BC_PERIODIC = 0, HYROM_BC_OUTFLOW = 1, HYROM_BC_SHOCK = 2 };
enum { HYROM_SEL_RRE = 0, HYROM_SEL_TOPFRAC = 1 };
enum { HYROM_PREC_F64 = 0, HYROM_PREC_F32 = 1 };
/* Regression rows of the reduced solve: the ODEIM rows P (the paper's
 * form), or every dof row of the sample cells S-hat (which contain P). */
enum { HYROM_ROWS_ODEIM = 0, HYROM_ROWS_SAMPLE = 1 };
/* Precision of the sample-row normal matrix Phi_S^T Phi_S: FP32 products
 * on the CUDA cores (FP64 for FP64 states), or on the tensor cores TF32
 * products (inputs rounded to nearest, relative error 2^-11), BF16 products
 * (2^-8), or FP32-level products of a TF32 hi/lo split of each input; always
 * accumulated in at least FP32, factored and solved in FP64. */
enum { HYROM_RED_F32 = 0, HYROM_RED_TF32 = 1, HYROM_RED_BF16 = 2, HYROM_RED_TF32_SPLIT = 3 };

/* Run parameters.  HDM: Sec. 2.2 (Eqs. semi_disc, bdf, hdm) with
 * first-order FV fluxes (Burgers: Godunov; Euler, Sec. 3.1: Rusanov) and
 * BDF1 (backward Euler, Newton) or SSP-RK2 time stepping.  Boundary sides
 * are ordered left, right, bottom, top; HYROM_BC_SHOCK imposes the exact
 * planar shock: the state is shock_post where n.x < shock_d0 +
 * shock_speed*t, else shock_pre (conserved variables).
 * Algorithm 1: w snapshots, m POD modes, full HDM every z steps (z <= 0:
 * never after the warm-up), n_p ODEIM points; selection by the RRE
 * threshold delta (Eq. rre) or the top fraction top_frac of cells, then
 * dilation by `halo` cells; subiterations stop at ||dy||_2 < eps_y or jmax
 * (Sec. 2.3.2); filter passes stop at a relative decrease below eps_f or
 * jmax_f passes (Sec. 2.3.4) for each Shapiro order filt_orders[0..n_filt)
 * (n = 1, 2, 3 for orders 2, 4, 6).  POD keeps mode j when
 * sigma_j > pod_tol*sigma_1 and sigma_j > pod_abs*||X_raw||_F.  Arg-max ties
 * within relative tie_tol go to the lowest index.  The reduced coordinates
 * are fitted on the rows regress_rows selects (HYROM_ROWS_*), the sample-row
 * normal matrix in precision reduced_prec (HYROM_RED_*; the tensor-core
 * precisions need FP32 states).  odeim_batch (0 or 1: the paper's ODEIM, one
 * greedy point per scoring pass, Eq. odeim; 2..16: a cheaper variant that is
 * not the paper's, taking the odeim_batch best rows of each pass, ties to the
 * lowest index, before updating the sampled Gram matrix with all of them). */
typedef struct {
  int32_t pde, scheme, precision, nx, ny;
  int32_t bc[4];
  double dx, dy, dt, gamma;
  double shock_n[2], shock_d0, shock_speed, shock_pre[4], shock_post[4];
  int32_t w, m, z, n_p, sel_mode, halo, jmax, jmax_f, newton_max, n_filt;
  int32_t filt_orders[3], regress_rows, reduced_prec, odeim_batch;
  double delta, top_frac, eps_y, eps_f, pod_tol, pod_abs, tie_tol, newton_tol;
  uint64_t seed;
} hyrom_config;

/* What one call of hyrom_step / hyrom_advance / hyrom_update_basis did. */
typedef struct {
  int64_t k;            /* step index of the snapshot now held (gamma_k)   */
  int32_t was_full;     /* 1: full HDM solve (Algorithm 1)                  */
  int32_t rebuilt;      /* 1: basis, points and sets rebuilt               */
  int32_t J;            /* subiterations of the partial HDM (Sec. 2.3.2)   */
  int32_t n_s;          /* cells of S-hat used by this step                 */
  int32_t n_g;          /* cells picked by the error indicator (next step)  */
  int32_t n_p;          /* ODEIM points in effect                           */
  int32_t m_eff;        /* POD modes in effect                              */
  int32_t filt_passes;  /* filter passes run                                */
  int32_t newton_fail;  /* Newton solves that hit newton_max                */
  int32_t pad;
  double dy_last;       /* ||y^(J) - y^(J-1)||_2 of the last subiteration   */
} hyrom_step_info;

typedef struct hyrom_ctx hyrom_ctx;

/* ---- context lifetime ----------------------------------------------------
 * hyrom_init: validate cfg, allocate the context's device workspaces (the
 * w+1 snapshot ring, basis, points, masks, filter and reduction buffers)
 * and copy q0 (nvar*Nc doubles, host or device per q0_on_host) into
 * gamma_0 (the initial state of Algorithm 1), converting to the context
 * precision.
 * Errors: HYROM_EINVAL (bad config; *out untouched), HYROM_ENOMEM,
 * HYROM_ECUDA.  On error no context is returned. */
hyrom_status hyrom_init(const hyrom_config* cfg, const double* q0, int q0_on_host,
                        void* stream, hyrom_ctx** out);
void hyrom_destroy(hyrom_ctx* ctx);
const char* hyrom_last_error(const hyrom_ctx* ctx);
/* Bytes of device memory the context holds. */
size_t hyrom_device_bytes(const hyrom_ctx* ctx);
/* Kernels this library has launched since it was loaded (all contexts of
 * the process; counted on the host at each launch). */
uint64_t hyrom_kernel_launches(void);

/* Per-stage timing.  hyrom_profile(ctx, 1) creates CUDA events and from
 * then on records one pair on the context stream around each stage of
 * Algorithm 1 (ids below); the elapsed times are summed at the
 * synchronisation points of hyrom_advance / hyrom_update_basis.
 * hyrom_profile(ctx, 0) stops recording; both reset the totals.
 * hyrom_stage_times copies the totals (ms[HYROM_NSTAGE], and the number of
 * intervals into count[HYROM_NSTAGE] when count is not NULL). */
enum {
  HYROM_T_FULL = 0,     /* full HDM step                                   */
  HYROM_T_PARTIAL = 1,  /* partial HDM on S-hat                            */
  HYROM_T_GAPPY = 2,    /* gappy coordinates                               */
  HYROM_T_RECON = 3,    /* reconstruction on S-breve                       */
  HYROM_T_FILTER = 4,   /* SpatialFilter                                   */
  HYROM_T_SELECT = 5,   /* error indicator and G_{k+1}                     */
  HYROM_T_GRAM = 6,     /* ring Gram row of a new snapshot (FP32 POD)      */
  HYROM_T_EIG = 7,      /* window Gram centring + eigensolve (POD)         */
  HYROM_T_FORMPHI = 8,  /* basis formation and next psi                    */
  HYROM_T_ODEIM = 9,    /* ODEIM oversampling and the sampled pseudo-inverse */
  HYROM_T_MASKS = 10,   /* union / dilation / Neighbors                    */
  HYROM_T_DEIM = 11,    /* DEIM points, the first m of ODEIM               */
  /* parts of HYROM_T_DEIM / HYROM_T_ODEIM: */
  HYROM_T_OD_INIT = 12,   /* row-norm buckets + first eigensystem          */
  HYROM_T_OD_PROBE = 13,  /* bounds of the largest-norm rows, one exact   */
  HYROM_T_OD_SCREEN = 14, /* bounds from z_1, z_2 of the rows still open   */
  HYROM_T_OD_EXACT = 15,  /* exact scores, tie-aware pick, update setup    */
  HYROM_T_OD_UPDATE = 16, /* rank-one eigensystem update                   */
  HYROM_T_OD_LIST = 17,   /* full FP32 bounds of the rows passed on        */
  HYROM_T_SNORMAL = 18,   /* sample-row normal matrix and its factor       */
  HYROM_NSTAGE = 19
};
hyrom_status hyrom_profile(hyrom_ctx* ctx, int on);
/* Work counters of the last ODEIM call (rebuild or stage entry point):
 * out4[0] rows scored exactly by DEIM beyond the probe, out4[1] rows given
 * the full certified FP32 bound in oversampling (the probe rows and those the
 * z_1 bound does not exclude), out4[2] exact FP64 secular solves in
 * oversampling, out4[3] oversampling steps.  Synchronises. */
hyrom_status hyrom_odeim_counters(hyrom_ctx* ctx, int64_t* out4);
/* Sweeps of the one-sided Jacobi eigensolver (pivoted Cholesky, then
 * rotations of the factor's columns until no pair is rotated; at most 60) in
 * the last rebuild: out2[0] the POD eigenproblem of the window Gram matrix
 * (FP32 contexts; 0 for FP64 contexts, whose POD is a one-sided Jacobi SVD
 * of the window itself), out2[1] ODEIM's first m x m eigensystem (0 before
 * the first ODEIM call).  Synchronises. */
hyrom_status hyrom_eig_sweeps(hyrom_ctx* ctx, int32_t* out2);
hyrom_status hyrom_stage_times(const hyrom_ctx* ctx, double* ms, int64_t* count);

/* ---- Algorithm 1 --------------------------------------------------------
 * hyrom_advance: the advance part of Algorithm 1 for k+1: a full HDM step
 * or a hybrid step (predictor, partial HDM with subiterations, gappy coordinates,
 * reconstruction on S-breve, SpatialFilter).  Errors: HYROM_ESTATE when a
 * hybrid step is due but no basis exists, HYROM_ENOTCONV (state still
 * advanced), HYROM_ECUDA.
 * hyrom_update_basis: the basis-update part for the current k: psi initialisation,
 * G_{k+1} by the error indicator, POD_m, ODEIM_{n_p}, union / setdiff /
 * Neighbors, psi_{k+1}; does nothing when the rebuild test is false.
 * hyrom_step = hyrom_advance then hyrom_update_basis (one loop iteration).
 * info may be NULL.  These calls synchronise the stream once per call (they
 * return counts in info).
 * Statuses that report on a completed step: hyrom_advance returns
 * HYROM_ENONPHYS when the new Euler snapshot has cells with rho <= 0 or
 * p <= 0 (checked on every step; the state is kept so that it can be
 * inspected, but the run has left the ideal-gas model); hyrom_update_basis
 * returns HYROM_ERANK when a rebuild kept m_eff < m modes (Sec. 2.3.1, the
 * window's numerical rank) or found P^T Phi rank-deficient, which is
 * information only: the basis in effect is valid and the run may go on.
 * hyrom_step returns a failure of the rebuild first, then the advance's
 * status, then HYROM_ERANK. */
hyrom_status hyrom_advance(hyrom_ctx* ctx, hyrom_step_info* info);
hyrom_status hyrom_update_basis(hyrom_ctx* ctx, hyrom_step_info* info);
hyrom_status hyrom_step(hyrom_ctx* ctx, hyrom_step_info* info);

/* Checkpoint / resume.  hyrom_save writes the context's state that carries
 * from one step to the next (the step index, the w+1 snapshots, the basis,
 * psi, the ODEIM points and the sampled pseudo-inverse, the sampled sets and
 * the active tiles, the snapshot Gram matrix, the sample-row factor) to the
 * file `path` (binary, this library's layout; about (w + 1 + m) states).
 * hyrom_load reads such a file into a context created with the same grid,
 * scheme, precision, sides, w, m, n_p and regression rows (its other run
 * parameters are its own); the next hyrom_step continues the saved run
 * exactly.  Both synchronise the stream.  Errors: HYROM_EINVAL (null path,
 * file not opened, written or of another layout), HYROM_ENOMEM (pinned
 * staging buffer), HYROM_ECUDA.  The paper has no counterpart. */
hyrom_status hyrom_save(hyrom_ctx* ctx, const char* path);
hyrom_status hyrom_load(hyrom_ctx* ctx, const char* path);

/* hyrom_sample: the sampled set S-hat in effect for the next step, as
 * ascending cell ids in idx_dev (capacity cap; HYROM_ECAP if larger; the
 * count is always written to *n_out) and, when bitmap_dev is not NULL, as a
 * bitmap of ceil(Nc/32) words (bit c%32 of word c/32).  Algorithm 1, S-hat.
 * HYROM_ESTATE before the first rebuild. */
hyrom_status hyrom_sample(hyrom_ctx* ctx, int32_t* idx_dev, int64_t cap, int64_t* n_out,
                          uint32_t* bitmap_dev);

/* State access: gamma_k as nvar*Nc reals of the context precision. */
hyrom_status hyrom_get_state(hyrom_ctx* ctx, void* q, int q_on_host);
/* Overwrite gamma_k (and its snapshot-Gram entries).  Same layout.  For
 * FP32 contexts the snapshot-Gram row of the new gamma_k is formed by the
 * next Gram update (the next step's, in the same pass over the window as
 * that step's own row) or before the Gram matrix is next read, with the same
 * values as when formed at once. */
hyrom_status hyrom_set_state(hyrom_ctx* ctx, const void* q, int q_on_host);
/* Basis in effect: Phi (ndof x m_eff reals, column-major, device) and
 * *m_eff; psi (ndof reals, device); points (n_p int32 dof rows in the order
 * chosen, device) and *n_p.  Any output pointer may be NULL.
 * HYROM_ESTATE before the first rebuild. */
hyrom_status hyrom_get_basis(hyrom_ctx* ctx, void* phi_dev, int32_t* m_eff, void* psi_dev,
                             int32_t* points_dev, int32_t* n_p);

/* ---- stage entry points --------------------------------------------------
 * Each runs one step of the method on caller arrays (device pointers) with
 * the context's configuration, precision, stream and workspaces, leaving
 * the context's own state untouched.  They exist so that every stage can be
 * checked against an independent implementation on identical inputs.
 * `real` arrays follow the context precision. */

/* Full HDM step gamma_k = F_k(gamma_k) from q_prev (Algorithm 1):
 * SSP-RK2 from t_{k-1} to t_k, or BDF1 solved by Newton (Eq. hdm). */
hyrom_status hyrom_stage_full_step(hyrom_ctx* ctx, const void* q_prev, void* q_out, int64_t k);

/* Partial HDM on S-hat (Eq. partial_hdm2; Algorithm 1): q_io holds
 * the frozen values on the other cells and, for BDF1, the Newton start on
 * S-hat; on return it holds the HDM values on S-hat.  s_hat: bitmap. */
hyrom_status hyrom_stage_partial_step(hyrom_ctx* ctx, const void* q_prev, void* q_io,
                                      const uint32_t* s_hat, int64_t k);

/* Gappy reduced coordinates y = (P^T Phi)^+ P^T (v - psi) (Eq. red_coord)
 * by Householder QR in FP64.  phi: ndof x m (column-major), points: n_p dof
 * rows, y_out: m doubles (device).  Synchronises.  When P^T Phi is
 * rank-deficient (a pivot |R_jj| <= 64 n_p eps max|R_ii|, e.g. two equal rows
 * with n_p = m) every y_j is NaN and the status is HYROM_ERANK. */
hyrom_status hyrom_stage_gappy(hyrom_ctx* ctx, const void* phi, int32_t m, const int32_t* points,
                               int32_t n_p, const void* v, const void* psi, double* y_out);

/* Sample-row reduced coordinates: y minimising ||(Phi y - (v - psi))_S||_2
 * over every dof row of the n_cells cells (device int32, ascending), by the
 * normal equations with the context's reduced_prec normal matrix and an FP64
 * Cholesky solve.  phi: ndof x m (column-major, m <= 64), y_out: m doubles
 * (device).  HYROM_ENOTCONV if the normal matrix is not positive definite. */
hyrom_status hyrom_stage_gappy_rows(hyrom_ctx* ctx, const void* phi, int32_t m,
                                    const int32_t* cells, int32_t n_cells, const void* v,
                                    const void* psi, double* y_out);

/* Reconstruction on S-breve (Algorithm 1): q_io = psi + Phi y on
 * every cell whose bit in s_hat is clear (all cells when s_hat is NULL). */
hyrom_status hyrom_stage_reconstruct(hyrom_ctx* ctx, const void* phi, int32_t m, const double* y,
                                     const void* psi, const uint32_t* s_hat, void* q_io);

/* SpatialFilter (Algorithm 1, Sec. 2.3.4) of q_io in place, with
 * the BDF1 residual relative to q_prev at t_k.  *passes gets the passes
 * run (may be NULL). */
hyrom_status hyrom_stage_filter(hyrom_ctx* ctx, void* q_io, const void* q_prev, int64_t k,
                                int32_t* passes);

/* Pointwise reconstruction error per cell, eps = sum_v (g - psi - Phi y)^2
 * (Sec. 2.3.3); eps_out: Nc reals. */
hyrom_status hyrom_stage_cell_error(hyrom_ctx* ctx, const void* g, const void* psi,
                                    const void* phi, int32_t m, const double* y, void* eps_out);

/* G: the n_g cells first in (descending eps, ascending id) order, n_g from
 * the RRE threshold (Eq. rre) or the top fraction, with eps mapped to exact
 * fixed-point integer keys.  Writes a bitmap (ceil(Nc/32) words) and
 * returns n_g in *n_g (synchronises). */
hyrom_status hyrom_stage_select(hyrom_ctx* ctx, const void* eps, uint32_t* g_bitmap, int32_t* n_g);

/* POD_m (Eq. pod) of the window X (ndof x w, column-major, columns in time
 * order) centred at psi: phi_out gets ndof x m_eff orthonormal columns,
 * sigma_out (device, w doubles, may be NULL) the singular values in
 * descending order, *m_eff the kept rank (synchronises). */
hyrom_status hyrom_stage_pod(hyrom_ctx* ctx, const void* window, int32_t w, const void* psi,
                             void* phi_out, double* sigma_out, int32_t* m_eff);

/* ODEIM_{n_p} (Eq. odeim) of phi (ndof x m): points_out gets n_p dof rows
 * in the order chosen (the m DEIM points first).  With the context's
 * odeim_batch b > 1, the oversampling points are taken b per scoring pass
 * (the cheaper variant described at hyrom_config). */
hyrom_status hyrom_stage_odeim(hyrom_ctx* ctx, const void* phi, int32_t m, int32_t n_p,
                               int32_t* points_out);

/* Sampling sets (Algorithm 1): S-hat = union(G, cells of the
 * points) dilated by cfg.halo; S-tilde = Neighbors(S-hat) (cells within the
 * scheme's stencil reach, 1 for BDF1 and 2 for SSP-RK2, not in S-hat).
 * Bitmaps of ceil(Nc/32) words; *n_s gets |S-hat| (synchronises). */
hyrom_status hyrom_stage_masks(hyrom_ctx* ctx, const uint32_t* g_bitmap, const int32_t* points,
                               int32_t n_p, uint32_t* s_hat, uint32_t* s_tilde, int32_t* n_s);

/* ---- the paper's HDM (contexts with scheme HYROM_SCHEME_BDF2_MUSCL) --------
 * Sec. 3.1: MUSCL reconstruction of (rho, u, v, p) with minmod slopes, Roe
 * flux, BDF2 of Eq. bdf with a0 = 1/3, a1 = -4/3, a2 = 1, beta = 2/3 (BDF1
 * when q_prev2 is NULL), two ghost layers.  All arrays are N doubles (SoA,
 * device); other contexts get HYROM_EINVAL.
 * hyrom_stage_muscl_residual: r_out = R_k(q) of Eq. hdm on every cell.
 * hyrom_stage_muscl_jvp: jv_out = (d R_k / d q) v at q (exact directional
 *   derivative; bdf2 selects beta = 2/3 and a2 = 1, else BDF1), every cell.
 * hyrom_stage_muscl_step: R_k(q) = 0 by Newton-GMRES to max |R| <=
 *   newton_tol max(1, max |q_prev|); s_hat NULL: the full step (q_io is
 *   overwritten, the start is q_prev); else the partial HDM of Eq.
 *   partial_hdm2 on the cells of the bitmap s_hat, q_io holding the start on
 *   them and the frozen values elsewhere.  HYROM_ENOTCONV when a solve hit
 *   newton_max (q_io still updated).
 * hyrom_stage_muscl_filter: SpatialFilter (Sec. 2.3.4) of q_io in place,
 *   gated on R_k of Eq. hdm; *passes (nullable) gets the passes run.
 * All synchronise. */
hyrom_status hyrom_stage_muscl_residual(hyrom_ctx* ctx, const double* q, const double* q_prev,
                                        const double* q_prev2, int64_t k, double* r_out);
hyrom_status hyrom_stage_muscl_jvp(hyrom_ctx* ctx, const double* q, const double* v, int64_t k,
                                   int32_t bdf2, double* jv_out);
hyrom_status hyrom_stage_muscl_step(hyrom_ctx* ctx, const double* q_prev2, const double* q_prev,
                                    double* q_io, const uint32_t* s_hat, int64_t k);
hyrom_status hyrom_stage_muscl_filter(hyrom_ctx* ctx, double* q_io, const double* q_prev,
                                      const double* q_prev2, int64_t k, int32_t* passes);

/* ---- differentiation form ---------------------------------------------------
 * hyrom_stage_rk2_vjp: the adjoint of one SSP-RK2 HDM step of the Euler
 * equations (Sec. 2.2, the explicit scheme; Sec. 3.1, Rusanov flux): with
 * q_k = RK2_k(q_prev) on the cells of s_hat and q_prev elsewhere (the partial
 * HDM step of Algorithm 1; s_hat NULL = every cell, the full step),
 *   lam_in = (d q_k / d q_prev)^T lam_out.
 * Ghost cells: shock sides are fixed states (no share), outflow sides copy
 * their boundary cell (its share goes to that cell), periodic sides wrap;
 * at a tie of the two Rusanov wave speeds the left one is differentiated.
 * q_prev, lam_out, lam_in: N doubles each (dev, SoA), lam_in distinct from
 * both; work: 3 N doubles of device scratch (caller-owned); s_hat: cell
 * bitmap (dev) or NULL.  FP64 Euler SSP-RK2 contexts only (else
 * HYROM_EINVAL).  Synchronises. */
hyrom_status hyrom_stage_rk2_vjp(hyrom_ctx* ctx, const void* q_prev, const void* lam_out,
                                 void* lam_in, const uint32_t* s_hat, int64_t k, void* work);

/* hyrom_stage_reduced_vjp: the adjoint of the reduced step of a hybrid step
 * (Sec. 2.3.1, Eq. red_coord and the reconstruction of Algorithm 1): with
 *   y = argmin |Phi[rows] y - (v - psi)[rows]|   and
 *   v_final = v on the dofs of the cells in s_hat, psi + Phi y elsewhere,
 * a cotangent lam of v_final pulls back to lam_v (of v), lam_psi (of psi) and
 * lam_phi (of Phi), all overwritten.  Phi: N x m column-major doubles
 * (1 <= m <= 64); rows: m <= n_rows <= 4096 distinct dof indices (int32, dev;
 * the ODEIM rows: one CTA forms their normal matrix); y: the
 * m coordinates of the forward step (dev doubles); v, psi, lam, lam_v,
 * lam_psi: N doubles; lam_phi: N x m; work: hyrom_reduced_vjp_work_doubles(m,
 * n_rows) doubles of device scratch.  FP64 contexts only.  Synchronises.
 * Phi[rows] must have full column rank (its normal matrix is factored by
 * Cholesky). */
size_t hyrom_reduced_vjp_work_doubles(int32_t m, int32_t n_rows);
hyrom_status hyrom_stage_reduced_vjp(hyrom_ctx* ctx, const void* phi, int32_t m,
                                     const int32_t* rows, int32_t n_rows, const void* v,
                                     const void* psi, const double* y, const uint32_t* s_hat,
                                     const void* lam, void* lam_v, void* lam_psi, void* lam_phi,
                                     void* work);

/* hyrom_stage_pod_vjp: the adjoint of POD_m (Eq. pod) of one window as
 * hyrom_adjoint applies it (thin-SVD derivative, distinct singular values):
 * for the window X (N x w column-major, w = cfg.w, time order) centred at
 * psi and the cotangent lphi (N x m) of the m kept, signed modes (the POD
 * must keep exactly m), lam_window (N x w, overwritten) gets the cotangent
 * of the window columns and lpsi_out (N, overwritten) that of psi (minus the
 * sum of lam_window's columns).  FP64 contexts.  Synchronises.
 * hyrom_stage_filter_vjp: the adjoint of SpatialFilter (Sec. 2.3.4) at q
 * with the residual relative to q_prev at t_k, the forward passes' keep
 * masks and stops held: the filter runs on a copy of q recording each pass,
 * then lam_io <- the passes' transposes in reverse order applied to lam_io.
 * FP64 Euler SSP-RK2 contexts.  Synchronises. */
hyrom_status hyrom_stage_pod_vjp(hyrom_ctx* ctx, const double* window, int32_t w,
                                 const double* psi, const double* lphi, int32_t m,
                                 double* lam_window, double* lpsi_out);
hyrom_status hyrom_stage_filter_vjp(hyrom_ctx* ctx, const double* q, const double* q_prev,
                                    int64_t k, double* lam_io);

/* hyrom_adjoint: the gradient of the time-integrated box pressure
 *   J = sum_{k=1..steps} dt sum_{box} p(gamma_k) dx dy
 * with respect to the initial state gamma_0, through Algorithm 1 with the
 * forward run's decisions held (the sampled sets, G, the ODEIM points, every
 * filter pass's keep mask and stop, the POD rank and each mode's sign; the
 * bases and reference states are differentiated as functions of the
 * snapshots, by the thin-SVD derivative, distinct singular values).  The
 * context must be at k = 0 (fresh from hyrom_init); the call runs `steps`
 * steps of Algorithm 1 recording what the reverse sweep needs (every state,
 * and per hybrid step the predictor, coordinates, sets and keep masks; about
 * 2 N doubles per step), then one reverse sweep: per step the output term,
 * the transposed filter passes, the reduced step's adjoint, the step adjoint,
 * and per rebuild the POD adjoint (each basis recomputed from its window in
 * reverse) and the window means'.  box: {i0, i1, j0, j1} host int32 (cells
 * [i0, i1) x [j0, j1)); J_out: host double (nullable); dJdq0: N device
 * doubles.  FP64 Euler SSP-RK2 contexts on ODEIM rows.  The context is left
 * at k = steps.  Synchronises.  dJ/dtheta for parameters of the initial
 * state is (dq0/dtheta)^T dJdq0.  Errors: HYROM_EINVAL, HYROM_ESTATE (not at
 * k = 0, or a window of rank below m), HYROM_ENOMEM, HYROM_ECUDA, and those of
 * hyrom_step. */
hyrom_status hyrom_adjoint(hyrom_ctx* ctx, int32_t steps, const int32_t* box, double* J_out,
                           double* dJdq0);

/* ---- batching form ---------------------------------------------------------
 * Many independent instances of Algorithm 1 (each its own context, grid,
 * basis size, window and sample fraction) stepped together by a pool of host
 * threads.  hyrom_batch_create takes n distinct contexts (the caller keeps
 * them: they must outlive the batch and not be used by another thread while
 * a batch call runs) and starts `threads` host threads (0: half the host's
 * hardware threads, between 1 and 8; never more than the number of distinct
 * streams among the contexts).
 * hyrom_batch_step runs `nsteps` calls of hyrom_step on every instance, in
 * the form hyrom_batch_set_mode selects (below).  In the streams form each
 * thread takes one instance at a time, largest device footprint first, and
 * runs its steps on the instance's own stream, so up to `threads` instances
 * are on the GPU at once.  In either form an instance's steps stay in order
 * and compute what they compute when it is stepped alone, so its results are
 * the same bits.
 * Contexts that share a stream (the legacy default stream included) are
 * stepped by one thread in turn, so that a stream being captured into one
 * instance's CUDA graph sees no other instance's work: they keep their
 * results and lose the overlap.  infos (n entries, nullable) receives each
 * instance's last step; status (n entries, nullable) each instance's first
 * non-OK status; an instance stops at a failure other than HYROM_ENOTCONV
 * (HYROM_ERANK, information only, is not reported: see m_eff in infos).
 * Returns when every instance is done (synchronised): HYROM_OK or the first
 * failing instance's status (by index).  Errors of hyrom_batch_create:
 * HYROM_EINVAL (n <= 0, threads < 0, a null or repeated context),
 * HYROM_ENOMEM, HYROM_ECUDA. */
typedef struct hyrom_batch hyrom_batch;
hyrom_status hyrom_batch_create(hyrom_ctx* const* ctxs, int32_t n, int32_t threads,
                                hyrom_batch** out);
/* hyrom_init_batch: n instances at once (the batching form's constructor): for
 * each i a stream of its own (non-blocking) and a context hyrom_init(&cfgs[i],
 * q0[i], q0_on_host, that stream), then hyrom_batch_create over them.  The
 * batch owns these contexts and streams and hyrom_batch_destroy releases them;
 * ctxs_out (nullable, n entries) receives the contexts for state access
 * (the caller must not destroy them).  On failure nothing is left allocated.
 * Errors: those of hyrom_init and hyrom_batch_create, HYROM_ECUDA. */
hyrom_status hyrom_init_batch(const hyrom_config* cfgs, const double* const* q0,
                              int32_t q0_on_host, int32_t n, int32_t threads,
                              hyrom_ctx** ctxs_out, hyrom_batch** out);
hyrom_status hyrom_batch_step(hyrom_batch* batch, int32_t nsteps, hyrom_step_info* infos,
                              int32_t* status);
int32_t hyrom_batch_threads(const hyrom_batch* batch);
/* hyrom_batch_set_mode: how hyrom_batch_step runs a step (Algorithm 1's
 * hybrid step, applied to every instance).
 *   HYROM_BATCH_STREAMS: as described above, each instance's steps run
 *   whole on its own stream, up to `threads` instances at a time.
 *   HYROM_BATCH_FUSED (the default): the instances advance one step at a
 *   time together.
 *   The threads run every instance's step up to its ODEIM oversampling loop
 *   (Sec. 2.3.1, Eq. odeim: the greedy steps after the first m points); the
 *   loops of all instances then run as one launch per pass over all
 *   instances (a CTA finds its instance in a work list in device memory),
 *   replayed from a CUDA graph on a stream of the batch, with the scoring
 *   passes' rows per CTA picked by timing four candidates over the first
 *   eight steps; then the threads finish every instance's step.  Each instance
 *   gets the same points, hence the same results, as stepped alone.
 * Errors: HYROM_EINVAL (null batch, unknown mode).
 * hyrom_batch_tuning: the fused form's autotuner: *rows_per_cta (nullable)
 * receives the rows per CTA in use (0 while still timing), ms_per_step (n
 * entries, nullable) the measured ms per greedy step of each candidate (-1:
 * not timed).  Returns the number of candidates, 0 before the first fused
 * step, -1 for a null batch. */
enum { HYROM_BATCH_STREAMS = 0, HYROM_BATCH_FUSED = 1 };
hyrom_status hyrom_batch_set_mode(hyrom_batch* batch, int32_t mode);
int32_t hyrom_batch_tuning(const hyrom_batch* batch, int32_t* rows_per_cta, float* ms_per_step,
                           int32_t n);
void hyrom_batch_destroy(hyrom_batch* batch);

/* ---- diagnostics -----------------------------------------------------------
 * hyrom_selftest_math: the library's own FP64 reciprocal (which = 0: 1 / x
 * from an FP32 seed and two Newton steps, used where an FP64 division would
 * sit on a dependent chain) and reciprocal square root (which = 1: 1 /
 * sqrt(x), x > 0, likewise) applied to n doubles x (device) into y (device),
 * so that tests can hold them against CUDA's division and square root.
 * Enqueued on `stream` (NULL = legacy default); does not synchronise.
 * Errors: HYROM_EINVAL (null pointer, n < 0, which not 0 or 1),
 * HYROM_ECUDA (launch). */
hyrom_status hyrom_selftest_math(int32_t which, const double* x, double* y, int64_t n,
                                 void* stream);
/* hyrom_probe_fp64: a dense FP64 FMA loop for measuring this GPU's FP64 rate
 * (the roofline of the FP64-bound stages; the paper has no counterpart):
 * `blocks` blocks of 256 threads, each thread 8 independent FMA chains of
 * `iters` steps, i.e. blocks * 256 * 16 * iters flops; out receives one
 * double per thread (device, blocks * 256 entries).  Enqueued on `stream`;
 * the caller times it.  Errors: HYROM_EINVAL, HYROM_ECUDA. */
hyrom_status hyrom_probe_fp64(double* out, int32_t blocks, int32_t iters, void* stream);

/* ---- allocation-free variant ---------------------------------------------
 * hyrom_gappy_static: the gappy reduced coordinates of hyrom_stage_gappy,
 * y = (P^T Phi)^+ P^T (v - psi), for callers that cannot allocate device memory: host applications that
 * budget all device memory up front and pass only pointers into their own
 * pools, plugins that must not use the CUDA allocator of the program that
 * loads them, and time-critical loops where cudaMalloc / cudaFree would add
 * an implicit device synchronisation.  It needs no context and never calls
 * cudaMalloc, cudaFree or an allocating library routine.  The paper has no
 * counterpart: this is a property of the library, not of the method.
 *   phi: ndof x m (column-major), points: n_p dof rows in [0, ndof) (not
 *   checked: the caller guarantees the range), v, psi: ndof values; all
 *   device arrays of `precision` (HYROM_PREC_F64 -> double, HYROM_PREC_F32
 *   -> float) except points (int32).  y_out: m doubles on the device.  Work is
 *   enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and
 *   the call does not synchronise.  A rank-deficient P^T Phi (same
 *   test as hyrom_stage_gappy) sets every y_j to NaN; the status, returned
 *   before the work runs, stays HYROM_OK.
 *   err, err_len: optional caller buffer (may be NULL / 0) that receives a
 *   NUL-terminated reason on failure and an empty string on success.
 * Limits: 1 <= m <= 64 and m <= n_p <= min(128, ndof); other sizes return
 * HYROM_EINVAL before any work is enqueued.
 * Scratch: file-scope device arrays of 64 x 128 doubles plus a counter
 * (about 64 KB), present on every GPU that loads the library until the
 * process exits.  Each call clears the counter itself on `stream`; the
 * pseudo-inverse is written in full before it is read, so nothing needs to
 * start at zero.  Every call on a device shares this scratch: calls whose
 * work can overlap on the GPU (different streams without ordering between
 * them) race on it and must be serialised by the caller.
 * Set-up: the first call on each device (with that device current) looks up
 * the scratch's device address with cudaGetSymbolAddress; make that first
 * call before any stream capture on that device. */
hyrom_status hyrom_gappy_static(const void* phi, int64_t ndof, int32_t m, const int32_t* points,
                                int32_t n_p, const void* v, const void* psi, int32_t precision,
                                double* y_out, void* stream, char* err, int32_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* HYROM_H */
