"""Plain FP64 CPU oracle of the hybrid-snapshot adaptive ROM (Zucatti & Zahr,
"An adaptive, training-free reduced-order model for convection-dominated
problems based on hybrid snapshots").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg do.  It
shares no code with the CUDA path (paper_2301_01718_gb300/); the only common
module is workloads.py, which holds seeded inputs and no method arithmetic.

Every function follows the paper's definitions in the paper's order, with
numpy/LAPACK primitives (matmul, SVD, eigh, lstsq, solve) as steps and no
blocking or fusion.  Where the paper is silent the reading taken is stated in
the docstring of the function that takes it.

Modules
  hdm     - conservation laws, FV fluxes, residual R_k (Eq. hdm), BDF1 /
            SSP-RK2 steps, partial HDM (Eq. partial_hdm2)          [Sec. 2.1-2.3]
  rom     - POD_m (Eq. pod), gappy coordinates (Eq. red_coord), DEIM and
            ODEIM points (Eq. odeim), reference state (Eq. mean)   [Sec. 2.3.1]
  select  - reconstruction error, RRE ordering and threshold (Eq. rre),
            sampling-set algebra (union, setdiff, Neighbors)        [Sec. 2.3.3, 2.4]
  filt    - Shapiro filters and the residual-gated filter loop     [Sec. 2.3.4]
  arom    - Algorithm 1 driver and the metrics of Sec. 3.1
  tangent - tangent-linear model of Algorithm 1 with the forward run's
            decisions held (the differentiation form): JVPs of the HDM
            step, gappy coordinates, POD and filter; dJ/dtheta of a
            time-integrated output
  adjoint - its reverse mode: the transposes of those JVPs and one
            reverse sweep over the recorded run for dJ/dq0
  hdm_muscl - the paper's own HDM: MUSCL + minmod + Roe, BDF2 solved by
            Newton-GMRES                                      [Sec. 3.1]
"""
