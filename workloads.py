"""Seeded synthetic workloads for the hybrid-snapshot adaptive ROM.

This module is the only code shared by the CUDA path's tests/bench and the
CPU oracle.  It holds *inputs only*: run parameters, analytic initial
conditions, the fixed time step chosen from them, and the constants of the
exact planar-shock boundary state.  None of the method's arithmetic (fluxes,
residuals, POD, ODEIM, selection, filtering) lives here.

Random draws use splitmix64 (Steele, Lea & Flood 2014) on a 64-bit seed, so
every workload is reproducible bit for bit on any machine.

Workloads (paper sections in brackets):
  * burgers_sine   - 1D inviscid Burgers, periodic, u0 = 1 + A sin(2 pi x)
                     (conservation law of Sec. 2.1 with c = 1).
  * euler_vortex   - 2D Euler (Sec. 3.1), periodic isentropic vortex plus a
                     Gaussian density pulse.
  * euler_oblique_shock - 2D Euler, planar Mach-3 shock at a seeded angle,
                     exact-solution inflow on the left/bottom sides and
                     zero-gradient outflow on the right/top sides.
  * euler_riemann_x - 1D-in-x Riemann problem (Sod, Sec. 3.2) used by pins.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict, replace

import numpy as np

# --- enumerations shared with the C ABI (include/hyrom.h) -------------------
PDE_BURGERS, PDE_EULER = 0, 1
SCHEME_BE, SCHEME_RK2 = 0, 1            # backward Euler (BDF1), SSP-RK2
SCHEME_BDF2_MUSCL = 2                   # the paper's HDM (MUSCL-Roe, BDF2)
BC_PERIODIC, BC_OUTFLOW, BC_SHOCK = 0, 1, 2
SEL_RRE, SEL_TOPFRAC = 0, 1             # RRE threshold delta, top fraction
PREC_F64, PREC_F32 = 0, 1
ROWS_ODEIM, ROWS_SAMPLE = 0, 1          # regression rows of the reduced solve
RED_F32, RED_TF32, RED_BF16, RED_TF32_SPLIT = 0, 1, 2, 3   # sample-row normal matrix precisions

MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """One splitmix64 step: returns (new_state, 64-bit output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class Rng:
    """U[0,1) draws from splitmix64 (53-bit mantissa)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def uniform(self, lo=0.0, hi=1.0):
        self.state, z = splitmix64(self.state)
        return lo + (hi - lo) * ((z >> 11) * (1.0 / (1 << 53)))


@dataclass
class ArConfig:
    """Run parameters of Algorithm 1 plus the HDM definition."""
    pde: int = PDE_EULER
    scheme: int = SCHEME_RK2
    nx: int = 64
    ny: int = 64
    dx: float = 1.0
    dy: float = 1.0
    dt: float = 1e-3
    gamma: float = 1.4
    bc: tuple = (BC_PERIODIC,) * 4      # left, right, bottom, top
    # exact planar shock used by BC_SHOCK sides: the state at x is `post`
    # where n.x < d0 + speed*t, else `pre` (conserved variables)
    shock_n: tuple = (1.0, 0.0)
    shock_d0: float = 0.0
    shock_speed: float = 0.0
    shock_pre: tuple = (1.0, 0.0, 0.0, 2.5)
    shock_post: tuple = (1.0, 0.0, 0.0, 2.5)
    # Algorithm 1 parameters
    w: int = 8
    m: int = 4
    z: int = 0                          # 0 means z = infinity
    n_p: int = 8
    sel_mode: int = SEL_TOPFRAC
    delta: float = 0.9
    top_frac: float = 0.05
    halo: int = 0
    eps_y: float = 1e-4
    jmax: int = 10
    eps_f: float = 1e-2
    jmax_f: int = 10
    filt_orders: tuple = (1, 2, 3)      # Shapiro n: orders 2n = 2, 4, 6
    pod_tol: float = 1e-10
    pod_abs: float = 1e-13
    tie_tol: float = 1e-12
    newton_tol: float = 1e-13
    newton_max: int = 50
    regress_rows: int = ROWS_ODEIM
    reduced_prec: int = RED_F32
    # ODEIM oversampling points taken per scoring pass (1: the paper's greedy,
    # one point per pass; b > 1: the b best rows of each pass, a cheaper variant)
    odeim_batch: int = 1
    precision: int = PREC_F64
    seed: int = 0

    @property
    def nvar(self) -> int:
        return 1 if self.pde == PDE_BURGERS else 4

    @property
    def ncell(self) -> int:
        return self.nx * self.ny

    @property
    def ndof(self) -> int:
        return self.nvar * self.ncell

    def as_dict(self):
        return asdict(self)

    def with_(self, **kw):
        return replace(self, **kw)


# --- Euler helpers (primitive -> conserved; wave speed for the time step) ---

def _conserved(gamma, rho, u, v, p):
    E = p / ((gamma - 1.0) * rho) + 0.5 * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, rho * E])


def _cfl_dt(gamma, q, dx, dy, cfl):
    rho, mx, my, en = q
    u, v = mx / rho, my / rho
    p = (gamma - 1.0) * (en - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(gamma * p / rho)
    rate = (np.abs(u) + c) / dx + (np.abs(v) + c) / dy
    return float(cfl / rate.max())


def burgers_sine(n=1024, seed=1, steps=200, **kw):
    """1D Burgers on periodic [0,1]: u0 = 1 + A sin(2 pi x), A ~ U[0.3, 0.7].

    Time step dt = 0.5 dx / max|u0| (CFL 0.5).  Basis k = 10 from the last
    20 snapshots, top 10 % of cells plus a 2-cell halo, n_p = 2k points.
    Returns (q0 [1, n], cfg, steps).
    """
    rng = Rng(seed)
    amp = rng.uniform(0.3, 0.7)
    x = (np.arange(n) + 0.5) / n
    u0 = 1.0 + amp * np.sin(2.0 * np.pi * x)
    dx = 1.0 / n
    cfg = ArConfig(pde=PDE_BURGERS, scheme=SCHEME_BE, nx=n, ny=1, dx=dx, dy=1.0,
                   dt=0.5 * dx / float(np.abs(u0).max()), bc=(BC_PERIODIC,) * 4,
                   w=20, m=10, z=0, n_p=20, sel_mode=SEL_TOPFRAC, top_frac=0.10,
                   halo=2, precision=PREC_F64, seed=seed)
    cfg = replace(cfg, **kw)
    return u0.reshape(1, n), cfg, steps


def euler_vortex(n=512, seed=2, steps=500, minf=0.5, **kw):
    """2D Euler on periodic [0,10]^2: isentropic vortex (strength 5, centre
    (5,5)) advected at Mach `minf` (0.5) along the diagonal, plus a Gaussian
    density pulse of amplitude 0.2 and radius 0.5 at a seeded point of
    [2,8]^2 with the pressure unchanged.  CFL 0.5, k = 20, w = 40, 5 % sample.
    Returns (q0 [4, n*n] cell index x-fastest, cfg, steps)."""
    gamma = 1.4
    rng = Rng(seed)
    xp, yp = rng.uniform(2.0, 8.0), rng.uniform(2.0, 8.0)
    L = 10.0
    dx = L / n
    xc = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc, indexing="xy")          # X varies along axis 1
    beta = 5.0
    cinf = math.sqrt(gamma)
    uinf = minf * cinf / math.sqrt(2.0)
    vinf = uinf
    xr, yr = X - 5.0, Y - 5.0
    r2 = xr * xr + yr * yr
    g = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = uinf - g * yr
    v = vinf + g * xr
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    rho = rho + 0.2 * np.exp(-((X - xp) ** 2 + (Y - yp) ** 2) / 0.25)
    q0 = _conserved(gamma, rho, u, v, p).reshape(4, n * n)
    dt = _cfl_dt(gamma, q0, dx, dx, 0.5)
    cfg = ArConfig(pde=PDE_EULER, scheme=SCHEME_RK2, nx=n, ny=n, dx=dx, dy=dx, dt=dt,
                   gamma=gamma, bc=(BC_PERIODIC,) * 4, w=40, m=20, z=0, n_p=40,
                   sel_mode=SEL_TOPFRAC, top_frac=0.05, halo=0,
                   pod_tol=1e-6, pod_abs=1e-6, precision=PREC_F32, seed=seed)
    cfg = replace(cfg, **kw)
    return q0, cfg, steps


def euler_batch(n_inst=64, seed=5, nmin=128, nmax=1024, kmin=8, kmax=48, fmin=0.02,
                fmax=0.20, mach=(0.3, 2.0)):
    """The batching form: n_inst independent Euler instances, each the
    vortex-plus-pulse problem (euler_vortex) on an n x n grid with n drawn
    log-uniformly from [nmin, nmax] (so cell counts are log-uniform too),
    free-stream Mach ~ U[mach], its own basis size k ~ U{kmin..kmax} with
    w = n_p = 2k, and its own sample fraction ~ U[fmin, fmax] (uneven masks).
    Returns a list of (q0, cfg)."""
    rng = Rng(seed)
    out = []
    for i in range(n_inst):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        m_inf = rng.uniform(*mach)
        k = kmin + int(rng.uniform(0.0, 1.0) * (kmax - kmin + 1))
        k = min(k, kmax)
        frac = rng.uniform(fmin, fmax)
        q0, cfg, _ = euler_vortex(n=n, seed=seed * 1000 + i, minf=m_inf, w=2 * k, m=k,
                                  n_p=2 * k, top_frac=frac)
        out.append((q0, cfg))
    return out


# Parameters of the differentiation form's initial state, in order: vortex
# strength beta, vortex centre x0, y0, vortex radius R, pulse amplitude,
# pulse centre xp, yp, free-stream Mach number.  The default centre sits
# off the grid's mirror lines: a vortex centred on a face line gives mirror
# cells equal wave speeds, where the Rusanov flux is not differentiable.
VORTEX_THETA_NAMES = ("beta", "x0", "y0", "radius", "pulse_amp", "pulse_x", "pulse_y", "mach")
VORTEX_THETA0 = (5.0, 5.13, 4.87, 1.0, 0.2, 3.5, 6.0, 0.5)


def euler_vortex_theta(n, theta, gamma=1.4, L=10.0):
    """The isentropic vortex plus density pulse of euler_vortex as a function
    of its parameters theta (VORTEX_THETA_NAMES) on the periodic [0, L]^2
    with n x n cells: with r = |x - x_c| / R,
      u = u_inf - beta/(2 pi) exp((1 - r^2)/2) (y - y0)/R,
      v = v_inf + beta/(2 pi) exp((1 - r^2)/2) (x - x0)/R,
      T = 1 - (gamma - 1) beta^2 / (8 gamma pi^2) exp(1 - r^2),
      rho = T^(1/(gamma - 1)) + A exp(-|x - x_p|^2 / 0.25),  p = T^(gamma/(gamma-1)),
    free stream along the diagonal at Mach M (|u_inf| = M sqrt(gamma)).
    R = 1 and theta = (5, 5, 5, 1, 0.2, xp, yp, 0.5) give euler_vortex.
    Every operation is analytic in theta, so a complex theta gives the
    derivative by the complex step.  Returns q0 [4, n*n]."""
    beta, x0, y0, R, amp, xp, yp, mach = theta
    dx = L / n
    xc = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    cinf = math.sqrt(gamma)
    uinf = mach * cinf / math.sqrt(2.0)
    xr, yr = (X - x0) / R, (Y - y0) / R
    r2 = xr * xr + yr * yr
    g = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = uinf - g * yr
    v = uinf + g * xr
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    rho = rho + amp * np.exp(-((X - xp) ** 2 + (Y - yp) ** 2) / 0.25)
    return _conserved(gamma, rho, u, v, p).reshape(4, n * n)


def normal_shock_states(gamma, mach, rho1, p1):
    """Pre/post states of a normal shock of Mach `mach` moving into gas at
    rest (Rankine-Hugoniot jump relations).  Returns (rho2, u2, p2, speed)."""
    c1 = math.sqrt(gamma * p1 / rho1)
    speed = mach * c1
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    u2 = speed * (1.0 - rho1 / rho2)
    return rho2, u2, p2, speed


def euler_oblique_shock(n=2048, seed=3, steps=20, k=64, frac=0.05, **kw):
    """2D Euler on [0,1]^2: a planar Mach-3 shock at angle theta ~ U[25,35]
    degrees moving into still gas (rho = 1.4, p = 1).  The shock passes
    through (0.3, 0.3) at t = 0.  Left/bottom sides take the exact moving
    shock state as Dirichlet data; right/top sides are zero-gradient outflow.
    k POD modes from w = 2k snapshots, n_p = 2k points, top `frac` of cells.
    Returns (q0 [4, n*n], cfg, steps)."""
    gamma = 1.4
    rng = Rng(seed)
    theta = math.radians(rng.uniform(25.0, 35.0))
    nvec = (math.cos(theta), math.sin(theta))
    rho1, p1 = 1.4, 1.0
    rho2, u2, p2, speed = normal_shock_states(gamma, 3.0, rho1, p1)
    d0 = 0.3 * (nvec[0] + nvec[1])
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    post = (nvec[0] * X + nvec[1] * Y) < d0
    rho = np.where(post, rho2, rho1)
    u = np.where(post, u2 * nvec[0], 0.0)
    v = np.where(post, u2 * nvec[1], 0.0)
    p = np.where(post, p2, p1)
    q0 = _conserved(gamma, rho, u, v, p).reshape(4, n * n)
    pre_q = tuple(float(a) for a in _conserved(gamma, np.array(rho1), np.array(0.0),
                                               np.array(0.0), np.array(p1)))
    post_q = tuple(float(a) for a in _conserved(gamma, np.array(rho2), np.array(u2 * nvec[0]),
                                                np.array(u2 * nvec[1]), np.array(p2)))
    dt = _cfl_dt(gamma, q0, dx, dx, 0.5)
    cfg = ArConfig(pde=PDE_EULER, scheme=SCHEME_RK2, nx=n, ny=n, dx=dx, dy=dx, dt=dt,
                   gamma=gamma, bc=(BC_SHOCK, BC_OUTFLOW, BC_SHOCK, BC_OUTFLOW),
                   shock_n=nvec, shock_d0=d0, shock_speed=speed,
                   shock_pre=pre_q, shock_post=post_q,
                   w=2 * k, m=k, z=0, n_p=2 * k, sel_mode=SEL_TOPFRAC, top_frac=frac,
                   halo=0, pod_tol=1e-6, pod_abs=1e-6, precision=PREC_F32, seed=seed)
    cfg = replace(cfg, **kw)
    return q0, cfg, steps


def euler_riemann_x(n=200, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.5,
                    cfl=0.5, **kw):
    """Riemann problem along x on [0,1] (one cell high, outflow sides).
    left/right are primitive (rho, u, p); Sod's tube by default (Sec. 3.2).
    Returns (q0 [4, n], cfg)."""
    gamma = 1.4
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    L = xc < x0
    rho = np.where(L, left[0], right[0])
    u = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    q0 = _conserved(gamma, rho, u, np.zeros_like(u), p).reshape(4, n)
    dt = _cfl_dt(gamma, q0, dx, 1e30, cfl)
    cfg = ArConfig(pde=PDE_EULER, scheme=SCHEME_RK2, nx=n, ny=1, dx=dx, dy=1.0, dt=dt,
                   gamma=gamma, bc=(BC_OUTFLOW,) * 4, precision=PREC_F64)
    cfg = replace(cfg, **kw)
    return q0, cfg


def random_field(shape, seed, lo=-1.0, hi=1.0):
    """Seeded uniform array (numpy PCG64 seeded from splitmix64)."""
    _, s = splitmix64(seed)
    return np.random.Generator(np.random.PCG64(s)).uniform(lo, hi, size=shape)


def random_spectrum_window(nrow, w, seed, decay=0.5, offset=1.0):
    """Snapshot window X = offset + U diag(sigma) V^T with orthonormal U, V
    and sigma_j = decay**j: a window of known, well-separated spectrum for
    POD tests.  Returns (X [nrow, w], sigma)."""
    g = np.random.Generator(np.random.PCG64(splitmix64(seed)[1]))
    U, _ = np.linalg.qr(g.standard_normal((nrow, w)))
    V, _ = np.linalg.qr(g.standard_normal((w, w)))
    sig = decay ** np.arange(w)
    return offset + (U * sig) @ V.T, sig


def splitmix64_array(seed: int, n: int) -> np.ndarray:
    """The first n splitmix64 outputs of `seed`, vectorised (uint64 numpy
    arithmetic wraps modulo 2^64 exactly as the scalar generator does)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def front_basis(nrow, m, seed, period=700, width=90.0):
    """A localised N x m basis like one POD builds around a moving front,
    made only from splitmix64 draws and IEEE-exact operations (+, -, *, /), so
    that it is the same bits on every machine: column j is uniform noise in
    [-1/2, 1/2) times the rational bump 1 / (1 + (d / width)^2) + 1e-3 of the
    distance d = (row mod period) - c_j to a seeded centre c_j.  Not
    orthonormal (the point-selection stages do not need it).  Returns
    float64 [nrow, m]."""
    u = (splitmix64_array(seed, nrow * m) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    u = u.reshape(nrow, m) - 0.5
    cj = (splitmix64_array(seed ^ 0x5DEECE66D, m) % np.uint64(period)).astype(np.float64)
    d = (np.arange(nrow) % period).astype(np.float64)[:, None] - cj[None, :]
    t = d / width
    return u * (1.0 / (1.0 + t * t) + 1e-3)
