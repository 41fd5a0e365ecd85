"""Exact solutions used to pin the oracle's HDM (test helper).

* Euler: the exact Riemann solver for the ideal-gas Euler equations, written
  from the gas-dynamics relations (shock Hugoniot and isentropic
  rarefaction branches of the pressure function, star-state pressure by
  bisection, self-similar sampling in x/t).
* Burgers: the entropy solution of a periodic up-step/down-step problem
  (rarefaction fan plus a shock moving at the Rankine-Hugoniot speed
  (uL + uR)/2).
"""
import math

import numpy as np


def _f_branch(p, rho, pk, ck, gamma):
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * ck / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)

    def F(p):
        return _f_branch(p, rl, pl, cl, gamma) + _f_branch(p, rr, pr, cr, gamma) + (ur - ul)

    lo, hi = 1e-12, 1e3 * max(pl, pr)
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if F(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (_f_branch(ps, rr, pr, cr, gamma) - _f_branch(ps, rl, pl, cl, gamma))
    return ps, us


def sample(left, right, xi, gamma=1.4):
    """Primitive (rho, u, p) at x/t = xi for every entry of xi."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    ps, us = star_state(left, right, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, xi.size))
    for n, s in enumerate(xi):
        if s <= us:
            if ps > pl:
                SL = ul - cl * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + (gamma - 1.0) / (2.0 * gamma))
                if s <= SL:
                    out[:, n] = (rl, ul, pl)
                else:
                    out[:, n] = (rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps)
            else:
                shl = ul - cl
                csl = cl * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
                stl = us - csl
                if s <= shl:
                    out[:, n] = (rl, ul, pl)
                elif s >= stl:
                    out[:, n] = (rl * (ps / pl) ** (1.0 / gamma), us, ps)
                else:
                    base = 2.0 / (gamma + 1.0) + (gamma - 1.0) / ((gamma + 1.0) * cl) * (ul - s)
                    out[:, n] = (rl * base ** (2.0 / (gamma - 1.0)),
                                 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * ul + s),
                                 pl * base ** (2.0 * gamma / (gamma - 1.0)))
        else:
            if ps > pr:
                SR = ur + cr * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + (gamma - 1.0) / (2.0 * gamma))
                if s >= SR:
                    out[:, n] = (rr, ur, pr)
                else:
                    out[:, n] = (rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps)
            else:
                shr = ur + cr
                csr = cr * (ps / pr) ** ((gamma - 1.0) / (2.0 * gamma))
                str_ = us + csr
                if s >= shr:
                    out[:, n] = (rr, ur, pr)
                elif s <= str_:
                    out[:, n] = (rr * (ps / pr) ** (1.0 / gamma), us, ps)
                else:
                    base = 2.0 / (gamma + 1.0) - (gamma - 1.0) / ((gamma + 1.0) * cr) * (ur - s)
                    out[:, n] = (rr * base ** (2.0 / (gamma - 1.0)),
                                 2.0 / (gamma + 1.0) * (-cr + 0.5 * (gamma - 1.0) * ur + s),
                                 pr * base ** (2.0 * gamma / (gamma - 1.0)))
    return out


def burgers_step_exact(x, t, a=0.25, b=0.5, uh=2.0):
    """u0 = uh on [a, b), 0 elsewhere (periodic, t <= b - a): a rarefaction
    fan from a and a shock at b + uh t / 2."""
    u = np.zeros_like(x)
    fan = (x >= a) & (x < a + uh * t)
    u[fan] = (x[fan] - a) / t
    plateau = (x >= a + uh * t) & (x < b + 0.5 * uh * t)
    u[plateau] = uh
    return u
