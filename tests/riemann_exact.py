"""Exact solution of the 1D Euler Riemann problem for an ideal gas (test
infrastructure), written from the textbook construction (Toro, Riemann
Solvers and Numerical Methods for Fluid Dynamics, ch. 4), which the paper
names as the source of the exact Sod and Lax solutions (Sec. 5.1):
  * the star pressure p* solves f_L(p) + f_R(p) + u_R - u_L = 0, where f_K is
    the shock branch sqrt(A_K / (p + B_K)) (p - p_K) for p > p_K and the
    rarefaction branch 2 c_K / (gamma - 1) ((p / p_K)^((gamma-1)/(2 gamma)) - 1)
    otherwise, with A_K = 2 / ((gamma + 1) rho_K), B_K = (gamma-1)/(gamma+1) p_K;
  * u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2;
  * the solution is self-similar in x/t and sampled wave by wave.
"""
import numpy as np


def _f(p, rho, pk, ck, gamma):
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        val = (p - pk) * np.sqrt(A / (p + B))
        der = np.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:
        e = (gamma - 1.0) / (2.0 * gamma)
        val = 2.0 * ck / (gamma - 1.0) * ((p / pk) ** e - 1.0)
        der = (1.0 / (rho * ck)) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return val, der


def star_state(left, right, gamma=1.4, tol=1e-14):
    """(p*, u*) of the Riemann problem with primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    if 2.0 * (cl + cr) / (gamma - 1.0) <= ur - ul:
        raise ValueError("vacuum generated")
    p = max(tol, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _f(p, rl, pl, cl, gamma)
        fr, dr = _f(p, rr, pr, cr, gamma)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        pn = max(pn, tol)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, cl, gamma)
    fr, _ = _f(p, rr, pr, cr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, s, gamma=1.4):
    """Primitive (rho, u, p) at the similarity coordinates s = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    ps, us = star_state(left, right, gamma)
    g1, g2 = (gamma - 1.0) / (gamma + 1.0), (gamma - 1.0) / (2.0 * gamma)
    s = np.asarray(s, dtype=np.float64)
    rho, u, p = np.empty_like(s), np.empty_like(s), np.empty_like(s)
    for idx, x in np.ndenumerate(s):
        if x <= us:                                         # left of the contact
            if ps > pl:                                     # left shock
                sl = ul - cl * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + g2)
                st = (rl, ul, pl) if x <= sl else (rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps)
            else:                                           # left rarefaction
                cs = cl * (ps / pl) ** g2
                if x <= ul - cl:
                    st = (rl, ul, pl)
                elif x >= us - cs:
                    st = (rl * (ps / pl) ** (1.0 / gamma), us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * (ul - x))
                    uu = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * ul + x)
                    st = (rl * (c / cl) ** (2.0 / (gamma - 1.0)), uu, pl * (c / cl) ** (1.0 / g2))
        else:                                               # right of the contact
            if ps > pr:                                     # right shock
                sr = ur + cr * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + g2)
                st = (rr, ur, pr) if x >= sr else (rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps)
            else:                                           # right rarefaction
                cs = cr * (ps / pr) ** g2
                if x >= ur + cr:
                    st = (rr, ur, pr)
                elif x <= us + cs:
                    st = (rr * (ps / pr) ** (1.0 / gamma), us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) * (cr - 0.5 * (gamma - 1.0) * (ur - x))
                    uu = 2.0 / (gamma + 1.0) * (-cr + 0.5 * (gamma - 1.0) * ur + x)
                    st = (rr * (c / cr) ** (2.0 / (gamma - 1.0)), uu, pr * (c / cr) ** (1.0 / g2))
        rho[idx], u[idx], p[idx] = st
    return rho, u, p
