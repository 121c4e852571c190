"""Initial data of the paper's Euler test problems, pointwise (oracle).

Problem descriptions are plain dicts (built by the seeded input generators):
  {"kind": "radial", "center": (..), "radius": R, "inner": (rho, vel.., p),
   "outer": (rho, vel.., p), "cell_rho_factor": array over cells or None}
      Sec. 5.8 Eq. (RP3D) explosion (inner state for r <= R); its 2D circular
      analogue uses the same rule.  An optional per-cell density factor
      multiplies rho inside each cell (seeded noise, constant per cell).
  {"kind": "planar", "normal": (n_1, .., n_d), "offset": c, "inner": (rho,
   vel.., p), "outer": (..)}: the inner state where n . x < c (a planar front,
      the oblique shock of the double-Mach problem, Sec. 5.4), else outer.
  {"kind": "quadrant", "center": (xc, yc), "states": 4 x (rho, u, v, p),
   "vortex": None or {"center": (xv, yv), "strength": beta}}
      Sec. 5.6: state 1 for x > xc and y > yc, 2 for x <= xc and y > yc,
      3 for x <= xc and y <= yc, 4 for x > xc and y <= yc.
      Optional isentropic vortex of Sec. 5.2 superposed on the quadrant state.

Vortex (Sec. 5.2): du = -y' beta/(2 pi) e^{(1-r^2)/2}, dv = x' beta/(2 pi)
e^{(1-r^2)/2}, T = p/rho + dT, rho <- rho (T/T0)^{1/(gamma-1)}, p = rho T.
Reading: the printed temperature perturbation carries beta where the radial
momentum balance dp/dr = rho v_theta^2 / r of a steady vortex (the paper's
statement that the vortex is an exact, translating solution) requires beta^2:
dT = -(gamma - 1) beta^2 / (8 gamma pi^2) e^{1 - r^2}.  The tests check that
balance numerically.
"""
import numpy as np

from . import euler


def vortex_perturbation(xp, yp, beta, gamma):
    r2 = xp * xp + yp * yp
    e = np.exp(0.5 * (1.0 - r2))
    du = -yp * beta / (2.0 * np.pi) * e
    dv = xp * beta / (2.0 * np.pi) * e
    dT = -(gamma - 1.0) * beta * beta / (8.0 * gamma * np.pi * np.pi) * e * e
    return du, dv, dT


def primitive(problem, X, gamma, cell_index=None):
    """Primitive fields (rho, [vel..], p) at points X = (x, y[, z]) arrays.
    `cell_index` (tuple of integer arrays, same shape) selects the per-cell
    density factor of radial problems."""
    kind = problem["kind"]
    dim = len(X)
    if kind == "radial":
        c = problem["center"]
        r2 = sum((X[k] - c[k]) ** 2 for k in range(dim))
        inside = r2 <= problem["radius"] ** 2
        si, so = problem["inner"], problem["outer"]
        rho = np.where(inside, si[0], so[0])
        vel = [np.where(inside, si[1 + k], so[1 + k]) for k in range(dim)]
        p = np.where(inside, si[1 + dim], so[1 + dim])
        fac = problem.get("cell_rho_factor")
        if fac is not None:
            rho = rho * fac[cell_index]
        return rho, vel, p
    if kind == "planar":
        nrm, off = problem["normal"], problem["offset"]
        behind = sum(nrm[k] * X[k] for k in range(dim)) < off
        si, so = problem["inner"], problem["outer"]
        rho = np.where(behind, si[0], so[0])
        vel = [np.where(behind, si[1 + k], so[1 + k]) for k in range(dim)]
        p = np.where(behind, si[1 + dim], so[1 + dim])
        return rho, vel, p
    if kind == "quadrant":
        xc, yc = problem["center"]
        x, y = X[0], X[1]
        st = np.asarray(problem["states"], dtype=np.float64)
        q = np.where(x > xc, np.where(y > yc, 0, 3), np.where(y > yc, 1, 2))
        rho, u, v, p = st[q, 0], st[q, 1], st[q, 2], st[q, 3]
        vx = problem.get("vortex")
        if vx is not None:
            du, dv, dT = vortex_perturbation(x - vx["center"][0], y - vx["center"][1],
                                             vx["strength"], gamma)
            T0 = p / rho
            T = T0 + dT
            rho = rho * (T / T0) ** (1.0 / (gamma - 1.0))
            p = rho * T
            u = u + du
            v = v + dv
        return rho, [u, v], p
    raise ValueError(kind)


def conserved(problem, X, gamma, cell_index=None):
    rho, vel, p = primitive(problem, X, gamma, cell_index)
    return euler.prim_to_cons(rho, vel, p, gamma)


def vortex_exact(problem, X, t, gamma, domain_lo, domain_len):
    """Exact solution of a pure translating vortex (all quadrant states equal,
    periodic box): the initial data shifted by velocity * t, wrapped."""
    st = problem["states"][0]
    u0, v0 = st[1], st[2]
    xs = domain_lo[0] + np.mod(X[0] - u0 * t - domain_lo[0], domain_len[0])
    ys = domain_lo[1] + np.mod(X[1] - v0 * t - domain_lo[1], domain_len[1])
    return conserved(problem, (xs, ys), gamma)
