"""A-posteriori MOOD detector on subcell averages (oracle).

Sec. 4.3:
  PAD  Eq. (positivity): rho > 0 and p > 0.  Read on the subcell averages of
       the candidate, v* = P(u*) ("on a subcell basis" in the Sec. 4.4 summary).
       Comparisons are written so that NaN fails.
  NAD  Eq. (dmp): componentwise  m_i - delta <= v* <= M_i + delta  on every
       subcell, where m_i / M_i are the min / max of the subcell data v^n over
       the Voronoi neighbourhood V_i (the cell and every cell sharing a node
       with it: the 3^d block; wrapped at periodic boundaries; at a reflective
       wall the mirror images of the cells across it take part, with their
       wall-normal momentum bounds negated and swapped; cells outside a
       transmissive or inflow boundary are left out).
  Eq. (relax): delta = eps (M - m), eps = 1e-3.  Reading: a floor is added,
       delta = max(eps (M - m), floor * max(1, |M|, |m|)) with floor = 1e-4.
       The literal Eq. (relax) (floor = 0), or a round-off-only floor such as
       1e-12, flags the smooth isentropic vortex of Sec. 5.2 in its far field
       every step: there the density varies by ~1e-13 across V_i while the
       truncation error of the coupled momentum field moves it by ~1e-10.
       Sec. 5.2 states the limiter stays off on that smooth problem on fine
       enough grids; with floor = 1e-4 it does (pinned by the tests).  The
       floor is a parameter, so the literal relation can still be run.
  beta_i = 1 when PAD or NAD fails in any subcell of cell i.
"""
import numpy as np

from . import euler
from .dg import REFLECTIVE

EPS = 1e-3
FLOOR = 1e-4


def _shift_pad(amin, amax, grid):
    """Pad every cell axis (axes 1..d) of the per-cell minima / maxima by one
    cell: wrap if periodic; at a reflective wall the mirror image of the
    boundary cell (its wall-normal momentum bounds negated and swapped);
    otherwise +inf / -inf, which leaves the outside cell out of V_i.  Axes are
    padded in order, so corner images combine the axes' rules."""
    pmin, pmax = amin, amax
    for k in range(grid.dim):
        ax = 1 + k
        pads = []
        for side, i in ((-1, 0), (1, -1)):
            kind = grid.kind(k, side)
            if grid.periodic(k):
                j = -1 if side < 0 else 0
                lo, hi = np.take(pmin, [j], axis=ax), np.take(pmax, [j], axis=ax)
            elif kind == REFLECTIVE:
                lo, hi = np.take(pmin, [i], axis=ax).copy(), np.take(pmax, [i], axis=ax).copy()
                lo[1 + k], hi[1 + k] = -hi[1 + k], -lo[1 + k]
            else:
                shp = list(pmin.shape)
                shp[ax] = 1
                lo, hi = np.full(shp, np.inf), np.full(shp, -np.inf)
            pads.append((lo, hi))
        pmin = np.concatenate([pads[0][0], pmin, pads[1][0]], axis=ax)
        pmax = np.concatenate([pads[0][1], pmax, pads[1][1]], axis=ax)
    return pmin, pmax


def neighbourhood_bounds(cmin, cmax, grid):
    """(m, M) over V_i from per-cell minima / maxima (shape (nvar, cells...))."""
    pmin, pmax = _shift_pad(cmin, cmax, grid)
    m = np.full(cmin.shape, np.inf)
    M = np.full(cmax.shape, -np.inf)
    d = grid.dim
    for off in np.ndindex(*([3] * d)):
        sl = (slice(None),) + tuple(slice(o, o + grid.ncell[k]) for k, o in enumerate(off))
        m = np.minimum(m, pmin[sl])
        M = np.maximum(M, pmax[sl])
    return m, M


def cell_minmax(V, dim):
    """Per-cell, per-variable min / max over the trailing `dim` subcell axes."""
    axes = tuple(range(V.ndim - dim, V.ndim))
    return V.min(axis=axes), V.max(axis=axes)


def relaxation(m, M, eps=EPS, floor=FLOOR):
    scale = np.maximum(1.0, np.maximum(np.abs(M), np.abs(m)))
    return np.maximum(eps * (M - m), floor * scale)


def detect(vstar, m, M, gamma, dim, eps=EPS, floor=FLOOR):
    """beta (int array over cells): 1 where PAD or the relaxed DMP fails."""
    axes = tuple(range(vstar.ndim - dim, vstar.ndim))
    rho = vstar[0]
    p = euler.pressure(vstar, gamma)
    sub_axes = tuple(a - 1 for a in axes)          # same axes without the variable index
    pad_ok = np.all((rho > 0.0) & (p > 0.0), axis=sub_axes)
    delta = relaxation(m, M, eps, floor)
    exp = (Ellipsis,) + (None,) * dim
    lo = (m - delta)[exp]
    hi = (M + delta)[exp]
    dmp_ok = np.all((vstar >= lo) & (vstar <= hi), axis=axes)   # per variable
    dmp_ok = np.all(dmp_ok, axis=0)
    return (~(pad_ok & dmp_ok)).astype(np.int32)


def admissible(V, gamma, dim):
    """PAD of Eq. (positivity) on subcell data V (nvar, ..., N_s^dim): True
    where rho > 0 and p > 0 on every subcell of the trailing dim axes (NaN
    fails)."""
    axes = tuple(range(V.ndim - 1 - dim, V.ndim - 1))
    ok = (V[0] > 0.0) & (euler.pressure(V, gamma) > 0.0)
    return np.all(ok, axis=axes)


def detector_margin(vstar, m, M, gamma, dim, eps=EPS, floor=FLOOR):
    """Per cell, the smallest relative distance of any detector quantity to its
    threshold: min |x - bound| / max(1, |bound|).  Cells with a margin below
    1e-10 may legitimately flip between two correct FP64 implementations."""
    axes = tuple(range(vstar.ndim - dim, vstar.ndim))
    delta = relaxation(m, M, eps, floor)
    exp = (Ellipsis,) + (None,) * dim
    lo = (m - delta)[exp]
    hi = (M + delta)[exp]
    rel = lambda x, b: np.abs(x - b) / np.maximum(1.0, np.abs(b))
    marg = np.minimum(rel(vstar, lo), rel(vstar, hi)).min(axis=axes).min(axis=0)
    p = euler.pressure(vstar, gamma)
    sub_axes = tuple(a - 1 for a in axes)
    marg = np.minimum(marg, np.minimum(rel(vstar[0], 0.0), rel(p, 0.0)).min(axis=sub_axes))
    return marg
