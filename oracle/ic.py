"""Initial DG data, exact subcell averages and initial detection (oracle).

Sec. 4.4 (last paragraph): the initial DG data is the L2 projection of
Q(x, 0); the detector (PAD + relaxed DMP) is applied to it with respect to the
exact initial condition, and cells that fail start with their subcell
representation at t = 0.

Readings:
  * the L2 projection and the exact subcell averages use one composite GL rule
    per cell: N_s equal subintervals (the subcells) times N + 2 GL points per
    axis; the nodal L2 projection is u_i = (1/W_i) int_T Q0 Phi_i (the GL mass
    matrix W is exact for the degree-N basis);
  * DMP bounds at t = 0 come from the exact subcell averages over V_i, the
    candidate is P(u^0);
  * a flagged cell stores the exact subcell averages as v^0 and its DG data
    becomes R(v^0) (a cell with beta = 1 runs DG from R(v^n)).
"""
import numpy as np

from . import detect as det
from .basis import gauss_legendre, lagrange_values
from .problems import conserved
from .step import State


def composite_rule(N):
    """Points / weights on [0, 1]: N_s subintervals x (N+2) GL points."""
    Ns = 2 * N + 1
    xq, wq = gauss_legendre(N + 2)
    pts = ((np.arange(Ns)[:, None] + xq[None, :]) / Ns).ravel()
    wts = np.tile(wq / Ns, Ns)
    return pts, wts


def project_problem(sch, problem):
    """(u0, vexact): nodal L2 projection (nvar, cells..., n^d) and exact
    subcell averages (nvar, cells..., Ns^d) of the problem's initial data."""
    g, N, d = sch.grid, sch.N, sch.dim
    Ns = sch.Ns
    pts, wts = composite_rule(N)
    nq = len(pts)
    Lq = lagrange_values(sch.basis.xi, pts)               # (nq, n)
    # quadrature point coordinates per axis and cell: (n_k, nq)
    coords = [g.x0[k] + (np.arange(g.ncell[k])[:, None] + pts[None, :]) * g.dx[k]
              for k in range(d)]
    # full tensor grid of points, shape (cells..., nq, .., nq) laid out as
    # (n_1, .., n_d, nq_1, .., nq_d)
    shape = g.ncell + (nq,) * d
    X = []
    for k in range(d):
        sh = [1] * (2 * d)
        sh[k] = g.ncell[k]
        sh[d + k] = nq
        X.append(np.broadcast_to(coords[k].reshape(sh), shape))
    cidx = tuple(np.broadcast_to(np.arange(g.ncell[k]).reshape(
        [g.ncell[k] if j == k else 1 for j in range(d)] + [1] * d), shape) for k in range(d))
    Q = conserved(problem, tuple(X), sch.gamma, cidx)     # (nvar, cells..., nq..)
    U = Q
    for k in range(d):
        ax = U.ndim - d + k
        U = np.moveaxis(np.tensordot(U, (Lq * wts[:, None]) / sch.basis.w[None, :],
                                     axes=([ax], [0])), -1, ax)
    # subcell averages: subinterval s holds points s*(N+2) .. (s+1)*(N+2)-1
    A = np.zeros((Ns, nq))
    for s in range(Ns):
        A[s, s * (N + 2):(s + 1) * (N + 2)] = wts[s * (N + 2):(s + 1) * (N + 2)] * Ns
    V = Q
    for k in range(d):
        ax = V.ndim - d + k
        V = np.moveaxis(np.tensordot(V, A, axes=([ax], [1])), -1, ax)
    return U, V


def initial_state(sch, U0, Vexact, detect_ic=True):
    """beta^0 and the stored subcell data from the initial detection."""
    d = sch.dim
    Vs = np.full(Vexact.shape, np.nan)
    beta = np.zeros(sch.grid.ncell, dtype=np.int32)
    U = U0.copy()
    if detect_ic:
        cmin, cmax = det.cell_minmax(Vexact, d)
        m, M = det.neighbourhood_bounds(cmin, cmax, sch.grid)
        beta = det.detect(sch.P(U0), m, M, sch.gamma, d, sch.eps, sch.floor)
        sel = (slice(None),) + (beta == 1,)
        Vs[sel] = Vexact[sel]
        U[sel] = sch.R(Vexact[sel])
    return State(U, beta, Vs)
