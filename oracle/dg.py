"""ADER-DG predictor and corrector on a Cartesian grid (oracle).

Sec. 2.2 Eq. (pde.nc.dg2): element-local space-time predictor solved by Picard
iteration.  With the nodal GL basis every integral of Eq. (pde.nc.dg2) is exact
under GL quadrature; dividing by the spatial mass W_i leaves, at each spatial
node i and time node m,

    sum_l K1[m, l] q_{i,l} = phi_m(0) u_i - w_m sum_d (dt/dx_d) (D x_d f_d(q))_{i,m}

and since K1 1 = phi(0), q = u (x) 1 - Ktau x_tau sum_d (dt/dx_d) D x_d f_d(q).
Iteration r -> r+1 evaluates the right-hand side at q^r, starting from
q^0 = u (x) 1, for a fixed number of sweeps.

Sec. 2.3 Eq. (pde.nc.gw2): one-step corrector.  With the diagonal GL mass matrix
|T| W_k, the time-averaged nodal flux fbar_i = sum_m w_m f(q_{i,m}) and the
time-averaged face flux Gbar_b = sum_m w_m G(q^-_{b,m}, q^+_{b,m}):

    u*_k = u_k - (dt/dx)(1/w_a)[phi_a(1) Gbar^+_b - phi_a(0) Gbar^-_b
                                - sum_a' w_a' D[a', a] fbar_(a',b)]  - (same in y, z)

where k = (a, b) splits the node index into the normal and tangential parts.

Sec. 2.4 Eq. (cfl): dt = CFL * min_d dx_d / |lambda_max|.  Reading: lambda_max
is taken over the subcell averages v^n of every cell (P(u^n), or the stored
subgrid data of troubled cells); nodal values of a DG polynomial near a shock
can leave the admissible set, the averages that passed the detector do not.
"""
import numpy as np

from . import euler

PERIODIC = 0
TRANSMISSIVE = 1
REFLECTIVE = 2
INFLOW = 3
FRONT = 4


class Grid:
    """Cartesian grid: cells per axis, lower corner, spacing, and boundary kind
    per face (bc[2k] low side, bc[2k+1] high side of axis k); `states` gives the
    conserved state of every INFLOW face (dict face -> vector).

    Boundary kinds (the paper's tests name periodic, transmissive/outflow,
    reflecting-wall and inflow/Dirichlet boundaries without formulas; the
    ghost rules are this oracle's reading):
      PERIODIC      wrap;
      TRANSMISSIVE  the ghost copies the interior (zero-gradient);
      REFLECTIVE    the ghost is the mirror image with the wall-normal momentum
                    negated;
      INFLOW        the ghost is the face's fixed state;
      FRONT         the face is split at a point moving along one tangential
                    axis, x_f(t) = a + b t: points with x < x_f(t) follow one
                    of the kinds above ("before"), the others another
                    ("after") -- the double-Mach boundaries of Sec. 5.4 (the
                    moving shock on the upper boundary; post-shock inflow
                    before the wall on the lower one).  `fronts` gives, per
                    FRONT face, dict(axis, a, b, before=(kind, state or None),
                    after=(kind, state or None))."""

    def __init__(self, ncell, x0, dx, bc, states=None, fronts=None):
        self.dim = len(ncell)
        self.ncell = tuple(int(c) for c in ncell)
        self.x0 = tuple(float(v) for v in x0)
        self.dx = tuple(float(v) for v in dx)
        self.bc = tuple(int(b) for b in bc)
        self.states = {int(f): np.asarray(q, dtype=np.float64) for f, q in (states or {}).items()}
        self.fronts = {int(f): fr for f, fr in (fronts or {}).items()}
        for k in range(self.dim):
            if (self.bc[2 * k] == PERIODIC) != (self.bc[2 * k + 1] == PERIODIC):
                raise ValueError("periodic boundaries must come in pairs")
        for f, b in enumerate(self.bc):
            if b == INFLOW and f not in self.states:
                raise ValueError(f"inflow face {f} needs a state")
            if b == FRONT and f not in self.fronts:
                raise ValueError(f"front face {f} needs its front")

    def periodic(self, k):
        return self.bc[2 * k] == PERIODIC

    def kind(self, k, side):
        """Boundary kind of the low (side -1) or high (side +1) face of axis k."""
        return self.bc[2 * k + (1 if side > 0 else 0)]

    def front_before(self, face, pos, t):
        """True where a point at coordinate `pos` (along the front's axis) lies
        before the front of FRONT face `face` at time t."""
        fr = self.fronts[face]
        return pos < fr["a"] + fr["b"] * t

    def ghost(self, Q, k, side, pos=None, t=0.0):
        """Ghost state beyond the low / high face of axis k for the interior
        state Q[v, ...] next to that face (non-periodic kinds).  For a FRONT
        face, pos (broadcastable to Q[0]) is each point's coordinate along the
        front's axis and t the time."""
        face = 2 * k + (1 if side > 0 else 0)
        kind = self.bc[face]
        if kind == FRONT:
            fr = self.fronts[face]
            before = np.broadcast_to(self.front_before(face, pos, t), Q.shape[1:])
            Gb = _ghost_of_kind(Q, k, *fr["before"])
            Ga = _ghost_of_kind(Q, k, *fr["after"])
            return np.where(before[None], Gb, Ga)
        return _ghost_of_kind(Q, k, kind, self.states.get(face))


def _ghost_of_kind(Q, k, kind, state):
    if kind == REFLECTIVE:
        G = Q.copy()
        G[1 + k] = -G[1 + k]
        return G
    if kind == INFLOW:
        q = np.asarray(state, dtype=np.float64)
        return np.broadcast_to(q.reshape((-1,) + (1,) * (Q.ndim - 1)), Q.shape).copy()
    return Q.copy()


def along(M, X, axis):
    """Apply matrix M along one axis: Y[.., a, ..] = sum_b M[a, b] X[.., b, ..]."""
    return np.moveaxis(np.tensordot(M, X, axes=([1], [axis])), 0, axis)


def euler_flux_fn(gamma):
    return lambda Q, k: euler.flux(Q, gamma, k)


def predictor(U, dt_over_dx, basis, flux_fn, n_iter):
    """Space-time predictor q (Eq. pde.nc.dg2) by n_iter Picard sweeps.

    U: (nvar, batch..., n, .., n) spatial nodal values, d trailing node axes.
    Returns q: U's shape plus a trailing time-node axis."""
    d = len(dt_over_dx)
    n = basis.n
    q = np.repeat(U[..., None], n, axis=-1)
    for _ in range(n_iter):
        S = np.zeros_like(q)
        for k in range(d):
            axis = q.ndim - 1 - d + k
            S = S + dt_over_dx[k] * along(basis.D, flux_fn(q, k), axis)
        q = U[..., None] - along(basis.Ktau, S, q.ndim - 1)
    return q


def _face_points(grid, k, face, xi, t0, dt, shape):
    """Coordinate along the front axis of FRONT face `face` of every node of a
    boundary trace of axis k (shape (cells..., tangential nodes..., time
    nodes)), and the node times t0 + tau_m dt."""
    d = grid.dim
    j = grid.fronts[face]["axis"]
    node_ax = d + (j if j < k else j - 1)          # node axis of axis j in the trace
    sh_c = [1] * len(shape)
    sh_c[j] = grid.ncell[j]
    sh_n = [1] * len(shape)
    sh_n[node_ax] = len(xi)
    pos = grid.x0[j] + (np.arange(grid.ncell[j]).reshape(sh_c) + xi.reshape(sh_n)) * grid.dx[j]
    sh_t = [1] * len(shape)
    sh_t[-1] = len(xi)
    t = t0 + xi.reshape(sh_t) * dt
    return pos, t


def _face_states(qlo, qhi, cell_axis, grid, k, xi=None, t0=0.0, dt=0.0):
    """Left/right states on the n_k + 1 faces of axis k.

    qlo / qhi: traces at the low / high face of every cell.  Face f lies
    between cells f-1 and f.  Periodic: wrap.  Otherwise the missing side is
    the boundary's ghost of the interior trace at the same node (transmissive:
    a copy, so the flux there is F(q^-); reflective: normal momentum negated;
    inflow: the face's state; front: either, by the node's position and time
    t0 + tau dt)."""
    nk = qlo.shape[cell_axis]
    take = lambda a, i: np.take(a, [i], axis=cell_axis)
    if grid.periodic(k):
        left0, rightN = take(qhi, nk - 1), take(qlo, 0)
    else:
        ends = []
        for side, tr in ((-1, take(qlo, 0)), (1, take(qhi, nk - 1))):
            face = 2 * k + (1 if side > 0 else 0)
            if grid.bc[face] == FRONT:
                pos, t = _face_points(grid, k, face, xi, t0, dt, tr.shape[1:])
                ends.append(grid.ghost(tr, k, side, pos, t))
            else:
                ends.append(grid.ghost(tr, k, side))
        left0, rightN = ends
    left = np.concatenate([left0, qhi], axis=cell_axis)
    right = np.concatenate([qlo, rightN], axis=cell_axis)
    return left, right


def corrector(U, q, dt, basis, grid, gamma, face_flux=euler.rusanov, t0=0.0):
    """Candidate u* of Eq. (pde.nc.gw2) and the DG face fluxes.

    Returns (Ustar, Gbar) where Gbar[k] has shape
    (nvar, cells with axis k extended to n_k + 1 faces, tangential nodes...):
    the time-averaged numerical flux (Rusanov unless `face_flux` says
    otherwise) at each tangential GL node of each face."""
    d = grid.dim
    w, D = basis.w, basis.D
    Ustar = U.copy()
    Gbar = []
    Mvol = (D.T * w[None, :]) / w[:, None]      # Mvol[a, a'] = w_a' D[a', a] / w_a
    for k in range(d):
        c = dt / grid.dx[k]
        node_axis = U.ndim - d + k              # spatial node axis of direction k in U
        qnode_axis = q.ndim - 1 - d + k         # same axis in q
        # volume term
        fbar = np.tensordot(euler.flux(q, gamma, k), w, axes=([q.ndim - 1], [0]))
        Ustar = Ustar + c * along(Mvol, fbar, node_axis)
        # face term
        qlo = np.tensordot(q, basis.phi0, axes=([qnode_axis], [0]))
        qhi = np.tensordot(q, basis.phi1, axes=([qnode_axis], [0]))
        left, right = _face_states(qlo, qhi, 1 + k, grid, k, basis.xi, t0, dt)
        G = face_flux(left, right, gamma, k)
        Gb = np.tensordot(G, w, axes=([G.ndim - 1], [0]))
        Gbar.append(Gb)
        nk = grid.ncell[k]
        Ghi = np.expand_dims(np.take(Gb, np.arange(1, nk + 1), axis=1 + k), node_axis)
        Glo = np.expand_dims(np.take(Gb, np.arange(0, nk), axis=1 + k), node_axis)
        shape = [1] * U.ndim
        shape[node_axis] = basis.n
        Ustar = Ustar - c * ((basis.phi1 / w).reshape(shape) * Ghi
                             - (basis.phi0 / w).reshape(shape) * Glo)
    return Ustar, Gbar


def max_dt(Q, grid, gamma, cfl):
    """Eq. (cfl) with lambda_max = max over the states Q[v, ...] of
    max_k |v_k| + c; `cfl` already contains the factor 1/(d (2N+1))."""
    lam = max(float(np.max(euler.max_signal_speed(Q, gamma, k))) for k in range(grid.dim))
    if not np.isfinite(lam) or lam <= 0.0:
        raise ValueError("no admissible wave speed")
    return cfl * min(grid.dx) / lam
