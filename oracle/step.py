"""One full ADER-DG + a-posteriori subcell-limiter time step (oracle).

Sec. 4.4, the five acts, plus the neighbour flux correction that follows them:
  1. unlimited ADER-DG candidate u* (dg.predictor, dg.corrector);
  2. scatter v* = P(u*);
  3. detection (PAD + relaxed DMP) against bounds from v^n over V_i, where
     v^n = P(u^n) if beta^n = 0 and the stored A(v^{n-1}) if beta^n = 1
     (Eq. ader.icbc) -> beta^{n+1};
  4. troubled cells (beta^{n+1} = 1) are recomputed from v^n on the subgrid by
     the ADER-WENO3 operator A, with ghost data from V_i built the same way;
  5. gather u^{n+1} = R(v^{n+1}) for troubled cells; v^{n+1} is kept for the
     next step.
With cascade=False each zone is decremented at most once, as in the paper's
experiments.  With cascade=True (default) the extra MOOD layer of Sec. 6
(Fig. algo2) follows act 4: a troubled cell whose WENO3 result fails PAD is
recomputed from v^n by the first-order Rusanov scheme on its subgrid
(godunov.godunov1), and every troubled WENO3 neighbour sharing a face with it
takes that first-order flux on the shared face instead of its own, so each
face carries one flux (its subcells next to the face are corrected by
-+(dt/h)(F_new - F_old) in the order axis 0 low, high, axis 1 low, ...).  The
first-order result is not checked again.  Unlimited cells that
share a face with a troubled cell have their DG face flux on that face
replaced by the sub-face ADER-WENO fluxes (flux correction of Sec. 4.4): with
the sub-face flux constant on each sub-face, the exact integral against the
test function gives, at tangential node b,
    Fsub_b = (1 / W_b) sum_e Fbar_e prod_j P1[e_j, b_j] / N_s^{d-1}
and the correction  -(dt/dx)(phi_a(1)/w_a)(Fsub_b - Gbar_b)  on a high face,
+(dt/dx)(phi_a(0)/w_a)(Fsub_b - Gbar_b) on a low face.  Corrected neighbours
are not detected again.

Subgrid ghost data at a transmissive boundary: the global subcell index is
clamped into the domain (constant extrapolation of the boundary subcell).
"""
import numpy as np

from . import detect as det
from . import dg
from . import euler
from .dg import FRONT as FRONT_KIND
from .dg import INFLOW as INFLOW_KIND
from .dg import REFLECTIVE as REFLECTIVE_KIND
from .basis import Basis
from .godunov import godunov1
from .subcell import projection_matrix, project, reconstruct, reconstruction_matrix
from .weno import ader_weno


class Scheme:
    """Fixed operators of one (grid, N, gamma) configuration."""

    def __init__(self, grid, N, gamma, eps=det.EPS, floor=det.FLOOR, n_iter=None, cascade=True,
                 flux="rusanov"):
        self.grid = grid
        self.N = N
        self.gamma = gamma
        self.basis = Basis(N)
        self.Ns = 2 * N + 1
        self.P1 = projection_matrix(self.basis, self.Ns)
        self.R1 = reconstruction_matrix(self.P1)
        self.eps = eps
        self.floor = floor
        self.n_iter = N + 1 if n_iter is None else n_iter
        self.cascade = cascade
        self.flux = flux                 # numerical flux of DG faces and WENO3 sub-faces

    @property
    def dim(self):
        return self.grid.dim

    def P(self, U):
        return project(U, self.P1, self.dim)

    def R(self, V):
        return reconstruct(V, self.R1, self.dim)


class State:
    """u (nvar, cells..., n^d nodes), beta (cells...), Vs (nvar, cells..., N_s^d)
    holding v^n for cells with beta = 1 (NaN elsewhere)."""

    def __init__(self, U, beta, Vs, t=0.0):
        self.U = U
        self.beta = beta
        self.Vs = Vs
        self.t = t                       # simulated time (time-dependent boundaries)

    def copy(self):
        return State(self.U.copy(), self.beta.copy(), self.Vs.copy(), self.t)


def subcell_data(sch, st):
    """v^n for every cell (Eq. ader.icbc)."""
    Vp = sch.P(st.U)
    sel = (slice(None),) + (st.beta == 1,)
    Vp[sel] = st.Vs[sel]
    return Vp


def stable_dt(sch, st, cfl):
    """Eq. (cfl) evaluated on the subcell data v^n of every cell."""
    return dg.max_dt(subcell_data(sch, st), sch.grid, sch.gamma, cfl)


def global_subgrid(V, dim):
    """(nvar, cells..., Ns...) -> (nvar, n_1*Ns, ..., n_d*Ns)."""
    nv = V.shape[0]
    cells = V.shape[1:1 + dim]
    Ns = V.shape[-1]
    order = [0]
    for k in range(dim):
        order += [1 + k, 1 + dim + k]
    G = np.transpose(V, order)
    return G.reshape((nv,) + tuple(c * Ns for c in cells))


def patch(sch, G, cell, width=3, t=0.0):
    """(nvar, L, .., L) subgrid patch around `cell` (local -width..N_s+width-1,
    L = N_s + 2 width).  Ghost subcells outside the domain: periodic wrap;
    transmissive clamp (constant extrapolation); reflective mirror index
    (-1 - g below, 2 n - 1 - g above) with the wall-normal momentum negated;
    inflow the face's state; front: one of those by the position of the ghost
    subcell's centre along the front's axis (its unmapped global index) at
    time t.  The per-axis transforms apply in axis order."""
    Ns = sch.Ns
    g_ = sch.grid
    d = sch.dim
    L = Ns + 2 * width
    raw = [cell[k] * Ns - width + np.arange(L) for k in range(d)]
    # per axis and element: (mapped index, transform): transform 0 none,
    # 1 mirror, ("in", state) inflow -- decided per element because a front's
    # part depends on the position along another axis
    idx = np.empty((d,) + (L,) * d, dtype=np.int64)
    kinds = np.zeros((d,) + (L,) * d, dtype=np.int64)        # 0 none, 1 mirror, 2 inflow
    states = {}
    grids = np.meshgrid(*raw, indexing="ij")
    for k in range(d):
        nk = g_.ncell[k] * Ns
        gk = grids[k].copy()
        if g_.periodic(k):
            idx[k] = np.mod(gk, nk)
            continue
        out_idx = gk.copy()
        for side, sel in ((-1, gk < 0), (1, gk >= nk)):
            if not sel.any():
                continue
            face = 2 * k + (1 if side > 0 else 0)
            kind = g_.bc[face]
            if kind == FRONT_KIND:
                fr = g_.fronts[face]
                j = fr["axis"]
                pos = g_.x0[j] + (grids[j] + 0.5) * (g_.dx[j] / Ns)
                before = g_.front_before(face, pos, t)
                parts = ((sel & before, fr["before"]), (sel & ~before, fr["after"]))
            else:
                parts = ((sel, (kind, g_.states.get(face))),)
            for psel, (pkind, pstate) in parts:
                if pkind == REFLECTIVE_KIND:
                    out_idx = np.where(psel, (-1 - gk) if side < 0 else (2 * nk - 1 - gk), out_idx)
                    kinds[k][psel] = 1
                elif pkind == INFLOW_KIND:
                    kinds[k][psel] = 2
                    states[(k, side, id(pstate))] = (psel, np.asarray(pstate, dtype=np.float64))
        idx[k] = np.clip(out_idx, 0, nk - 1)
    P = G[(slice(None),) + tuple(idx[k] for k in range(d))].copy()
    for k in range(d):
        mirror = kinds[k] == 1
        P[1 + k][mirror] = -P[1 + k][mirror]
        for (kk, side, _), (psel, q) in states.items():
            if kk != k:
                continue
            for v in range(P.shape[0]):
                P[v][psel] = q[v]
    return P


def neighbour(sch, cell, k, side):
    """Face neighbour of `cell` along axis k (side -1 low, +1 high), or None."""
    c = list(cell)
    c[k] += side
    nk = sch.grid.ncell[k]
    if c[k] < 0 or c[k] >= nk:
        if not sch.grid.periodic(k):
            return None
        c[k] %= nk
    return tuple(c)


def cascade_layer(sch, troubled, fallback, patches, vnew, faces, dt, h):
    """First-order layer after WENO3 (in place on vnew / faces)."""
    d, Ns = sch.dim, sch.Ns
    v1, f1 = godunov1(patches[:, fallback], dt, h, sch.gamma, d)
    for i, t in enumerate(fallback):
        vnew[:, t] = v1[:, i]
        for k in range(d):
            for s in (0, 1):
                faces[k][s][:, t] = f1[k][s][:, i]
    slot = {c: t for t, c in enumerate(troubled)}
    is_fb = set(fallback)
    for t, c in enumerate(troubled):
        if t in is_fb:
            continue
        for k in range(d):
            for side in (-1, 1):
                nb = neighbour(sch, c, k, side)
                tf = slot.get(nb) if nb is not None else None
                if tf is None or tf not in is_fb:
                    continue
                own = 0 if side == -1 else 1          # this cell's face
                new = faces[k][1 - own][:, tf]        # the fallback cell's side of it
                diff = (dt / h[k]) * (new - faces[k][own][:, t])
                layer = [slice(None)] * (1 + d)
                layer[1 + k] = 0 if side == -1 else Ns - 1
                vt = vnew[:, t]
                if side == -1:
                    vt[tuple(layer)] += diff
                else:
                    vt[tuple(layer)] -= diff


def step(sch, st, dt, force_all=False):
    """Advance `st` by dt; returns (new state, info dict)."""
    g, gam, b, d = sch.grid, sch.gamma, sch.basis, sch.dim
    U = st.U
    # act 1: unlimited candidate
    q = dg.predictor(U, [dt / g.dx[k] for k in range(d)], b, dg.euler_flux_fn(gam), sch.n_iter)
    ff = euler.numerical_flux(sch.flux)
    Ustar, Gbar = dg.corrector(U, q, dt, b, g, gam, ff, t0=st.t)
    # act 2 + 3: scatter and detect against bounds from v^n over V_i
    Vn = subcell_data(sch, st)
    cmin, cmax = det.cell_minmax(Vn, d)
    m, M = det.neighbourhood_bounds(cmin, cmax, g)
    vstar = sch.P(Ustar)
    beta = det.detect(vstar, m, M, gam, d, sch.eps, sch.floor)
    if force_all:
        beta[...] = 1
    Unew = Ustar.copy()
    Vs_new = np.full((U.shape[0],) + g.ncell + (sch.Ns,) * d, np.nan)
    troubled = [tuple(int(x) for x in c) for c in np.argwhere(beta == 1)]
    info = {"troubled": len(troubled), "fallback": 0, "beta": beta.copy(), "m": m, "M": M,
            "vstar": vstar, "Ustar": Ustar.copy(), "fixed": 0}
    if not troubled:
        return State(Unew, beta, Vs_new, st.t + dt), info
    # act 4: subcell ADER-WENO3 from v^n
    G = global_subgrid(Vn, d)
    patches = np.stack([patch(sch, G, c, t=st.t) for c in troubled], axis=1)
    h = [g.dx[k] / sch.Ns for k in range(d)]
    walls = np.array([[[g.kind(k, side) == REFLECTIVE_KIND and
                        c[k] == (0 if side < 0 else g.ncell[k] - 1)
                        for side in (-1, 1)] for k in range(d)] for c in troubled])
    vnew, faces = ader_weno(patches, dt, h, gam, d, ff, walls=walls)
    if sch.cascade:
        fallback = [t for t in range(len(troubled)) if not det.admissible(vnew[:, t], gam, d)]
        info["fallback"] = len(fallback)
        if fallback:
            cascade_layer(sch, troubled, fallback, patches, vnew, faces, dt, h)
    # act 5: gather, keep v^{n+1}
    for t, c in enumerate(troubled):
        sel = (slice(None),) + c
        Vs_new[sel] = vnew[:, t]
        Unew[sel] = sch.R(vnew[:, t])
    # flux correction of unlimited face neighbours
    Mt = (sch.P1.T / sch.Ns) / b.w[:, None]            # Mt[b, e] = P1[e, b] / (N_s w_b)
    fixed = 0
    for t, c in enumerate(troubled):
        for k in range(d):
            for side in (-1, 1):
                nb = neighbour(sch, c, k, side)
                if nb is None or beta[nb] == 1:
                    continue
                # faces[k] = (low, high) of the troubled cell; the neighbour on
                # the troubled cell's low side sees it through its own high face
                Fsub = faces[k][0 if side == -1 else 1][:, t]
                for j in range(d - 1):
                    Fsub = dg.along(Mt, Fsub, 1 + j)
                # DG face flux on the same face (faces indexed 0..n_k along axis k)
                fidx = c[k] if side == -1 else c[k] + 1
                gsel = [slice(None)] + list(c)
                gsel[1 + k] = fidx
                Gdg = Gbar[k][tuple(gsel)]                 # (nvar, tangential nodes)
                diff = Fsub - Gdg
                node_axis = 1 + k                           # node axis k in (nvar, nodes...)
                shape = [1] * (1 + d)
                shape[node_axis] = b.n
                diff = np.expand_dims(diff, node_axis)
                cdt = dt / g.dx[k]
                if side == -1:   # neighbour below: its high face
                    corr = -cdt * (b.phi1 / b.w).reshape(shape) * diff
                else:            # neighbour above: its low face
                    corr = cdt * (b.phi0 / b.w).reshape(shape) * diff
                Unew[(slice(None),) + nb] += corr
                fixed += 1
    info["faces"] = faces
    info["fixed"] = fixed
    return State(Unew, beta, Vs_new, st.t + dt), info
