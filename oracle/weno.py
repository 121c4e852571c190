"""Third-order one-step ADER-WENO finite volume update on the subgrid (oracle).

Sec. 4.3 Eq. (aderweno) names the operator A and defers its details to the
cited one-step ADER-WENO literature; the paper fixes only: third order, P2
(WENO3) reconstruction, one-step (space-time predictor) time integration,
Cartesian subgrid of N_s^d equal subcells, initial and boundary data from
Eq. (ader.icbc).  Parity unpinned by the paper for this operator: the reading
below is fixed here and pinned by the tests only through mathematics (exact
for quadratics, constant preservation, conservation, third-order convergence).

Reading:
  * patch: the cell's N_s^d subcells plus 3 ghost layers taken from V_i;
  * dimension-by-dimension WENO in conserved variables: a 1D sweep along x
    on every row, then along y on every x-nodal value, then along z; each 1D
    reconstruction returns values at the 3 GL nodes of the subcell;
  * 1D WENO: stencils {s-2..s}, {s-1..s+1}, {s..s+2}; each gives the quadratic
    with the stencil's three subcell averages; oscillation indicator
    sigma = int_0^1 (p')^2 + (p'')^2 dxi on the unit subcell; weights
    w_k ~ lambda_k / (sigma_k + 1e-14)^8 with lambda = (1, 1e5, 1);
  * degree-2 space-time predictor of Eq. (pde.nc.dg2) on every subcell
    (3 GL nodes per axis and in time, 3 Picard sweeps);
  * sub-face flux: Rusanov (or the scheme's other numerical flux, the
    Osher-type flux) at the 3^(d-1) x 3 tangential x time GL points,
    averaged with the GL weights;
  * update v^{n+1} = v^n - sum_d (dt/h_d)(Fbar_{+} - Fbar_{-}), h_d = dx_d / N_s.
"""
import numpy as np

from . import euler
from .basis import Basis, gauss_legendre
from .dg import along, predictor

LAMBDA = (1.0, 1.0e5, 1.0)
WENO_EPS = 1e-14
WENO_R = 8
OFFSETS = (-2, -1, 0)       # first subcell of the left, central and right stencil


def stencil_coefficient_matrices():
    """C[k]: monomial coefficients (1, xi, xi^2) of the quadratic whose averages
    over [o, o+1], o = OFFSETS[k] + (0, 1, 2), are the stencil's data."""
    C = []
    for o0 in OFFSETS:
        A = np.zeros((3, 3))
        for r in range(3):
            o = o0 + r
            for p in range(3):
                A[r, p] = ((o + 1.0) ** (p + 1) - float(o) ** (p + 1)) / (p + 1)
        C.append(np.linalg.inv(A))
    return C


class Weno3:
    def __init__(self):
        self.C = stencil_coefficient_matrices()
        self.xi, self.w = gauss_legendre(3)
        self.E = np.vander(self.xi, 3, increasing=True)      # E[j, p] = xi_j^p

    def smoothness(self, c):
        """sigma = int_0^1 (p')^2 + (p'')^2, exact by 3-point GL (c[..., p])."""
        d1 = c[..., 1, None] + 2.0 * c[..., 2, None] * self.xi
        d2 = 2.0 * c[..., 2, None]
        return ((d1 * d1 + d2 * d2) * self.w).sum(axis=-1)

    def line(self, u, axis):
        """1D WENO along `axis` of length L: returns the nodal values of the
        subcells 2..L-3 of that axis (axis shrinks by 4) in a new last axis."""
        u = np.moveaxis(u, axis, -1)
        L = u.shape[-1]
        s = np.arange(2, L - 2)
        num = 0.0
        den = 0.0
        for k, o0 in enumerate(OFFSETS):
            sten = np.stack([u[..., s + o0 + r] for r in range(3)], axis=-1)   # (..., L-4, 3)
            c = sten @ self.C[k].T                                            # (..., L-4, 3)
            sigma = self.smoothness(c)
            wt = LAMBDA[k] / (sigma + WENO_EPS) ** WENO_R
            num = num + wt[..., None] * (c @ self.E.T)                        # nodal values
            den = den + wt
        out = num / den[..., None]                                            # (..., L-4, 3)
        return np.moveaxis(out, -2, axis)


def ader_weno(patch, dt, h, gamma, dim, face_flux=euler.rusanov, walls=None):
    """One subcell ADER-WENO3 step on a batch of patches.

    patch: (nvar, T, L, .., L) with L = N_s + 6 (local index -3..N_s+2).
    h: subcell widths per axis.  Returns (v_new (nvar, T, N_s, .., N_s),
    faces) where faces[k] = (low, high) sub-face fluxes on the cell's two
    faces normal to axis k, each (nvar, T, N_s, .., N_s) over the d-1
    tangential subcell axes (in axis order).

    walls: optional bool array (T, dim, 2); where walls[t, k, side] is set, the
    cell's low (0) / high (1) face on axis k is a reflecting wall and its
    sub-face fluxes are taken between the interior trace and its mirror image
    (wall-normal momentum negated), like the DG flux at a wall, so that the
    wall passes exactly no mass and no energy."""
    wn = Weno3()
    b3 = Basis(2)
    L = patch.shape[2]
    Ns = L - 6
    # dimension-by-dimension reconstruction over the block -1..N_s
    W = patch
    for k in range(dim):
        W = wn.line(W, 2 + k)
    # W: (nvar, T, Ns+2 (x), .., nodes (alpha, beta, ..))
    q = predictor(W, [dt / h[k] for k in range(dim)], b3,
                  lambda Q, kk: euler.flux(Q, gamma, kk), 3)
    vnew = patch[(slice(None), slice(None)) + (slice(3, 3 + Ns),) * dim].copy()
    faces = []
    for k in range(dim):
        node_axis = q.ndim - 1 - dim + k
        qlo = np.tensordot(q, b3.phi0, axes=([node_axis], [0]))
        qhi = np.tensordot(q, b3.phi1, axes=([node_axis], [0]))
        sl_left = [slice(None), slice(None)] + [slice(1, Ns + 1)] * dim
        sl_right = list(sl_left)
        sl_left[2 + k] = slice(0, Ns + 1)
        sl_right[2 + k] = slice(1, Ns + 2)
        QL, QR = qhi[tuple(sl_left)], qlo[tuple(sl_right)]
        if walls is not None and np.any(walls[:, k]):
            QL, QR = QL.copy(), QR.copy()
            for side, f in ((0, 0), (1, Ns)):
                t = np.nonzero(walls[:, k, side])[0]
                if len(t) == 0:
                    continue
                sel = [slice(None)] * QL.ndim
                sel[1] = t
                sel[2 + k] = f
                sel = tuple(sel)
                if side == 0:                    # ghost on the left of the low wall
                    QL[sel] = QR[sel]
                    QL[(1 + k,) + sel[1:]] = -QR[(1 + k,) + sel[1:]]
                else:                            # ghost on the right of the high wall
                    QR[sel] = QL[sel]
                    QR[(1 + k,) + sel[1:]] = -QL[(1 + k,) + sel[1:]]
        G = face_flux(QL, QR, gamma, k)
        # average over the d-1 tangential nodes and time with GL weights
        for _ in range(dim):
            G = np.tensordot(G, b3.w, axes=([G.ndim - 1], [0]))
        # G: (nvar, T, subcell axes with axis k of length Ns+1)
        hi = np.take(G, np.arange(1, Ns + 1), axis=2 + k)
        lo = np.take(G, np.arange(0, Ns), axis=2 + k)
        vnew = vnew - (dt / h[k]) * (hi - lo)
        faces.append((np.take(G, 0, axis=2 + k), np.take(G, Ns, axis=2 + k)))
    return vnew, faces
