"""Subcell projection P and reconstruction R (oracle).

Sec. 4.2 Eq. (subcell.p): v_{i,j} = (1/|S_ij|) int_{S_ij} u_h dx on N_s^d
equidistant subcells; per axis P1[s, a] = N_s int_{s/N_s}^{(s+1)/N_s} phi_a.

Sec. 4.2 Eqs. (subcell.r), (subcell.r.constraint): R solves the (over-
determined, N_s >= N+1) subcell-integral conditions by least squares subject to
conservation of the cell mean.  Because the subcells are equal and the constant
vector lies in the range of P, the normal equations of the unconstrained
problem already enforce the constraint, so R = P^+ = (x)_axes R1 with
R1 = (P1^T P1)^{-1} P1^T.  `constrained_reconstruction_matrix` builds the
literal constrained problem so the tests can confirm the two agree.
"""
import numpy as np

from .basis import gauss_legendre, lagrange_values
from .dg import along


def projection_matrix(basis, Ns):
    """P1[s, a]: exact subcell averages of phi_a (GL rule with n points per
    subinterval integrates the degree-N basis exactly)."""
    xq, wq = gauss_legendre(basis.n)
    P1 = np.zeros((Ns, basis.n))
    for s in range(Ns):
        pts = (s + xq) / Ns
        P1[s] = wq @ lagrange_values(basis.xi, pts)
    return P1


def reconstruction_matrix(P1):
    return np.linalg.solve(P1.T @ P1, P1.T)


def constrained_reconstruction_matrix(basis, P1, dim):
    """Literal constrained least squares of Eq. (subcell.r) + (subcell.r.constraint)
    in dim dimensions, solved through its KKT system; returns the matrix that maps
    the N_s^dim subcell averages to the n^dim nodal DOFs."""
    P = P1
    W = basis.w
    for _ in range(dim - 1):
        P = np.kron(P, P1)
        W = np.kron(W, basis.w)
    m, nd = P.shape
    # mean of u_h over the cell = sum_i W_i u_i;  mean of v = (1/m) sum_j v_j
    KKT = np.zeros((nd + 1, nd + 1))
    KKT[:nd, :nd] = P.T @ P
    KKT[:nd, nd] = W
    KKT[nd, :nd] = W
    rhs = np.zeros((nd + 1, m))
    rhs[:nd] = P.T
    rhs[nd] = 1.0 / m
    return np.linalg.solve(KKT, rhs)[:nd]


def project(U, P1, dim):
    """P(u): the trailing `dim` node axes become subcell axes."""
    V = U
    for k in range(dim):
        V = along(P1, V, V.ndim - dim + k)
    return V


def reconstruct(V, R1, dim):
    """R(v): the trailing `dim` subcell axes become node axes."""
    U = V
    for k in range(dim):
        U = along(R1, U, U.ndim - dim + k)
    return U
