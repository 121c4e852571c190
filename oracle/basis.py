"""Nodal Gauss-Legendre basis on the reference interval [0, 1] (oracle).

Sec. 2.1 Eq. (ansatz.uh): the spatial basis is the tensor product of Lagrange
polynomials through the Gauss-Legendre (GL) points; Sec. 2.2 uses the same
construction in space-time on [0, 1]^{d+1}.  Everything here is one-dimensional;
multi-dimensional operators are applied axis by axis.
"""
import numpy as np


def legendre_and_derivative(n, x):
    """P_n(x) and P_n'(x) on [-1, 1] by the three-term recurrence."""
    p0 = np.ones_like(x)
    p1 = x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    return p1, dp


def gauss_legendre(n):
    """n GL nodes and weights mapped to [0, 1] (weights sum to 1).

    Newton iteration on P_n from the Chebyshev-like first guess
    cos(pi (k + 3/4) / (n + 1/2)); weights w = 2 / ((1 - x^2) P_n'(x)^2) on
    [-1, 1], halved for [0, 1].
    """
    k = np.arange(n, dtype=np.float64)
    x = np.cos(np.pi * (k + 0.75) / (n + 0.5))
    for _ in range(100):
        p, dp = legendre_and_derivative(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-17:
            break
    p, dp = legendre_and_derivative(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    x, w = x[order], w[order]
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes, x):
    """L[j, a] = phi_a(x_j): Lagrange polynomials through `nodes` at points x."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for a in range(n):
        for b in range(n):
            if b != a:
                L[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return L


def lagrange_derivatives(nodes, x):
    """Ld[j, a] = phi_a'(x_j), by the product rule over the factors of phi_a."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    Ld = np.zeros((len(x), n))
    for a in range(n):
        for c in range(n):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(n):
                if b != a and b != c:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            Ld[:, a] += term
    return Ld


class Basis:
    """All 1D operators of the degree-N nodal GL basis (n = N + 1 nodes).

    xi, w   GL nodes / weights on [0, 1]
    D       D[a, b] = phi_b'(xi_a)  (nodal differentiation)
    phi0    phi_a(0), phi1 = phi_a(1)  (boundary extrapolation)
    K1      time stiffness of Eq. (pde.nc.dg2) divided by the spatial mass:
            K1[m, l] = phi_m(1) phi_l(1) - w_l D[l, m]
            (from [theta_k, theta_l]^1 - <d/dtau theta_k, theta_l>, exact under
            GL quadrature for the nodal basis)
    Ktau    K1^{-1} diag(w): the predictor fixed point is
            q = u (x) 1 - Ktau x_tau sum_d (dt/dx_d) D x_d f_d(q)
    """

    def __init__(self, N):
        self.N = N
        self.n = n = N + 1
        self.xi, self.w = gauss_legendre(n)
        self.D = lagrange_derivatives(self.xi, self.xi)
        self.phi0 = lagrange_values(self.xi, 0.0)[0]
        self.phi1 = lagrange_values(self.xi, 1.0)[0]
        self.K1 = np.outer(self.phi1, self.phi1) - (self.w[:, None] * self.D).T
        self.Ktau = np.linalg.solve(self.K1, np.diag(self.w))
