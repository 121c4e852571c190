"""Compressible Euler equations, ideal gas (oracle).

Sec. 5 (opening equations): conserved Q = (rho, rho v, rho E) with nu = d + 2
components, flux F = (rho v, rho v v + p I, v (rho E + p)) and the perfect-gas
EOS p = (gamma - 1)(rho E - rho |v|^2 / 2).  Sec. 2.3 (after Eq. pde.nc.gw2)
names two numerical fluxes: the Rusanov (local Lax-Friedrichs) flux and the
universal Osher-type flux of Dumbser and Toro (the one used for the vortex
table of Sec. 5.2).

All functions take arrays with the variable index first, Q[v, ...].
"""
import numpy as np


def pressure(Q, gamma):
    d = Q.shape[0] - 2
    rho = Q[0]
    kin = sum(Q[1 + k] * Q[1 + k] for k in range(d)) / rho
    return (gamma - 1.0) * (Q[1 + d] - 0.5 * kin)


def flux(Q, gamma, k):
    """Physical flux in direction k (0 = x), same shape as Q."""
    d = Q.shape[0] - 2
    rho = Q[0]
    p = pressure(Q, gamma)
    vk = Q[1 + k] / rho
    F = np.empty_like(Q)
    F[0] = Q[1 + k]
    for j in range(d):
        F[1 + j] = Q[1 + j] * vk
    F[1 + k] = F[1 + k] + p
    F[1 + d] = vk * (Q[1 + d] + p)
    return F


def sound_speed(Q, gamma):
    return np.sqrt(gamma * pressure(Q, gamma) / Q[0])


def max_signal_speed(Q, gamma, k):
    """|v_k| + c, the largest eigenvalue modulus of dF_k/dQ."""
    return np.abs(Q[1 + k] / Q[0]) + sound_speed(Q, gamma)


def rusanov(QL, QR, gamma, k):
    """Rusanov flux through a face with normal +e_k, evaluated pointwise:
    G = (F(QL) + F(QR))/2 - s_max (QR - QL)/2, s_max = max(|v_k| + c) of both
    sides at the same point (pointwise reading of the wave-speed estimate)."""
    s = np.maximum(max_signal_speed(QL, gamma, k), max_signal_speed(QR, gamma, k))
    return 0.5 * (flux(QL, gamma, k) + flux(QR, gamma, k)) - 0.5 * s * (QR - QL)


def jacobian(Q, gamma, k):
    """A_k = dF_k/dQ at the states Q[v, ...]; returns (..., nv, nv) with row =
    flux component, column = conserved variable."""
    d = Q.shape[0] - 2
    nv = d + 2
    rho = Q[0]
    u = [Q[1 + j] / rho for j in range(d)]
    q2 = sum(uj * uj for uj in u)
    p = pressure(Q, gamma)
    H = (Q[1 + d] + p) / rho
    gm1 = gamma - 1.0
    A = np.zeros(Q.shape[1:] + (nv, nv))
    A[..., 0, 1 + k] = 1.0
    for i in range(d):                              # momentum i: m_k m_i / rho + p delta_ik
        A[..., 1 + i, 0] = -u[k] * u[i]
        A[..., 1 + i, 1 + i] += u[k]
        A[..., 1 + i, 1 + k] += u[i]
        if i == k:
            A[..., 1 + i, 0] += 0.5 * gm1 * q2
            for j in range(d):
                A[..., 1 + i, 1 + j] -= gm1 * u[j]
            A[..., 1 + i, 1 + d] += gm1
    A[..., 1 + d, 0] = u[k] * (0.5 * gm1 * q2 - H)  # energy: m_k (E + p) / rho
    for j in range(d):
        A[..., 1 + d, 1 + j] = -gm1 * u[k] * u[j]
    A[..., 1 + d, 1 + k] += H
    A[..., 1 + d, 1 + d] = gamma * u[k]
    return A


def abs_jacobian(Q, gamma, k):
    """|A_k| by Sylvester's formula: A_k is diagonalizable with the three
    distinct eigenvalues mu = v_k - c, v_k, v_k + c, so |A_k| = p(A_k) for the
    quadratic p that interpolates |x| at those three values:
        |A_k| = sum_i |mu_i| prod_{j != i} (A_k - mu_j I) / (mu_i - mu_j)."""
    A = jacobian(Q, gamma, k)
    nv = A.shape[-1]
    vk = Q[1 + k] / Q[0]
    c = sound_speed(Q, gamma)
    mu = [vk - c, vk, vk + c]
    eye = np.eye(nv)
    out = 0.0
    for i in range(3):
        term = np.abs(mu[i])[..., None, None] * np.broadcast_to(eye, A.shape)
        for j in range(3):
            if j != i:
                term = term @ ((A - mu[j][..., None, None] * eye) / (mu[i] - mu[j])[..., None, None])
        out = out + term
    return out


OSHER_POINTS = 3


def osher(QL, QR, gamma, k, points=OSHER_POINTS):
    """Universal Osher-type flux (Dumbser and Toro) through a face with normal
    +e_k, pointwise: G = (F(QL) + F(QR))/2 - (1/2) [sum_j w_j |A_k(psi(s_j))|]
    (QR - QL) along the straight path psi(s) = QL + s (QR - QL), with the
    `points`-point Gauss-Legendre rule on [0, 1] (reading: 3 points)."""
    x, w = np.polynomial.legendre.leggauss(points)
    s, w = 0.5 * (x + 1.0), 0.5 * w
    dQ = QR - QL
    M = 0.0
    for sj, wj in zip(s, w):
        M = M + wj * abs_jacobian(QL + sj * dQ, gamma, k)
    diss = np.einsum("...ij,j...->i...", M, dQ)
    return 0.5 * (flux(QL, gamma, k) + flux(QR, gamma, k)) - 0.5 * diss


def numerical_flux(name):
    """The face flux function (QL, QR, gamma, k) for 'rusanov' or 'osher'."""
    return {"rusanov": rusanov, "osher": osher}[name]


def prim_to_cons(rho, vel, p, gamma):
    """(rho, velocity components list, p) -> Q[v, ...]."""
    d = len(vel)
    Q = np.empty((d + 2,) + np.shape(rho))
    Q[0] = rho
    kin = 0.0
    for j in range(d):
        Q[1 + j] = rho * vel[j]
        kin = kin + vel[j] * vel[j]
    Q[1 + d] = p / (gamma - 1.0) + 0.5 * rho * kin
    return Q
