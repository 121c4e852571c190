"""Compressible Euler equations, ideal gas (oracle).

Sec. 5 (opening equations): conserved Q = (rho, rho v, rho E) with nu = d + 2
components, flux F = (rho v, rho v v + p I, v (rho E + p)) and the perfect-gas
EOS p = (gamma - 1)(rho E - rho |v|^2 / 2).  The Rusanov (local Lax-Friedrichs)
flux is the numerical flux named in Sec. 2.3 after Eq. (pde.nc.gw2).

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
