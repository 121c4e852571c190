"""Pins of the oracle's Euler flux, EOS and Rusanov flux (Sec. 5, Sec. 2.3)."""
import numpy as np
import pytest

from oracle import euler

GAMMA = 1.4


def _state(rng, d):
    rho = rng.uniform(0.2, 2.0)
    vel = rng.uniform(-1.0, 1.0, size=d)
    p = rng.uniform(0.1, 2.0)
    return euler.prim_to_cons(np.array(rho), [np.array(v) for v in vel], np.array(p), GAMMA), rho, vel, p


@pytest.mark.parametrize("d", [2, 3])
def test_flux_jacobian_eigenvalues(d):
    """The eigenvalues of dF_k/dQ are v_k - c, v_k (d times), v_k + c: pins the
    flux, the EOS and the sound speed together by finite differences."""
    rng = np.random.default_rng(7 + d)
    for _ in range(5):
        Q, rho, vel, p = _state(rng, d)
        c = np.sqrt(GAMMA * p / rho)
        for k in range(d):
            J = np.zeros((d + 2, d + 2))
            for j in range(d + 2):
                h = 1e-6 * max(1.0, abs(Q[j]))
                Qp, Qm = Q.copy(), Q.copy()
                Qp[j] += h
                Qm[j] -= h
                J[:, j] = (euler.flux(Qp, GAMMA, k) - euler.flux(Qm, GAMMA, k)) / (2 * h)
            ev = np.sort(np.linalg.eigvals(J).real)
            expect = np.sort([vel[k] - c] + [vel[k]] * d + [vel[k] + c])
            np.testing.assert_allclose(ev, expect, atol=1e-6)
            assert abs(euler.max_signal_speed(Q, GAMMA, k) - (abs(vel[k]) + c)) < 1e-14


def test_flux_of_resting_contact():
    """A resting contact (u = 0, equal p) carries only the pressure in the
    momentum flux."""
    Q = euler.prim_to_cons(np.array(0.3), [np.array(0.0), np.array(0.0)], np.array(0.7), GAMMA)
    np.testing.assert_allclose(euler.flux(Q, GAMMA, 0), [0.0, 0.7, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(euler.flux(Q, GAMMA, 1), [0.0, 0.0, 0.7, 0.0], atol=1e-15)


def test_rotational_invariance():
    """F_y(Q) equals F_x of the state with the velocity components swapped,
    with the momentum components swapped back."""
    rng = np.random.default_rng(3)
    Q, *_ = _state(rng, 2)
    Qs = Q[[0, 2, 1, 3]]
    np.testing.assert_allclose(euler.flux(Q, GAMMA, 1), euler.flux(Qs, GAMMA, 0)[[0, 2, 1, 3]],
                               rtol=1e-15)


def test_rusanov_consistency_and_upwinding():
    rng = np.random.default_rng(5)
    QL, *_ = _state(rng, 2)
    QR, *_ = _state(rng, 2)
    for k in range(2):
        np.testing.assert_allclose(euler.rusanov(QL, QL, GAMMA, k), euler.flux(QL, GAMMA, k),
                                   rtol=1e-15)
        # mirror symmetry: swapping sides and reversing the normal flips the flux
        mirror = np.ones(4)
        mirror[1 + k] = -1.0
        G = euler.rusanov(QL, QR, GAMMA, k)
        Gm = euler.rusanov(QR * mirror, QL * mirror, GAMMA, k)
        np.testing.assert_allclose(G, -(Gm * mirror), rtol=1e-14, atol=1e-14)
