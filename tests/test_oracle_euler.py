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


def _fd_jacobian(Q, k):
    d = Q.shape[0] - 2
    J = np.zeros((d + 2, d + 2))
    for j in range(d + 2):
        h = 1e-6 * max(1.0, abs(Q[j]))
        Qp, Qm = Q.copy(), Q.copy()
        Qp[j] += h
        Qm[j] -= h
        J[:, j] = (euler.flux(Qp, GAMMA, k) - euler.flux(Qm, GAMMA, k)) / (2 * h)
    return J


@pytest.mark.parametrize("d", [2, 3])
def test_analytic_jacobian_matches_finite_differences(d):
    rng = np.random.default_rng(21 + d)
    for _ in range(4):
        Q, *_ = _state(rng, d)
        for k in range(d):
            np.testing.assert_allclose(euler.jacobian(Q, GAMMA, k), _fd_jacobian(Q, k),
                                       rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("d", [2, 3])
def test_abs_jacobian_spectrum(d):
    """|A| commutes with A, squares to A^2 and has trace sum |lambda| over the
    eigenvalues v_k - c, v_k (d times), v_k + c; for a supersonic state |A| = A."""
    rng = np.random.default_rng(31 + d)
    for _ in range(4):
        Q, rho, vel, p = _state(rng, d)
        c = np.sqrt(GAMMA * p / rho)
        for k in range(d):
            A = euler.jacobian(Q, GAMMA, k)
            M = euler.abs_jacobian(Q, GAMMA, k)
            sc = np.abs(A).max()
            np.testing.assert_allclose(M @ A, A @ M, atol=1e-12 * sc * sc)
            np.testing.assert_allclose(M @ M, A @ A, atol=1e-12 * sc * sc)
            lam = [vel[k] - c] + [vel[k]] * d + [vel[k] + c]
            assert abs(np.trace(M) - np.abs(lam).sum()) < 1e-12 * sc
    Q = euler.prim_to_cons(np.array(1.0), [np.array(3.0)] + [np.array(0.2)] * (d - 1),
                           np.array(1.0), GAMMA)
    np.testing.assert_allclose(euler.abs_jacobian(Q, GAMMA, 0), euler.jacobian(Q, GAMMA, 0),
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_osher_flux(d):
    """Consistency F(Q, Q) = F(Q); mirror symmetry; the straight-path integral
    of A dQ reproduces F(QR) - F(QL) when the rule is refined (so the path and
    the Jacobian are right); and for a supersonic pair the flux is the upwind
    flux F(QL) up to the quadrature error of the path integral."""
    rng = np.random.default_rng(41 + d)
    nv = d + 2
    for _ in range(3):
        QL, *_ = _state(rng, d)
        QR, *_ = _state(rng, d)
        for k in range(d):
            np.testing.assert_allclose(euler.osher(QL, QL, GAMMA, k), euler.flux(QL, GAMMA, k),
                                       rtol=1e-13, atol=1e-14)
            mirror = np.ones(nv)
            mirror[1 + k] = -1.0
            G = euler.osher(QL, QR, GAMMA, k)
            Gm = euler.osher(QR * mirror, QL * mirror, GAMMA, k)
            np.testing.assert_allclose(G, -(Gm * mirror), rtol=1e-12, atol=1e-13)
            x, w = np.polynomial.legendre.leggauss(24)
            dQ = QR - QL
            integral = sum(0.5 * wj * euler.jacobian(QL + 0.5 * (xj + 1.0) * dQ, GAMMA, k) @ dQ
                           for xj, wj in zip(x, w))
            np.testing.assert_allclose(integral, euler.flux(QR, GAMMA, k) - euler.flux(QL, GAMMA, k),
                                       rtol=1e-11, atol=1e-12)
    # supersonic along +x on both sides and on the whole path
    rho = [0.8, 1.3]
    QL = euler.prim_to_cons(np.array(rho[0]), [np.array(4.0)] + [np.array(0.3)] * (d - 1),
                            np.array(0.9), GAMMA)
    QR = euler.prim_to_cons(np.array(rho[1]), [np.array(4.5)] + [np.array(-0.2)] * (d - 1),
                            np.array(1.1), GAMMA)
    np.testing.assert_allclose(euler.osher(QL, QR, GAMMA, 0, points=24), euler.flux(QL, GAMMA, 0),
                               rtol=1e-10, atol=1e-10)
    G3 = euler.osher(QL, QR, GAMMA, 0)
    assert np.max(np.abs(G3 - euler.flux(QL, GAMMA, 0))) < 1e-3 * np.abs(euler.flux(QL, GAMMA, 0)).max()
