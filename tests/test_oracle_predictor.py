"""Pins of the oracle's space-time predictor (Sec. 2.2 Eq. pde.nc.dg2)."""
import numpy as np
import pytest

from oracle import dg, euler
from oracle.basis import Basis

GAMMA = 1.4


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_linear_advection_exact_translation(N):
    """f = a q with data of total degree N: the translated solution
    u(xi - a dt tau / dx) stays of degree N in time, Picard is nilpotent, and
    q^{N+1} equals it at every space-time node (numpy polyval2d as the judge)."""
    b = Basis(N)
    n = b.n
    rng = np.random.default_rng(N)
    a = (0.7, -1.3)
    dtdx = (0.4, 0.25)
    X, Y = np.meshgrid(b.xi, b.xi, indexing="ij")
    coefs = []
    U = np.zeros((1, 3, n, n))
    for cell in range(3):
        C = rng.uniform(-1, 1, size=(n, n))
        C[np.add.outer(np.arange(n), np.arange(n)) > N] = 0.0     # total degree <= N
        coefs.append(C)
        U[0, cell] = np.polynomial.polynomial.polyval2d(X, Y, C)
    flux_fn = lambda q, k: a[k] * q
    q = dg.predictor(U, dtdx, b, flux_fn, N + 1)
    qmore = dg.predictor(U, dtdx, b, flux_fn, N + 3)
    np.testing.assert_allclose(q, qmore, atol=1e-12)
    for cell in range(3):
        for m, tau in enumerate(b.xi):
            exact = np.polynomial.polynomial.polyval2d(X - a[0] * dtdx[0] * tau,
                                                       Y - a[1] * dtdx[1] * tau, coefs[cell])
            np.testing.assert_allclose(q[0, cell, :, :, m], exact, atol=1e-11)


@pytest.mark.parametrize("N", [2, 4])
def test_fewer_iterations_are_not_exact(N):
    """Dropping one Picard sweep leaves a visible error on linear advection,
    so the iteration count matters (guards against a silently skipped sweep)."""
    b = Basis(N)
    n = b.n
    U = np.random.default_rng(1).uniform(-1, 1, size=(1, 1, n, n))
    flux_fn = lambda q, k: q
    full = dg.predictor(U, (0.5, 0.5), b, flux_fn, N + 1)
    short = dg.predictor(U, (0.5, 0.5), b, flux_fn, N - 1)
    assert np.max(np.abs(full - short)) > 1e-6


@pytest.mark.parametrize("d", [2, 3])
def test_constant_state_is_fixed_point(d):
    b = Basis(3)
    n = b.n
    Q = euler.prim_to_cons(np.array(0.8), [np.array(0.3)] * d, np.array(0.6), GAMMA)
    U = np.broadcast_to(Q.reshape((d + 2,) + (1,) * (1 + d)), (d + 2, 2) + (n,) * d).copy()
    q = dg.predictor(U, (0.1,) * d, b, dg.euler_flux_fn(GAMMA), 4)
    np.testing.assert_allclose(q, np.repeat(U[..., None], n, axis=-1), rtol=1e-14, atol=1e-15)
