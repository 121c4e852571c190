"""Pins of the oracle's basis (Sec. 2.1 / 2.2) against numpy and calculus."""
import numpy as np
import pytest

from oracle.basis import Basis, gauss_legendre, lagrange_values


@pytest.mark.parametrize("n", range(1, 12))
def test_gauss_legendre_matches_numpy(n):
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (xr + 1.0), rtol=0, atol=6e-16)
    np.testing.assert_allclose(w, 0.5 * wr, rtol=0, atol=6e-16)


@pytest.mark.parametrize("N", range(1, 10))
def test_differentiation_exact_on_monomials(N):
    b = Basis(N)
    for p in range(N + 1):
        vals = b.xi ** p
        der = p * b.xi ** (p - 1) if p > 0 else np.zeros_like(b.xi)
        np.testing.assert_allclose(b.D @ vals, der, atol=1e-11 * (N + 1) ** 2)


@pytest.mark.parametrize("N", range(1, 10))
def test_lagrange_partition_of_unity_and_boundaries(N):
    b = Basis(N)
    np.testing.assert_allclose(lagrange_values(b.xi, b.xi), np.eye(b.n), atol=1e-14)
    np.testing.assert_allclose(b.phi0.sum(), 1.0, atol=1e-13)
    np.testing.assert_allclose(b.phi1.sum(), 1.0, atol=1e-13)
    # phi(0), phi(1) reproduce boundary values of polynomials of degree <= N
    for p in range(N + 1):
        assert abs(b.phi0 @ b.xi ** p - (1.0 if p == 0 else 0.0)) < 1e-12
        assert abs(b.phi1 @ b.xi ** p - 1.0) < 1e-12


@pytest.mark.parametrize("N", range(1, 10))
def test_time_operator_identities(N):
    """K1 1 = phi(0) (so K1^{-1} phi(0) = 1), and Ktau is the exact time
    integral from 0 to tau on polynomials: Ktau tau^p = tau^{p+1}/(p+1)."""
    b = Basis(N)
    np.testing.assert_allclose(b.K1 @ np.ones(b.n), b.phi0, atol=1e-12)
    for p in range(N):
        np.testing.assert_allclose(b.Ktau @ b.xi ** p, b.xi ** (p + 1) / (p + 1),
                                   atol=1e-12 * (N + 1) ** 2)
