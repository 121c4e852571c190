"""Pins of the oracle's projection P and reconstruction R (Sec. 4.2)."""
import numpy as np
import pytest

from oracle.basis import Basis
from oracle.subcell import (constrained_reconstruction_matrix, project, projection_matrix,
                            reconstruct, reconstruction_matrix)


@pytest.mark.parametrize("N", range(1, 10))
def test_projection_exact_on_monomials(N):
    """P1 maps nodal values of x^p to its exact subcell averages (closed form)."""
    b = Basis(N)
    Ns = 2 * N + 1
    P1 = projection_matrix(b, Ns)
    np.testing.assert_allclose(P1.sum(axis=1), 1.0, atol=1e-13)
    lo = np.arange(Ns) / Ns
    hi = (np.arange(Ns) + 1) / Ns
    for p in range(N + 1):
        exact = (hi ** (p + 1) - lo ** (p + 1)) / ((p + 1) * (hi - lo))
        np.testing.assert_allclose(P1 @ b.xi ** p, exact, atol=1e-12)


@pytest.mark.parametrize("N", range(1, 10))
@pytest.mark.parametrize("dim", [2, 3])
def test_reconstruction_inverts_projection(N, dim):
    """Eq. (rid): R o P = I on random P_N data."""
    if dim == 3 and N > 6:
        pytest.skip("size")
    b = Basis(N)
    P1 = projection_matrix(b, 2 * N + 1)
    R1 = reconstruction_matrix(P1)
    U = np.random.default_rng(N).uniform(-1, 1, size=(2, 3) + (b.n,) * dim)
    np.testing.assert_allclose(reconstruct(project(U, P1, dim), R1, dim), U, atol=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_tensor_pseudoinverse_equals_constrained_least_squares(N):
    """The literal constrained least squares of Eqs. (subcell.r) and
    (subcell.r.constraint) equals R1 (x) R1 in 2D."""
    b = Basis(N)
    P1 = projection_matrix(b, 2 * N + 1)
    R1 = reconstruction_matrix(P1)
    Rc = constrained_reconstruction_matrix(b, P1, 2)
    np.testing.assert_allclose(Rc, np.kron(R1, R1), atol=1e-12)


@pytest.mark.parametrize("N", [1, 3, 6])
def test_reconstruction_keeps_mean_and_projector(N):
    b = Basis(N)
    Ns = 2 * N + 1
    P1 = projection_matrix(b, Ns)
    R1 = reconstruction_matrix(P1)
    V = np.random.default_rng(11).uniform(-1, 1, size=(1, 4, Ns, Ns))
    U = reconstruct(V, R1, 2)
    mean_u = np.einsum("vcab,a,b->vc", U, b.w, b.w)
    np.testing.assert_allclose(mean_u, V.mean(axis=(2, 3)), atol=1e-13)
    PR = project(U, P1, 2)
    np.testing.assert_allclose(project(reconstruct(PR, R1, 2), P1, 2), PR, atol=1e-12)
    assert np.max(np.abs(PR - V)) > 1e-3          # a projector, not the identity
