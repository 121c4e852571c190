"""Test helpers for grid-refinement error estimates: GL rules on [0, 1],
Lagrange evaluation, the coarse DG polynomials on the cells of the grid
refined by 2, and per-variable relative L1 distances (ABI layouts)."""
import numpy as np


def gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def weights(dim, n):
    _, W = gl(n)
    Wd = W
    for _ in range(dim - 1):
        Wd = np.outer(W, Wd).ravel()
    return Wd


def lagrange(xi, pts):
    """L[p][q] = phi_q(pts[p]) for the Lagrange basis on the nodes xi."""
    L = np.ones((len(pts), len(xi)))
    for q in range(len(xi)):
        for r in range(len(xi)):
            if r != q:
                L[:, q] *= (pts - xi[r]) / (xi[q] - xi[r])
    return L


def coarse_on_fine(Uc, ncell, N, dim):
    """The coarse DG polynomials (ABI layout [cell][var][node]) evaluated at
    the nodes of the 2^dim children of every cell, in the ABI layout of the
    grid refined by 2."""
    n = N + 1
    xi, _ = gl(n)
    L = [lagrange(xi, 0.5 * (a + xi)) for a in (0, 1)]
    nv = Uc.shape[1]
    if dim == 2:
        nx, ny = ncell
        A = Uc.reshape(ny, nx, nv, n, n)
        out = np.empty((ny, 2, nx, 2, nv, n, n))
        for b in (0, 1):
            for a in (0, 1):
                out[:, b, :, a] = np.einsum("yq,xr,JIvqr->JIvyx", L[b], L[a], A)
        return out.reshape(4 * nx * ny, nv, n * n)
    nx, ny, nz = ncell
    A = Uc.reshape(nz, ny, nx, nv, n, n, n)
    out = np.empty((nz, 2, ny, 2, nx, 2, nv, n, n, n))
    for c in (0, 1):
        for b in (0, 1):
            for a in (0, 1):
                out[:, c, :, b, :, a] = np.einsum("zp,yq,xr,KJIvpqr->KJIvzyx", L[c], L[b], L[a], A)
    return out.reshape(8 * nx * ny * nz, nv, n ** 3)


def rel_l1(A, B, Wd):
    """Per-variable relative L1 distance of A from B (ABI layout)."""
    num = np.einsum("cvl,l->v", np.abs(A - B), Wd)
    den = np.einsum("cvl,l->v", np.abs(B), Wd)
    return num / den
