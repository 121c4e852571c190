"""CPU pin of the refinement helper used by the mixed-precision accuracy bar."""
import numpy as np

from refine import coarse_on_fine, gl


def test_coarse_on_fine_is_exact_for_polynomials():
    """The refinement helper: a polynomial of degree N per cell evaluated on
    the children equals its own restriction (here a global polynomial of
    degree N, 2D and 3D)."""
    for dim, N in ((2, 3), (3, 2)):
        n = N + 1
        xi, _ = gl(n)
        nc = (3, 2) if dim == 2 else (2, 2, 3)

        def nodal(ncell, h):
            grids = []
            for k in range(dim):
                c = np.arange(ncell[k])[:, None]
                grids.append(((c + xi[None, :]) * h).ravel())
            X = np.meshgrid(*grids[::-1], indexing="ij")[::-1]     # x fastest
            f = 1.0 + X[0] ** N - 2.0 * X[1] ** (N - 1) * X[0] + (X[2] ** 2 if dim == 3 else 0.0)
            # (.., cells.., nodes..) -> ABI [cell][1][node]
            shp = []
            for k in range(dim)[::-1]:
                shp += [ncell[k], n]
            f = f.reshape(shp)
            order = [2 * k for k in range(dim)] + [2 * k + 1 for k in range(dim)]
            f = np.transpose(f, order).reshape(int(np.prod(ncell)), 1, n ** dim)
            return f

        Uc = nodal(nc, 1.0)
        Uf = nodal(tuple(2 * c for c in nc), 0.5)
        np.testing.assert_allclose(coarse_on_fine(Uc, nc, N, dim), Uf, rtol=1e-12, atol=1e-12)
