"""Pins of the oracle's detector (Sec. 4.3) against brute force from the definitions."""
import itertools

import numpy as np
import pytest

from oracle import detect as det
from oracle.dg import Grid

GAMMA = 1.4


def brute_force_flags(vstar, vn, ncell, periodic, eps, floor):
    """Loop-by-loop PAD + relaxed DMP straight from Eqs. (positivity), (dmp), (relax)."""
    d = len(ncell)
    nv = vstar.shape[0]
    flags = np.zeros(ncell, dtype=int)
    for cell in itertools.product(*[range(n) for n in ncell]):
        lo = [np.inf] * nv
        hi = [-np.inf] * nv
        for off in itertools.product((-1, 0, 1), repeat=d):
            nb = []
            ok = True
            for k in range(d):
                c = cell[k] + off[k]
                if c < 0 or c >= ncell[k]:
                    if periodic:
                        c %= ncell[k]
                    else:
                        ok = False
                nb.append(c)
            if not ok:
                continue
            for v in range(nv):
                vals = vn[(v,) + tuple(nb)].ravel()
                lo[v] = min(lo[v], vals.min())
                hi[v] = max(hi[v], vals.max())
        bad = False
        cand = vstar[(slice(None),) + cell].reshape(nv, -1)
        for j in range(cand.shape[1]):
            Q = cand[:, j]
            rho = Q[0]
            kin = sum(Q[1 + k] ** 2 for k in range(d)) / rho
            p = (GAMMA - 1) * (Q[-1] - 0.5 * kin)
            if not (rho > 0 and p > 0):
                bad = True
            for v in range(nv):
                delta = max(eps * (hi[v] - lo[v]), floor * max(1.0, abs(hi[v]), abs(lo[v])))
                if not (lo[v] - delta <= Q[v] <= hi[v] + delta):
                    bad = True
        flags[cell] = int(bad)
    return flags


def _random_subcell_data(rng, ncell, Ns, d):
    nv = d + 2
    shape = (ncell) + (Ns,) * d
    rho = rng.uniform(0.5, 1.5, size=shape)
    vel = [rng.uniform(-0.5, 0.5, size=shape) for _ in range(d)]
    p = rng.uniform(0.5, 1.5, size=shape)
    Q = np.empty((nv,) + shape)
    Q[0] = rho
    for k in range(d):
        Q[1 + k] = rho * vel[k]
    Q[-1] = p / (GAMMA - 1) + 0.5 * rho * sum(v * v for v in vel)
    return Q


@pytest.mark.parametrize("ncell", [(1, 1), (2, 2), (3, 3), (3, 2), (3, 3, 3), (2, 1, 3)])
@pytest.mark.parametrize("periodic", [True, False])
def test_flags_equal_brute_force(ncell, periodic):
    d = len(ncell)
    Ns = 3
    rng = np.random.default_rng(sum(ncell) + 10 * periodic)
    vn = _random_subcell_data(rng, ncell, Ns, d)
    # candidate: old data plus perturbations of varied size, some negative density
    vstar = vn * (1.0 + rng.normal(0, 0.05, size=vn.shape))
    vstar[0].flat[rng.integers(0, vstar[0].size)] *= -1.0
    g = Grid(ncell, (0.0,) * d, (1.0,) * d, (0 if periodic else 1,) * (2 * d))
    for eps, floor in [(1e-3, 1e-12), (0.3, 0.0), (1.0, 0.0)]:
        cmin, cmax = det.cell_minmax(vn, d)
        m, M = det.neighbourhood_bounds(cmin, cmax, g)
        got = det.detect(vstar, m, M, GAMMA, d, eps, floor)
        ref = brute_force_flags(vstar, vn, ncell, periodic, eps, floor)
        np.testing.assert_array_equal(got, ref)


def test_constant_state_needs_the_roundoff_floor():
    """A constant state plus round-off-size noise passes with the floor and
    fails with the literal delta = eps (M - m) = 0."""
    d, Ns = 2, 5
    vn = np.ones((4, 3, 3, Ns, Ns)) * np.array([1.0, 0.1, 0.2, 2.5])[:, None, None, None, None]
    vstar = vn * (1.0 + 1e-15 * np.random.default_rng(2).standard_normal(vn.shape))
    g = Grid((3, 3), (0, 0), (1, 1), (0, 0, 0, 0))
    m, M = det.neighbourhood_bounds(*det.cell_minmax(vn, d), g)
    assert det.detect(vstar, m, M, GAMMA, d).sum() == 0
    assert det.detect(vstar, m, M, GAMMA, d, floor=0.0).sum() > 0


def test_nan_candidate_is_flagged():
    d, Ns = 2, 3
    vn = np.ones((4, 2, 2, Ns, Ns))
    vn[3] = 3.0
    vstar = vn.copy()
    vstar[2, 1, 0, 1, 1] = np.nan
    g = Grid((2, 2), (0, 0), (1, 1), (1, 1, 1, 1))
    m, M = det.neighbourhood_bounds(*det.cell_minmax(vn, d), g)
    np.testing.assert_array_equal(det.detect(vstar, m, M, GAMMA, d), [[0, 0], [1, 0]])
