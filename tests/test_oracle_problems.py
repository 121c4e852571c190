"""Pins of the oracle's initial data (Sec. 5.2, 5.6, 5.8) and IC projection (Sec. 4.4)."""
import numpy as np

from oracle import euler
from oracle.dg import Grid
from oracle.ic import initial_state, project_problem
from oracle.problems import primitive, vortex_perturbation
from oracle.step import Scheme
from paper_1406_7416_gb300 import inputs

GAMMA = 1.4


def test_vortex_is_in_radial_equilibrium():
    """A steady vortex needs dp/dr = rho v_theta^2 / r.  The beta^2 temperature
    perturbation satisfies it; the printed single power of beta does not."""
    w = inputs.vortex_2d(8, 2)
    prob = dict(w["problem"])
    prob["states"] = [(1.0, 0.0, 0.0, 1.0)] * 4            # vortex at rest
    r = np.linspace(0.3, 3.0, 50)
    h = 1e-5
    rho, vel, p = primitive(prob, (r, 0.0 * r), GAMMA)
    _, _, pp = primitive(prob, (r + h, 0.0 * r), GAMMA)
    _, _, pm = primitive(prob, (r - h, 0.0 * r), GAMMA)
    dpdr = (pp - pm) / (2 * h)
    vtheta = vel[1]
    np.testing.assert_allclose(dpdr, rho * vtheta ** 2 / r, rtol=1e-6, atol=1e-9)
    # the alternative (single power of beta) breaks the balance
    beta = 5.0
    T = lambda rr: 1.0 - (GAMMA - 1) * beta / (8 * GAMMA * np.pi ** 2) * np.exp(1 - rr ** 2)
    P = lambda rr: T(rr) ** (GAMMA / (GAMMA - 1))
    alt = (P(r + h) - P(r - h)) / (2 * h)
    assert np.max(np.abs(alt - rho * vtheta ** 2 / r)) > 1e-2
    du, dv, dT = vortex_perturbation(np.array(1.0), np.array(0.0), beta, GAMMA)
    assert abs(du) < 1e-15 and dv > 0 and dT < 0


def test_quadrant_convention():
    st = [(1.0, 0.1, 0.2, 1.1), (2.0, 0.3, 0.4, 2.1), (3.0, 0.5, 0.6, 3.1), (4.0, 0.7, 0.8, 4.1)]
    prob = dict(kind="quadrant", center=(0.0, 0.0), states=st, vortex=None)
    x = np.array([0.5, -0.5, -0.5, 0.5, 0.0, 0.0])
    y = np.array([0.5, 0.5, -0.5, -0.5, 0.0, 0.1])
    rho, vel, p = primitive(prob, (x, y), GAMMA)
    np.testing.assert_array_equal(rho, [1.0, 2.0, 3.0, 4.0, 3.0, 2.0])
    np.testing.assert_array_equal(p, [1.1, 2.1, 3.1, 4.1, 3.1, 2.1])


def test_projection_of_constant_data_is_exact():
    w = inputs.explosion_2d(n=4, N=3)
    w["problem"]["radius"] = 100.0
    g = Grid(w["ncell"], w["x0"], w["dx"], w["bc"])
    sch = Scheme(g, 3, GAMMA)
    U, V = project_problem(sch, w["problem"])
    Q = euler.prim_to_cons(np.array(1.0), [np.array(0.0)] * 2, np.array(1.0), GAMMA)
    np.testing.assert_allclose(U, np.broadcast_to(Q[:, None, None, None, None], U.shape), rtol=1e-14)
    np.testing.assert_allclose(V, np.broadcast_to(Q[:, None, None, None, None], V.shape), rtol=1e-14)
    st = initial_state(sch, U, V)
    assert st.beta.sum() == 0


def test_per_cell_density_factor():
    w = inputs.explosion_3d(n=4, N=1)
    g = Grid(w["ncell"], w["x0"], w["dx"], w["bc"])
    sch = Scheme(g, 1, GAMMA)
    U, V = project_problem(sch, w["problem"])
    fac = w["problem"]["cell_rho_factor"]
    # every cell of this coarse grid lies outside r = 0.4 except the centre ones;
    # the outer cells are constant, scaled by their factor
    i, j, k = 0, 3, 2
    np.testing.assert_allclose(V[0, i, j, k], 0.125 * fac[i, j, k], rtol=1e-14)
