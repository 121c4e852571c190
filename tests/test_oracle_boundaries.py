"""Pins of the oracle's boundary kinds (reflective walls and inflow faces, the
boundaries of the paper's shock-tube, double-Mach and forward-step tests).

  * a closed box of reflecting walls keeps mass and energy to round-off, with
    the limiter active (a wall passes no mass and no energy);
  * the circular explosion centred on a wall equals, to round-off and with
    the same flags, the half of the same explosion on the doubled domain;
  * a uniform stream entering through an inflow face with its own state stays
    uniform;
  * the Sod and Lax shock tubes of Sec. 5.1 (Dirichlet in x, periodic in y)
    approach the exact Riemann solution, with errors falling under
    refinement."""
import numpy as np
import pytest

from oracle import euler
from oracle.dg import INFLOW, PERIODIC, REFLECTIVE, TRANSMISSIVE, Grid
from oracle.ic import initial_state, project_problem
from oracle.step import Scheme, stable_dt, step

import riemann_exact
from helpers import near_threshold_cells

GAMMA = 1.4


def _setup(grid, N, problem, **kw):
    sch = Scheme(grid, N, GAMMA, **kw)
    U0, V0 = project_problem(sch, problem)
    return sch, initial_state(sch, U0, V0)


def _totals(sch, U):
    """Integrals of every conserved variable (GL-weighted DOF sums)."""
    w = sch.basis.w
    Wd = w
    for _ in range(sch.dim - 1):
        Wd = np.multiply.outer(Wd, w)
    cell = np.prod(sch.grid.dx)
    axes = tuple(range(1, U.ndim))
    return (U * Wd).sum(axis=axes) * cell


def _explosion(center, radius=0.3):
    return dict(kind="radial", center=center, radius=radius, inner=(1.0, 0.0, 0.0, 1.0),
                outer=(0.125, 0.0, 0.0, 0.1), cell_rho_factor=None)


def test_closed_box_keeps_mass_and_energy():
    g = Grid((12, 10), (0.0, 0.0), (1.0 / 12, 1.0 / 10), (REFLECTIVE,) * 4)
    sch, st = _setup(g, 2, _explosion((0.31, 0.42)))
    tot0 = _totals(sch, st.U)
    limited = 0
    for _ in range(12):
        st, info = step(sch, st, 0.5 * stable_dt(sch, st, 0.9 / (2 * 5)))
        limited += info["troubled"]
    tot = _totals(sch, st.U)
    assert limited > 0
    for v in (0, 3):                              # mass, energy
        assert abs(tot[v] - tot0[v]) <= 1e-13 * abs(tot0[v]), (v, tot[v], tot0[v])
    assert abs(tot[1] - tot0[1]) > 1e-6          # the walls do push: x momentum changes


# problems symmetric about x = 0: an explosion centred there, and streams that
# collide there (x momentum of opposite signs on the two sides, so the wall's
# mirror images change the bounds of V_i)
SYMMETRIC = {
    "explosion": _explosion((0.0, 0.1), radius=0.45),
    "collision": dict(kind="quadrant", center=(0.0, 0.15), vortex=None,
                      states=[(1.0, -0.6, 0.1, 1.0), (1.0, 0.6, 0.1, 1.0),
                              (0.5, 0.4, -0.2, 0.8), (0.5, -0.4, -0.2, 0.8)]),
}


@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("name", sorted(SYMMETRIC))
def test_wall_equals_mirror_half_of_symmetric_problem(name, force):
    """A problem symmetric about x = 0 on the full domain [-1,1] x [-1,1]
    (transmissive) against the half domain [0,1] x [-1,1] with a reflecting
    wall at x = 0.  The full solution is mirror-symmetric, so its right half
    is the half-domain solution, flags included."""
    N = 2
    full = Grid((16, 12), (-1.0, -1.0), (0.125, 2.0 / 12), (TRANSMISSIVE,) * 4)
    half = Grid((8, 12), (0.0, -1.0), (0.125, 2.0 / 12), (REFLECTIVE, TRANSMISSIVE, TRANSMISSIVE,
                                                          TRANSMISSIVE))
    prob = SYMMETRIC[name]
    sf, stf = _setup(full, N, prob)
    sh, sth = _setup(half, N, prob)
    np.testing.assert_array_equal(stf.beta[8:], sth.beta)
    for _ in range(5):
        dt = 0.5 * stable_dt(sf, stf, 0.9 / (2 * 5))
        stf, inf = step(sf, stf, dt, force_all=force)
        sth, inh = step(sh, sth, dt, force_all=force)
        if not force:
            near = near_threshold_cells(sh, inh)
            assert not np.any((stf.beta[8:] != sth.beta) & ~near)
            np.testing.assert_array_equal(stf.beta[8:], sth.beta)
    scale = np.abs(stf.U).max(axis=(1, 2, 3, 4))[:, None, None, None, None]
    np.testing.assert_allclose(sth.U / scale, stf.U[:, 8:] / scale, rtol=0, atol=1e-12)
    assert inh["troubled"] > 0


def test_inflow_keeps_a_uniform_stream():
    q = euler.prim_to_cons(np.array(1.3), [np.array(0.7), np.array(-0.2)], np.array(0.9), GAMMA)
    g = Grid((8, 6), (0.0, 0.0), (0.125, 1.0 / 6), (INFLOW, TRANSMISSIVE, PERIODIC, PERIODIC),
             states={0: q})
    prob = dict(kind="quadrant", center=(0.0, 0.0), states=[(1.3, 0.7, -0.2, 0.9)] * 4, vortex=None)
    sch, st = _setup(g, 3, prob)
    U0 = st.U.copy()
    for _ in range(4):
        st, info = step(sch, st, stable_dt(sch, st, 0.9 / (2 * 7)))
        assert info["troubled"] == 0
    np.testing.assert_allclose(st.U, U0, rtol=1e-14, atol=1e-14)


SHOCK_TUBES = {"sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.2),
               "lax": ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.14)}


def _shock_tube_error(name, n, N):
    left, right, t_end = SHOCK_TUBES[name]
    L = euler.prim_to_cons(np.array(left[0]), [np.array(left[1]), np.array(0.0)],
                           np.array(left[2]), GAMMA)
    R = euler.prim_to_cons(np.array(right[0]), [np.array(right[1]), np.array(0.0)],
                           np.array(right[2]), GAMMA)
    g = Grid((n, 1), (0.0, -0.5), (1.0 / n, 1.0), (INFLOW, INFLOW, PERIODIC, PERIODIC),
             states={0: L, 1: R})
    lprim = (left[0], left[1], 0.0, left[2])
    rprim = (right[0], right[1], 0.0, right[2])
    prob = dict(kind="quadrant", center=(0.5, 0.0), states=[rprim, lprim, lprim, rprim], vortex=None)
    sch, st = _setup(g, N, prob)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(stable_dt(sch, st, 0.9 / (2 * (2 * N + 1))), t_end - t)
        st, _ = step(sch, st, dt)
        t += dt
    # L1 density error with an (N+3)-point Gauss rule per cell (x only)
    xq, wq = np.polynomial.legendre.leggauss(N + 3)
    xq, wq = 0.5 * (xq + 1.0), 0.5 * wq
    from oracle.basis import lagrange_values
    Lx = lagrange_values(sch.basis.xi, xq)               # (q, n)
    rho = st.U[0][:, 0]                                  # (cells x, nodes x, nodes y)
    rq = np.einsum("qa,cab->cqb", Lx, rho).mean(axis=-1)  # data constant in y
    x = (np.arange(n)[:, None] + xq[None, :]) / n
    ex = riemann_exact.sample(left, right, (x - 0.5) / t)[0]
    return float(np.sum(np.abs(rq - ex) * wq[None, :]) / n)


@pytest.mark.parametrize("name", ["sod", "lax"])
def test_shock_tube_approaches_exact_solution(name):
    e1 = _shock_tube_error(name, 24, 3)
    e2 = _shock_tube_error(name, 48, 3)
    bound = {"sod": 0.012, "lax": 0.04}[name]
    assert e1 < bound, (name, e1)
    assert e2 < 0.75 * e1, (name, e1, e2)


@pytest.mark.parametrize("d", [2, 3])
def test_wall_bounds_equal_mirrored_domain_bounds(d):
    """The V_i bounds at a reflecting wall are those of the doubled domain
    holding the mirror image (normal momentum negated): per-cell extremes on
    the half domain, mirrored across x = 0, give on the full domain exactly
    the half domain's bounds in its right half, for every variable."""
    from oracle import detect as det
    rng = np.random.default_rng(5 + d)
    nh = (4,) + (5,) * (d - 1)
    nv = d + 2
    a = rng.normal(size=(nv,) + nh)
    b = rng.normal(size=(nv,) + nh)
    cmin, cmax = np.minimum(a, b), np.maximum(a, b)
    # the mirror image over x: reversed cells, x momentum negated (min and max swap)
    mmin, mmax = cmin[:, ::-1].copy(), cmax[:, ::-1].copy()
    mmin[1], mmax[1] = -cmax[1, ::-1], -cmin[1, ::-1]
    fmin = np.concatenate([mmin, cmin], axis=1)
    fmax = np.concatenate([mmax, cmax], axis=1)
    bc_half = (REFLECTIVE, TRANSMISSIVE) + (TRANSMISSIVE,) * (2 * d - 2)
    half = Grid(nh, (0.0,) * d, (0.1,) * d, bc_half)
    full = Grid((2 * nh[0],) + nh[1:], (-0.4,) + (0.0,) * (d - 1), (0.1,) * d,
                (TRANSMISSIVE,) * (2 * d))
    mh, Mh = det.neighbourhood_bounds(cmin, cmax, half)
    mf, Mf = det.neighbourhood_bounds(fmin, fmax, full)
    np.testing.assert_array_equal(mh, mf[:, nh[0]:])
    np.testing.assert_array_equal(Mh, Mf[:, nh[0]:])


def test_double_mach_states_satisfy_rankine_hugoniot():
    """Sec. 5.4 prints the post-shock state as (1/gamma)(8.0, 8.25, 0.0, 116.5)
    ahead of (1, 0, 0, 1/gamma).  Read with 1/gamma on density and pressure
    only, the pair satisfies the jump conditions of a shock moving at Mach 10
    (speed 10: the sound speed ahead is 1) to the printed rounding; with the
    velocity scaled as well it does not."""
    from paper_1406_7416_gb300 import inputs
    post, pre = inputs.oblique_shock_states()

    def jumps(post):
        r1, u1, p1 = post[0], post[1], post[3]
        r0, u0, p0 = pre[0], pre[1], pre[3]
        E1 = p1 / (GAMMA - 1) + 0.5 * r1 * u1 * u1
        E0 = p0 / (GAMMA - 1) + 0.5 * r0 * u0 * u0
        s = 10.0
        return np.array([s * (r1 - r0) - (r1 * u1 - r0 * u0),
                         s * (r1 * u1 - r0 * u0) - (r1 * u1 * u1 + p1 - r0 * u0 * u0 - p0),
                         s * (E1 - E0) - (u1 * (E1 + p1) - u0 * (E0 + p0))]) / np.array(
                             [s * r1, s * r1 * u1, s * E1])
    assert np.abs(jumps(post)).max() < 2e-3
    scaled = (post[0], post[1] / GAMMA, 0.0, post[3])
    assert np.abs(jumps(scaled)).max() > 0.1


def test_isolated_oblique_shock_moves_with_its_front():
    """The double-Mach shock alone: both the lower and the upper boundary
    follow the exact moving shock (post-shock state behind it, pre-shock state
    ahead), the left is post-shock inflow, the right outflow.  After 20 steps
    the shock in the middle row stands where the exact solution puts it, to
    within one cell: x_s = (0.1 + 10 t + y sin 30) / cos 30."""
    from paper_1406_7416_gb300 import inputs
    w = inputs.double_mach(nx=48, ny=6, N=2, length=1.2, height=0.25)
    c, s = np.cos(np.radians(30.0)), np.sin(np.radians(30.0))
    post = w["bc_fronts"][3]["before"]
    pre = w["bc_fronts"][3]["after"]
    w["bc_fronts"][2] = dict(axis=0, a=0.1 / c, b=10.0 / c, before=post, after=pre)
    g = Grid(w["ncell"], w["x0"], w["dx"], w["bc"], w["bc_states"], w["bc_fronts"])
    sch, st = _setup(g, 2, w["problem"])
    for _ in range(80):
        st, _ = step(sch, st, stable_dt(sch, st, w["cfl"]))
    wq = sch.basis.w
    rho = (st.U[0] * np.outer(wq, wq)).sum(axis=(2, 3))      # cell averages (nx, ny)
    mid = 0.5 * (w["problem"]["inner"][0] + w["problem"]["outer"][0])
    for j in range(w["ncell"][1]):                             # every row, boundary rows too
        y = (j + 0.5) * w["dx"][1]
        row = rho[:, j]
        i = int(np.nonzero(row < mid)[0][0])                    # first cell ahead of the shock
        x = (i - 1 + 0.5 + (row[i - 1] - mid) / (row[i - 1] - row[i])) * w["dx"][0]
        exact = (0.1 + 10.0 * st.t + y * s) / c
        assert abs(x - exact) < 1.0 * w["dx"][0], (j, x, exact, st.t)
