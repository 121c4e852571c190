"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: DOFs and subcell data agree to 1e-12 relative to each variable's
magnitude over the grid; flags are identical except for cells whose detector
margin (min |x - bound| / max(1, |bound|)) is below 1e-10, where two correct
FP64 implementations may disagree -- such cells and their two-cell
neighbourhood are then excluded from the DOF comparison."""
import numpy as np
import pytest

from oracle import detect as odet
from oracle.step import stable_dt, step, subcell_data
from paper_1406_7416_gb300 import adg, build_lib, inputs

from helpers import (advance, assert_close_rel, beta_from_abi, from_abi, load_state,
                     near_threshold_cells, neighbourhood_mask, oracle_setup, to_abi)

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _periodic(w):
    return [w["bc"][2 * k] == 0 for k in range(w["dim"])]


def _compare_step(w, sch, st, dt, solver, force=False):
    """Load the oracle state, take one step on both sides, compare."""
    load_state(solver, sch, st)
    solver.step(dt)
    d, b, s = solver.read_full()
    assert solver.status() == adg.OK
    ref, info = step(sch, st, dt, force_all=force)
    beta_g = beta_from_abi(b, sch.grid.ncell)
    near = near_threshold_cells(sch, info) if not force else np.zeros_like(beta_g, bool)
    mism = beta_g != ref.beta
    assert not np.any(mism & ~near), f"flag mismatch at {np.argwhere(mism & ~near)[:5]}"
    excl = neighbourhood_mask(mism, 2, _periodic(w))
    U = from_abi(d, sch.dim, sch.grid.ncell, sch.N + 1)
    keep = (slice(None),) + (~excl,)
    err = assert_close_rel(U[keep], ref.U[keep], RTOL, "DOFs")
    Vs = from_abi(s, sch.dim, sch.grid.ncell, sch.Ns)
    tr = (ref.beta == 1) & ~excl
    sel = (slice(None),) + (tr,)
    if tr.any():
        assert_close_rel(Vs[sel], ref.Vs[sel], RTOL, "subcell data")
    return ref, info, err


CASES = {
    "explosion2d_N1_9x9": lambda: inputs.explosion_2d(n=9, N=1),
    "explosion2d_N2_10x10": lambda: inputs.explosion_2d(n=10, N=2),
    "explosion2d_N3_12x7": lambda: _ragged(inputs.explosion_2d(n=12, N=3), (12, 7)),
    "quadrants_N4_8x6": lambda: _ragged(inputs.quadrants_2d(n=8, N=4), (8, 6)),
    "quadvortex_N5_7x7": lambda: inputs.quadrants_vortex_2d(n=7, N=5),
    "quadrants_N6_5x6": lambda: _ragged(inputs.quadrants_2d(n=5, N=6), (5, 6)),
    "quadrants_N7_5x5": lambda: inputs.quadrants_2d(n=5, N=7),
    "quadrants_N8_4x4": lambda: inputs.quadrants_2d(n=4, N=8),
    "quadrants_N9_4x5": lambda: _ragged(inputs.quadrants_2d(n=4, N=9), (4, 5)),
    "explosion3d_N1_5": lambda: _no_noise(inputs.explosion_3d(n=5, N=1)),
    "explosion3d_N2_4": lambda: inputs.explosion_3d(n=4, N=2),
    "explosion3d_N3_4x3x5": lambda: _ragged(_no_noise(inputs.explosion_3d(n=4, N=3)), (4, 3, 5)),
}


def _ragged(w, ncell):
    """Same problem on a non-square grid over the same box."""
    L = [w["dx"][k] * w["ncell"][k] for k in range(w["dim"])]
    w["ncell"] = tuple(ncell)
    w["dx"] = tuple(L[k] / ncell[k] for k in range(w["dim"]))
    fac = w["problem"].get("cell_rho_factor")
    if fac is not None:
        w["problem"]["cell_rho_factor"] = np.ones(ncell)
    return w


def _no_noise(w):
    w["problem"]["cell_rho_factor"] = None
    return w


@pytest.mark.parametrize("name", sorted(CASES))
def test_step_parity(name):
    w = CASES[name]()
    sch, st, _, _ = oracle_setup(w)
    st = advance(sch, st, 2, 0.5 * w["cfl"])
    solver = adg.Solver.from_workload(w)
    for _ in range(2):
        dt = stable_dt(sch, st, 0.5 * w["cfl"])
        st, info, _ = _compare_step(w, sch, st, dt, solver)
    solver.close()


@pytest.mark.parametrize("name", ["explosion2d_N2_10x10", "quadvortex_N5_7x7",
                                  "explosion3d_N2_4"])
def test_step_parity_all_limited(name):
    """Every cell on the subgrid (limiter forced): the WENO3 path everywhere."""
    w = CASES[name]()
    sch, st, _, _ = oracle_setup(w)
    st = advance(sch, st, 1, 0.5 * w["cfl"])
    solver = adg.Solver.from_workload(w)
    solver.set_option(adg.OPT_FORCE_LIMITER, 1)
    dt = stable_dt(sch, st, 0.5 * w["cfl"])
    _compare_step(w, sch, st, dt, solver, force=True)
    solver.close()


IC_CASES = dict(CASES)
# even cell counts: the quadrant corner then lies on a cell face, never on a
# quadrature point, where rounding of the point coordinate would pick the side
IC_CASES["quadvortex_N5_8x8"] = lambda: inputs.quadrants_vortex_2d(n=8, N=5)
IC_CASES["quadrants_N9_4x6"] = lambda: _ragged(inputs.quadrants_2d(n=4, N=9), (4, 6))


@pytest.mark.parametrize("name", ["explosion2d_N3_12x7", "quadvortex_N5_8x8", "quadrants_N9_4x6",
                                  "explosion3d_N1_5", "explosion3d_N3_4x3x5"])
def test_initial_projection_and_detection(name):
    """adg_init_problem (device L2 projection + initial detection) against the
    oracle's projection and detection."""
    w = IC_CASES[name]()
    if w["problem"].get("cell_rho_factor") is not None:
        w["problem"]["cell_rho_factor"] = 1.0 + 0.01 * np.random.default_rng(1).uniform(
            -1, 1, size=w["ncell"])
    sch, st, U0, V0 = oracle_setup(w)
    solver = adg.Solver.from_workload(w)
    solver.init_problem(w["problem"])
    d, b, s = solver.read_full()
    np.testing.assert_array_equal(beta_from_abi(b, sch.grid.ncell), st.beta)
    assert_close_rel(from_abi(d, sch.dim, sch.grid.ncell, sch.N + 1), st.U, RTOL, "initial DOFs")
    Vs = from_abi(s, sch.dim, sch.grid.ncell, sch.Ns)
    sel = (slice(None),) + (st.beta == 1,)
    assert_close_rel(Vs[sel], st.Vs[sel], RTOL, "initial subcell data")
    # the wave-speed based time step agrees too
    np.testing.assert_allclose(solver.max_dt(w["cfl"]), stable_dt(sch, st, w["cfl"]), rtol=1e-13)
    solver.close()


def test_load_without_exact_averages_flags_nothing():
    w = CASES["explosion2d_N2_10x10"]()
    sch, st, U0, V0 = oracle_setup(w)
    solver = adg.Solver.from_workload(w)
    solver.load(to_abi(U0, 2))
    assert solver.flags().sum() == 0
    solver.load(to_abi(U0, 2), to_abi(V0, 2))
    np.testing.assert_array_equal(beta_from_abi(solver.flags(), sch.grid.ncell), st.beta)
    solver.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_conservation_and_free_stream(dim):
    """Periodic explosion: totals of all conserved variables constant to
    round-off over 6 limited steps; a constant state stays constant."""
    w = inputs.explosion_2d(n=16, N=3) if dim == 2 else _no_noise(inputs.explosion_3d(n=6, N=2))
    w["bc"] = (0,) * (2 * dim)
    solver = adg.Solver.from_workload(w)
    solver.init_problem(w["problem"])
    n = w["N"] + 1
    xi, wq = np.polynomial.legendre.leggauss(n)
    W = 0.5 * wq
    Wd = W if dim == 1 else (np.outer(W, W).ravel() if dim == 2 else
                             np.einsum("a,b,c->cba", W, W, W).ravel())
    tot0 = np.einsum("cvl,l->v", solver.read(), Wd)
    troubled = 0
    for _ in range(6):
        solver.step_cfl(0.5 * w["cfl"])
        troubled += solver.troubled_count()
    assert solver.status() == adg.OK
    assert troubled > 0
    tot = np.einsum("cvl,l->v", solver.read(), Wd)
    np.testing.assert_allclose(tot, tot0, rtol=0, atol=1e-13 * np.abs(tot0).max() * solver.cells)
    solver.close()
    # free stream
    w["problem"]["inner"] = w["problem"]["outer"]
    solver = adg.Solver.from_workload(w)
    solver.init_problem(w["problem"])
    U0 = solver.read()
    for _ in range(3):
        solver.step(0.01)
    np.testing.assert_allclose(solver.read(), U0, rtol=1e-14, atol=1e-15)
    assert solver.flags().sum() == 0
    solver.close()


@pytest.mark.parametrize("ncell,bc", [((1, 1), (0, 0, 0, 0)), ((1, 1), (1, 1, 1, 1)),
                                      ((1, 6), (0, 0, 1, 1)), ((2, 1), (1, 1, 0, 0))])
def test_degenerate_grids(ncell, bc):
    """A cell that is its own (periodic) neighbour, single-cell strips and
    transmissive single cells, with every cell limited."""
    w = inputs.quadrants_2d(n=4, N=2)
    L = 1.0
    w["ncell"], w["bc"] = ncell, bc
    w["dx"] = (L / ncell[0], L / ncell[1])
    sch, st, _, _ = oracle_setup(w)
    for force in (False, True):
        solver = adg.Solver.from_workload(w)
        if force:
            solver.set_option(adg.OPT_FORCE_LIMITER, 1)
        dt = stable_dt(sch, st, 0.5 * w["cfl"])
        _compare_step(w, sch, st, dt, solver, force=force)
        solver.close()


def test_capacity_overflow_is_reported():
    w = inputs.explosion_2d(n=8, N=2)
    solver = adg.Solver.from_workload(w)
    solver.set_option(adg.OPT_SLOT_CAPACITY, 3)
    solver.set_option(adg.OPT_FORCE_LIMITER, 1)
    with pytest.raises(adg.AdgError) as e:
        solver.init_problem(w["problem"])      # more than 3 cells flagged at t = 0
    assert e.value.code == adg.ERR_CAPACITY
    solver.close()
    solver = adg.Solver.from_workload(w)
    solver.set_option(adg.OPT_SLOT_CAPACITY, 40)
    solver.init_problem(w["problem"])
    solver.set_option(adg.OPT_FORCE_LIMITER, 1)
    solver.step(1e-3)
    with pytest.raises(adg.AdgError) as e:
        solver.status()
    assert e.value.code == adg.ERR_CAPACITY
    solver.close()


def _smooth_rough_state(sch, seed=3):
    """DOFs of a field that varies in every cell (smooth waves plus a density
    jump), nodal values at the GL points, no cell flagged."""
    from oracle import euler
    from oracle.step import State
    g = sch.grid
    n = sch.N + 1
    xi = 0.5 * (np.polynomial.legendre.leggauss(n)[0] + 1.0)
    nx, ny = g.ncell
    X = g.x0[0] + (np.arange(nx)[:, None, None, None] + xi[None, None, :, None]) * g.dx[0]
    Y = g.x0[1] + (np.arange(ny)[None, :, None, None] + xi[None, None, None, :]) * g.dx[1]
    X, Y = np.broadcast_arrays(X, Y)                    # (nx, ny, a, b)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) + 0.3 * (X > 0.1)
    vel = [0.3 * np.cos(2 * np.pi * Y), 0.2 * np.sin(2 * np.pi * X)]
    p = 1.0 + 0.1 * np.cos(2 * np.pi * (X + Y))
    U = euler.prim_to_cons(rho, vel, p, sch.gamma)
    nc = tuple(g.ncell)
    return State(U, np.zeros(nc, dtype=np.int32), np.full((4,) + nc + (sch.Ns,) * 2, np.nan))


def test_step_parity_literal_dmp():
    """The literal Eq. (relax), delta = eps (M - m) with no floor (ADG_OPT_DMP_FLOOR
    = 0), against the oracle run with floor 0, on a field that varies in every
    cell: the same bar as the other parity cases.  Without the floor smooth
    extrema are flagged too, so the step limits many cells."""
    w = inputs.quadrants_2d(n=4, N=3)
    w["ncell"], w["x0"], w["dx"] = (10, 8), (0.0, 0.0), (0.1, 0.125)
    w["bc"] = (0, 0, 0, 0)
    sch, _, _, _ = oracle_setup(w, floor=0.0)
    st = _smooth_rough_state(sch)
    solver = adg.Solver.from_workload(w)
    solver.set_option(adg.OPT_DMP_FLOOR, 0.0)
    flagged = 0
    compared = 0
    for _ in range(2):
        dt = stable_dt(sch, st, 0.5 * w["cfl"])
        ref, info, _ = _compare_step(w, sch, st, dt, solver)
        near = near_threshold_cells(sch, info)
        compared += int((~neighbourhood_mask(near, 2, _periodic(w))).sum())
        flagged += int(ref.beta.sum())
        st = ref
    solver.close()
    assert flagged > 0
    assert compared >= 80                  # most of the 2 x 80 cells were compared
