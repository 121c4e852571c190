"""GPU parity of the first-order layer after WENO3 (Sec. 6, Fig. algo2).

One step through the C ABI against the oracle's cascade step on data rough
enough that some WENO3 subcell results fail the admissibility test: with
every cell forced onto the subgrid (first-order cells next to WENO3 cells,
which take the first-order flux on the shared face) and with a few rough
cells in a uniform flow (first-order cells next to unlimited DG cells, which
take the first-order fluxes in the flux correction).  Same tolerance as the
other parity tests (1e-12 relative per variable); flags and the number of
recomputed cells are exact.  Then a whole run that loses positivity without
the layer (the 2D Riemann problem RP1) stays admissible with it."""
import numpy as np
import pytest

from oracle.dg import Grid
from oracle.step import Scheme, stable_dt, step
from paper_1406_7416_gb300 import adg, build_lib, inputs

from helpers import (assert_close_rel, beta_from_abi, from_abi, load_state, rough_forced_state,
                     rough_island_state)

pytestmark = pytest.mark.gpu
RTOL = 1e-12
GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _grid(d, n, bc=0):
    return Grid((n,) * d, (0.0,) * d, (1.0 / n,) * d, (bc,) * (2 * d))


def _forced(d, n, N, rough_cells, seed0, mild=False):
    """First seed whose forced step recomputes some cells but at most half."""
    g = _grid(d, n)
    for seed in range(seed0, seed0 + 40):
        sch = Scheme(g, N, GAMMA)
        st = rough_forced_state(sch, np.random.default_rng(seed), rough_cells, mild)
        dt = stable_dt(sch, st, 0.9 / (d * sch.Ns))
        _, info = step(sch, st, dt, force_all=True)
        if 0 < info["fallback"] <= (g.ncell[0] ** d) // 2 or (not mild and info["fallback"] > 0):
            return sch, st, dt
    raise AssertionError("no seed gave a partial first-order layer")


def _island(d, n, N, rough_cells, seed, bc=0):
    sch = Scheme(_grid(d, n, bc), N, GAMMA)
    st = rough_island_state(sch, np.random.default_rng(seed), rough_cells)
    return sch, st, stable_dt(sch, st, 0.9 / (d * sch.Ns))


CASES = {
    "forced2d_N1_4x4": lambda: _forced(2, 4, 1, [(1, 1), (2, 3)], 100) + (True,),
    "forced2d_N3_4x4": lambda: _forced(2, 4, 3, [(1, 2)], 200) + (True,),
    "forced3d_N1_4": lambda: _forced(3, 4, 1, [(1, 1, 1)], 300, mild=True) + (True,),
    "forced2d_N2_6x6_mild": lambda: _forced(2, 6, 2, [(2, 2)], 400, mild=True) + (True,),
    "island2d_N2_8x8": lambda: _island(2, 8, 2, [(3, 3), (4, 4)], 0) + (False,),
    "island2d_N5_6x6_transmissive": lambda: _island(2, 6, 5, [(0, 2), (3, 3)], 1, bc=1) + (False,),
    "island3d_N1_4": lambda: _island(3, 4, 1, [(1, 1, 1), (2, 2, 1)], 0) + (False,),
    "island3d_N2_4_transmissive": lambda: _island(3, 4, 2, [(0, 1, 2)], 2, bc=1) + (False,),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_cascade_step_matches_oracle(name):
    sch, st, dt, force = CASES[name]()
    ref, info = step(sch, st, dt, force_all=force)
    assert info["fallback"] > 0
    g = sch.grid
    s = adg.Solver(sch.dim, g.ncell, g.x0, g.dx, g.bc, sch.N, GAMMA)
    if force:
        s.set_option(adg.OPT_FORCE_LIMITER, 1)
    load_state(s, sch, st)
    s.step(dt)
    d, b, sub = s.read_full()
    assert s.status() == adg.OK
    assert s.fallback_count()[0] == info["fallback"]
    np.testing.assert_array_equal(beta_from_abi(b, g.ncell), ref.beta)
    assert_close_rel(from_abi(d, sch.dim, g.ncell, sch.N + 1), ref.U, RTOL, "DOFs")
    tr = (slice(None),) + (ref.beta == 1,)
    assert_close_rel(from_abi(sub, sch.dim, g.ncell, sch.Ns)[tr], ref.Vs[tr], RTOL, "subcell data")
    s.close()


def test_two_level_scheme_reports_inadmissible_cells():
    sch, st, dt, _ = CASES["forced2d_N1_4x4"]()
    g = sch.grid
    s = adg.Solver(2, g.ncell, g.x0, g.dx, g.bc, sch.N, GAMMA)
    s.set_option(adg.OPT_FORCE_LIMITER, 1)
    s.set_option(adg.OPT_CASCADE, 0)
    load_state(s, sch, st)
    s.step(dt)
    assert s.fallback_count() == (0, 0)
    assert s.status() == adg.WARN_SUBCELL_INADMISSIBLE
    s.close()


@pytest.mark.parametrize("prec", [adg.PREC_FP64, adg.PREC_MIXED_FP32])
@pytest.mark.parametrize("which", ["rp1", "explosion"])
def test_runs_stay_admissible(which, prec):
    """RP1 of Sec. 5.6 at CFL 0.9 of Eq. (cfl): without the layer the subcell
    WENO3 update of the low-pressure quadrant loses positivity after about 30
    steps (the oracle shows the same); with it every step ends admissible.
    The circular explosion runs alongside as a control."""
    w = inputs.riemann_2d(32, 3, 0) if which == "rp1" else inputs.explosion_2d(n=32, N=3)
    s = adg.Solver.from_workload(w, prec)
    s.init_problem(w["problem"])
    for _ in range(80):
        s.step_cfl(w["cfl"])
    assert s.status() == adg.OK
    d, b, sub = s.read_full()
    assert np.isfinite(d).all()
    if which == "rp1":
        assert s.fallback_count()[1] > 0
    s.close()
