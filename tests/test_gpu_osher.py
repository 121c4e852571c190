"""GPU parity of the Osher-type flux option (ADG_OPT_FLUX = ADG_FLUX_OSHER):
one step through the C ABI against the oracle with the same flux, on DG faces
(unlimited cells) and on WENO3 sub-faces (limited cells), 2D and 3D.  The
kernel builds |A| from the closed-form characteristic decomposition, the
oracle from Sylvester's formula on the analytic Jacobian.  Same tolerance as
the other parity tests."""
import numpy as np
import pytest

from oracle.step import stable_dt, step
from paper_1406_7416_gb300 import adg, build_lib, inputs

from helpers import assert_close_rel, beta_from_abi, from_abi, load_state, near_threshold_cells, oracle_setup

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _no_noise(w):
    w["problem"]["cell_rho_factor"] = None
    return w


CASES = {
    "explosion2d_N2_10x10": (lambda: inputs.explosion_2d(n=10, N=2), False),
    "quadvortex_N5_7x7": (lambda: inputs.quadrants_vortex_2d(n=7, N=5), False),
    "quadrants_N3_6x6_forced": (lambda: inputs.quadrants_2d(n=6, N=3), True),
    "rp1_N4_8x8": (lambda: inputs.riemann_2d(8, 4, 0), False),
    "explosion3d_N2_4": (lambda: _no_noise(inputs.explosion_3d(n=4, N=2)), False),
    "explosion3d_N1_4_forced": (lambda: _no_noise(inputs.explosion_3d(n=4, N=1)), True),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_osher_step_matches_oracle(name):
    make, force = CASES[name]
    w = make()
    sch, st, _, _ = oracle_setup(w, flux="osher")
    dt = 0.5 * stable_dt(sch, st, w["cfl"])
    s = adg.Solver.from_workload(w)
    s.set_option(adg.OPT_FLUX, adg.FLUX_OSHER)
    if force:
        s.set_option(adg.OPT_FORCE_LIMITER, 1)
    load_state(s, sch, st)
    s.step(dt)
    d, b, sub = s.read_full()
    assert s.status() == adg.OK
    ref, info = step(sch, st, dt, force_all=force)
    beta = beta_from_abi(b, sch.grid.ncell)
    if not force:
        near = near_threshold_cells(sch, info)
        assert not np.any((beta != ref.beta) & ~near)
    np.testing.assert_array_equal(beta, ref.beta)
    assert_close_rel(from_abi(d, sch.dim, sch.grid.ncell, sch.N + 1), ref.U, RTOL, "DOFs")
    tr = (slice(None),) + (ref.beta == 1,)
    if (ref.beta == 1).any():
        assert_close_rel(from_abi(sub, sch.dim, sch.grid.ncell, sch.Ns)[tr], ref.Vs[tr], RTOL,
                         "subcell data")
    s.close()


def test_flux_option_validated():
    w = inputs.explosion_2d(n=4, N=1)
    s = adg.Solver.from_workload(w)
    with pytest.raises(adg.AdgError):
        s.set_option(adg.OPT_FLUX, 2)
    s.close()
