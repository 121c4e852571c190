"""GPU: a state whose subcell data leave the admissible set has no CFL time
step.  Eq. (cfl) takes the largest signal speed |v| + c over the subcell data
v^n of every cell (stored data of troubled cells, the projection P(u^n)
elsewhere), and c needs a positive pressure; the oracle's stable_dt refuses
such a state.  adg_max_dt and adg_step_cfl must refuse it too (ADG_ERR_STATE),
also when a single subcell of an unlimited cell has a negative pressure while
its other subcells and its cell mean are admissible.  The controls (the same
states without the dip) give the oracle's time step."""
import numpy as np
import pytest

from paper_1406_7416_gb300 import adg, build_lib, inputs

from helpers import from_abi, oracle_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _uniform_state(w, dip):
    """rho = 1, v = 0, p = 1 at every node (ABI layout, unlimited cells);
    with dip, cell 5's total energy at its first node is set to -3, which
    makes the pressure of the subcells near that node negative."""
    dim, N = w["dim"], w["N"]
    cells, nodes = int(np.prod(w["ncell"])), (N + 1) ** dim
    U = np.zeros((cells, dim + 2, nodes))
    U[:, 0] = 1.0
    U[:, dim + 1] = 1.0 / (w["gamma"] - 1.0)
    if dip:
        U[5, dim + 1, 0] = -3.0
    beta = np.zeros(cells, dtype=np.uint8)
    sub = np.zeros((cells, dim + 2, (2 * N + 1) ** dim))
    return U, beta, sub


def _oracle_dt(w, U, cfl):
    from oracle.step import State, stable_dt
    sch, _, _, _ = oracle_setup(w, detect_ic=False)
    nc = sch.grid.ncell
    Uo = from_abi(U, w["dim"], nc, w["N"] + 1)
    beta = np.zeros(nc, dtype=np.int32)
    Vs = np.full((w["dim"] + 2,) + tuple(nc) + (sch.Ns,) * w["dim"], np.nan)
    return stable_dt(sch, State(Uo, beta, Vs), cfl)


CASES = {
    "2d_N3": lambda: inputs.explosion_2d(n=4, N=3),
    "2d_N5": lambda: inputs.quadrants_vortex_2d(n=4, N=5, steps=None),
    "3d_N2": lambda: inputs.explosion_3d(n=3, N=2),
}


@pytest.mark.parametrize("prec", [adg.PREC_FP64, adg.PREC_MIXED_FP32])
@pytest.mark.parametrize("name", sorted(CASES))
def test_negative_pressure_subcell_has_no_time_step(name, prec):
    w = CASES[name]()
    cfl = w["cfl"]
    U, beta, sub = _uniform_state(w, dip=True)
    # the oracle refuses the state ...
    with pytest.raises(ValueError):
        _oracle_dt(w, U, cfl)
    # ... and so does the library, for a requested step and a CFL step
    s = adg.Solver.from_workload(w, prec)
    s.load_full(U, beta, sub)
    with pytest.raises(adg.AdgError) as e:
        s.max_dt(cfl)
    assert e.value.code == adg.ERR_STATE
    s.close()
    s = adg.Solver.from_workload(w, prec)
    s.load_full(U, beta, sub)
    with pytest.raises(adg.AdgError) as e:
        s.step_cfl(cfl)
        s.status()
    assert e.value.code == adg.ERR_STATE
    s.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_control_state_takes_the_oracle_time_step(name):
    w = CASES[name]()
    U, beta, sub = _uniform_state(w, dip=False)
    s = adg.Solver.from_workload(w, adg.PREC_FP64)
    s.load_full(U, beta, sub)
    dt = s.max_dt(w["cfl"])
    s.close()
    assert dt == pytest.approx(_oracle_dt(w, U, w["cfl"]), rel=1e-13)
