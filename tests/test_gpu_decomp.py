"""GPU: one grid stepped as several slab states on one GPU, halos refilled
device to device before every step (adg_pack_cells / adg_unpack_cells), is
bit for bit the undivided grid in FP64: DOFs, flags and stored subcell data
after limited steps, with troubled cells on the slab edges."""
import numpy as np
import pytest

from paper_1406_7416_gb300 import adg, build_lib, inputs
from paper_1406_7416_gb300.decomp import Decomposed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


CASES = {
    # the quadrant corner (x = 0) sits on the slab edge; periodic in x
    "quadvortex_N3_16x12_x2": (lambda: inputs.quadrants_vortex_2d(n=16, N=3, steps=None), 0, 2),
    "quadvortex_N5_12x12_y3": (lambda: inputs.quadrants_vortex_2d(n=12, N=5, steps=None), 1, 3),
    "explosion2d_N2_12_x3": (lambda: inputs.explosion_2d(n=12, N=2), 0, 3),
    "explosion3d_N2_6_z2": (lambda: inputs.explosion_3d(n=6, N=2), 2, 2),
}


def _ragged(w, n):
    L = [w["dx"][k] * w["ncell"][k] for k in range(w["dim"])]
    w["ncell"] = tuple(n)
    w["dx"] = tuple(L[k] / n[k] for k in range(w["dim"]))
    return w


@pytest.mark.parametrize("name", sorted(CASES))
def test_slabs_equal_the_undivided_grid(name):
    make, axis, parts = CASES[name]
    w = make()
    if name.startswith("quadvortex_N3"):
        w = _ragged(w, (16, 12))
    if w["problem"].get("cell_rho_factor") is not None:
        w["problem"]["cell_rho_factor"] = None
    ref = adg.Solver.from_workload(w)
    ref.init_problem(w["problem"])
    start = ref.read_full()
    dec = Decomposed(w, parts, axis=axis)
    dec.load_full(*start)
    cfl = 0.5 * w["cfl"]
    # the time step all-reduce: the minimum of the slabs' steps is the grid's
    assert dec.max_dt(cfl) == ref.max_dt(cfl)
    troubled_on_edges = 0
    for _ in range(6):
        dt = ref.max_dt(cfl)
        ref.step(dt)
        dec.step(dt)
        flags = ref.flags().reshape(tuple(w["ncell"][::-1]))
        edges = [s.own[0] for s in dec.slabs]
        troubled_on_edges += int(np.take(flags, edges, axis=w["dim"] - 1 - axis).sum())
    got = dec.read_full()
    want = ref.read_full()
    assert all(st == adg.OK for st in dec.status()) and ref.status() == adg.OK
    assert troubled_on_edges > 0
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)
    ref.close()
    dec.close()


def test_cfl_steps_through_the_slabs():
    """step_cfl of the slabs (exchange, then the minimum of their CFL steps)
    follows the undivided grid's CFL steps (max_dt, then a step of that dt)."""
    w = inputs.explosion_2d(n=12, N=3)
    ref = adg.Solver.from_workload(w)
    ref.init_problem(w["problem"])
    dec = Decomposed(w, 2, axis=1)
    dec.load_full(*ref.read_full())
    for _ in range(5):
        dt = ref.max_dt(w["cfl"])
        ref.step(dt)
        assert dec.step_cfl(w["cfl"]) == dt
    for a, b in zip(dec.read_full(), ref.read_full()):
        np.testing.assert_array_equal(a, b)
    ref.close()
    dec.close()
