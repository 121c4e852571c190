"""GPU: the two forms of the FP32 subcell predictor (Sec. 4.3, degree 2 in
space and time on every subcell, three Picard sweeps) give the same results
bit for bit.

The register form holds one subcell per warp with its 27 spatial nodes one
per lane (2D: the 27 space-time nodes one per lane; 3D: each lane also holds
its node's three time nodes) and exchanges line operands by warp shuffles;
the shared-memory form keeps the subcell's nodes in shared memory.  With the
Rusanov sub-face flux the register form writes the subcells' face traces and
the fluxes are taken per sub-face from them; the shared-memory form stores
nodal values and the flux kernel forms the traces.  Both take every output
through the same operation sequence.  Every cell is forced through the
limiter in one run of each case, so every subcell of the grid runs the
predictor."""
import numpy as np
import pytest

from paper_1406_7416_gb300 import adg, build_lib, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _run(w, registers, steps, force):
    s = adg.Solver.from_workload(w, adg.PREC_MIXED_FP32)
    s.set_option(adg.OPT_SUBCELL_REGISTERS, registers)
    s.set_option(adg.OPT_FORCE_LIMITER, force)
    s.init_problem(w["problem"])
    for _ in range(steps):
        s.step_cfl(0.5 * w["cfl"])
    out = s.read_full()
    troubled = s.troubled_count()
    assert s.status() == adg.OK
    s.close()
    return out, troubled


CASES = {
    "explosion2d_N3_10": lambda: inputs.explosion_2d(n=10, N=3),
    "quadvortex_N5_8": lambda: inputs.quadrants_vortex_2d(n=8, N=5, steps=None),
    "explosion3d_N1_5": lambda: inputs.explosion_3d(n=5, N=1),
    "explosion3d_N2_5": lambda: inputs.explosion_3d(n=5, N=2),
    "explosion3d_N3_6": lambda: inputs.explosion_3d(n=6, N=3),
    # reflecting walls on every face (the sub-face fluxes' wall rule)
    "closed_box2d_N3_8": lambda: inputs.closed_box(n=8, N=3, dim=2),
    "closed_box3d_N2_4": lambda: inputs.closed_box(n=4, N=2, dim=3),
    "double_mach_N5": lambda: inputs.double_mach(nx=14, ny=4, N=5),
}


@pytest.mark.parametrize("force", [1, 0])
@pytest.mark.parametrize("name", sorted(CASES))
def test_register_and_shared_forms_are_bitwise_equal(name, force):
    w = CASES[name]()
    ref, troubled = _run(w, 0, 3, force)
    got, _ = _run(w, 1, 3, force)
    assert troubled > 0
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
