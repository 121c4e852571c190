"""Pins of the oracle's first-order subgrid layer (Sec. 6, Fig. algo2) and of
the cascade that applies it after the subcell ADER-WENO3 update.

The paper prints no formulas for this layer, so the pins are mathematical:
constant and contact preservation, conservation of the patch update, the
positivity that a first-order Rusanov step keeps under the CFL condition
(with a control that the same data do lose positivity at three times that
step), first-order convergence on the smooth vortex, and conservation and
locality of a whole cascade step on rough periodic data."""
import numpy as np
import pytest

from oracle import detect as det
from oracle import euler
from oracle.dg import Grid
from oracle.godunov import godunov1
from oracle.ic import project_problem
from oracle.step import Scheme, State, global_subgrid, stable_dt, step
from oracle.weno import ader_weno
from paper_1406_7416_gb300 import inputs

from helpers import rough_forced_state

GAMMA = 1.4


def _rough(shape, d, rng, mach=3.0):
    """Admissible conserved states with strong contrasts: rho, p log-uniform
    over two to three decades, velocities up to `mach` (nvar first)."""
    rho = np.exp(rng.uniform(np.log(0.02), np.log(5.0), size=shape))
    p = np.exp(rng.uniform(np.log(0.005), np.log(5.0), size=shape))
    vel = [rng.uniform(-mach, mach, size=shape) for _ in range(d)]
    return euler.prim_to_cons(rho, vel, p, GAMMA)


def _cfl_dt(patch, h, d, target):
    """dt with sum_d alpha_d dt / h_d = target, alpha_d = max(|u_d| + c)."""
    rate = sum(euler.max_signal_speed(patch, GAMMA, k).max() / h[k] for k in range(d))
    return target / rate


@pytest.mark.parametrize("d", [2, 3])
def test_constant_state_preserved(d):
    Q = euler.prim_to_cons(np.array(0.7), [np.array(-0.3)] * d, np.array(1.3), GAMMA)
    Ns = 3
    patch = np.broadcast_to(Q.reshape((d + 2,) + (1,) * (1 + d)), (d + 2, 2) + (Ns + 6,) * d)
    vnew, faces = godunov1(patch.copy(), 0.01, [0.1] * d, GAMMA, d)
    np.testing.assert_allclose(vnew, patch[(slice(None), slice(None)) + (slice(3, 3 + Ns),) * d],
                               rtol=1e-15, atol=1e-15)
    for k in range(d):
        np.testing.assert_allclose(faces[k][0], faces[k][1], rtol=1e-15)


def test_contact_preserved():
    """Uniform velocity and pressure with any density: the Euler equations
    only advect rho, and the first-order step leaves u, v and p unchanged."""
    d, Ns = 2, 5
    rng = np.random.default_rng(3)
    L = Ns + 6
    rho = rng.uniform(0.1, 3.0, size=(2, L, L))
    u = np.full_like(rho, 0.8)
    v = np.full_like(rho, -0.4)
    p = np.full_like(rho, 0.6)
    patch = euler.prim_to_cons(rho, [u, v], p, GAMMA)
    h = [0.05, 0.05]
    vnew, _ = godunov1(patch, _cfl_dt(patch, h, d, 0.9), h, GAMMA, d)
    np.testing.assert_allclose(vnew[1] / vnew[0], 0.8, rtol=1e-13)
    np.testing.assert_allclose(vnew[2] / vnew[0], -0.4, rtol=1e-13)
    np.testing.assert_allclose(euler.pressure(vnew, GAMMA), 0.6, rtol=1e-12)


def test_conservation_on_the_patch():
    d, Ns = 3, 3
    rng = np.random.default_rng(5)
    patch = _rough((2,) + (Ns + 6,) * d, d, rng)
    h = [0.02, 0.03, 0.025]
    dt = _cfl_dt(patch, h, d, 0.9)
    vnew, faces = godunov1(patch, dt, h, GAMMA, d)
    vold = patch[(slice(None), slice(None)) + (slice(3, 3 + Ns),) * d]
    cell = np.prod(h)
    change = (vnew - vold).sum(axis=(2, 3, 4)) * cell
    boundary = sum(-dt * (cell / h[k]) * (faces[k][1].sum(axis=(2, 3)) - faces[k][0].sum(axis=(2, 3)))
                   for k in range(d))
    np.testing.assert_allclose(change, boundary, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_positivity_under_the_cfl_condition(d):
    """Rough data at sum_d alpha dt/h_d = 0.95: every updated subcell keeps
    rho > 0 and p > 0; at 3x that time step the same data do not, which shows
    the data are rough enough for the check to bite."""
    rng = np.random.default_rng(11 + d)
    Ns = 5 if d == 2 else 3
    patch = _rough((64,) + (Ns + 6,) * d, d, rng, mach=4.0)
    h = [0.1] * d
    ok = []
    for target in (0.95, 2.85):
        dt = _cfl_dt(patch, h, d, target)
        vnew, _ = godunov1(patch, dt, h, GAMMA, d)
        ok.append(det.admissible(vnew, GAMMA, d))
    assert ok[0].all()
    assert not ok[1].all()


def test_first_order_convergence():
    """The first-order subgrid scheme run alone on the periodic subgrid of the
    smooth vortex converges at first order to the exact translated averages."""
    errs = []
    t_end = 0.5
    for n in (8, 16, 32):
        w = inputs.vortex_2d(n, 1)
        g = Grid(w["ncell"], w["x0"], w["dx"], w["bc"])
        sch = Scheme(g, 1, GAMMA)
        _, V0 = project_problem(sch, w["problem"])
        G = global_subgrid(V0, 2)
        h = [g.dx[k] / sch.Ns for k in range(2)]
        t = 0.0
        while t < t_end - 1e-14:
            P = np.pad(G, ((0, 0), (3, 3), (3, 3)), mode="wrap")[:, None]
            dt = min(_cfl_dt(P, h, 2, 0.9), t_end - t)
            G = godunov1(P, dt, h, GAMMA, 2)[0][:, 0]
            t += dt
        moved = dict(w["problem"])
        moved["vortex"] = dict(center=(t, t), strength=5.0)
        _, Vexact = project_problem(sch, moved)
        Gx = global_subgrid(Vexact, 2)
        errs.append(np.abs(G[0] - Gx[0]).sum() * h[0] * h[1])
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert 0.75 < rates[-1] < 1.3, (errs, rates)


def _cascade_case():
    g = Grid((4, 4), (0.0, 0.0), (0.25, 0.25), (0, 0, 0, 0))
    for seed in range(40):
        rng = np.random.default_rng(100 + seed)
        sch = Scheme(g, 1, GAMMA, cascade=True)
        st = rough_forced_state(sch, rng, [(1, 1), (2, 3)])
        dt = stable_dt(sch, st, 0.9 / (2 * 3))
        new, info = step(sch, st, dt, force_all=True)
        if 0 < info["fallback"] < 16:
            return sch, st, dt, new, info
    raise AssertionError("no seed produced a WENO3 result that fails PAD")


def test_cascade_step_conserves_and_is_local():
    """Rough periodic data, every cell on the subgrid: the step with the
    first-order layer keeps the totals (each face carries one flux), the
    cells it recomputes are admissible, and against the two-level step it
    changes only those cells and the subcell layers of their neighbours that
    touch them."""
    sch, st, dt, new, info = _cascade_case()
    d, Ns = 2, sch.Ns
    h2 = (sch.grid.dx[0] / Ns) * (sch.grid.dx[1] / Ns)
    tot0 = st.Vs.sum(axis=(1, 2, 3, 4)) * h2
    tot1 = new.Vs.sum(axis=(1, 2, 3, 4)) * h2
    np.testing.assert_allclose(tot1, tot0, rtol=1e-13, atol=1e-13)

    two = Scheme(sch.grid, sch.N, GAMMA, cascade=False)
    old, info2 = step(two, st, dt, force_all=True)
    assert info2["fallback"] == 0
    bad = ~det.admissible(old.Vs, GAMMA, d)             # the cells the layer recomputes
    assert bad.sum() == info["fallback"]
    assert det.admissible(new.Vs[:, bad], GAMMA, d).all()
    allowed = np.zeros((4, 4, Ns, Ns), dtype=bool)
    for c in np.argwhere(bad):
        i, j = c
        allowed[i, j] = True
        allowed[(i + 1) % 4, j, 0, :] = True             # right neighbour, its low x layer
        allowed[(i - 1) % 4, j, Ns - 1, :] = True        # left neighbour, its high x layer
        allowed[i, (j + 1) % 4, :, 0] = True
        allowed[i, (j - 1) % 4, :, Ns - 1] = True
    changed = np.any(new.Vs != old.Vs, axis=0)
    assert not np.any(changed & ~allowed)
    # every neighbour layer touching a recomputed cell did change
    touched = 0
    for c in np.argwhere(bad):
        i, j = c
        for nb, layer in ((((i + 1) % 4, j), (0, slice(None))), (((i - 1) % 4, j), (Ns - 1, slice(None))),
                          ((i, (j + 1) % 4), (slice(None), 0)), ((i, (j - 1) % 4), (slice(None), Ns - 1))):
            if not bad[nb]:
                assert changed[nb + layer].any()
                touched += 1
    assert touched > 0
