"""Pins of the oracle's full step (Sec. 4.4): conservation, free stream,
design order and a quiet limiter on the smooth vortex, symmetry, and planted
mistakes that those pins must catch."""
import numpy as np
import pytest

import oracle.step as ostep
from oracle import euler
from oracle.dg import Grid
from oracle.ic import initial_state, project_problem
from oracle.step import Scheme, State, stable_dt, step
from paper_1406_7416_gb300 import inputs

GAMMA = 1.4


def _setup(w, **kw):
    g = Grid(w["ncell"], w["x0"], w["dx"], w["bc"])
    sch = Scheme(g, w["N"], w["gamma"], **kw)
    U0, V0 = project_problem(sch, w["problem"])
    return sch, initial_state(sch, U0, V0)


def _totals(sch, U):
    W = sch.basis.w
    if sch.dim == 2:
        return np.einsum("vijab,a,b->v", U, W, W)
    return np.einsum("vijkabc,a,b,c->v", U, W, W, W)


def _periodic_explosion(n=12, N=2, dim=2):
    w = inputs.explosion_2d(n=n, N=N) if dim == 2 else inputs.explosion_3d(n=n, N=N)
    w["bc"] = (0,) * (2 * dim)
    w["problem"]["cell_rho_factor"] = None
    return w


@pytest.mark.parametrize("dim,n,N", [(2, 12, 2), (2, 8, 4), (3, 5, 1)])
def test_conservation_with_limiter(dim, n, N):
    w = _periodic_explosion(n, N, dim)
    sch, st = _setup(w)
    t0 = _totals(sch, st.U)
    troubled = 0
    for _ in range(3):
        dt = stable_dt(sch, st, 0.5 * w["cfl"])
        st, info = step(sch, st, dt)
        troubled += info["troubled"]
    assert troubled > 0
    scale = np.abs(t0).max()
    np.testing.assert_allclose(_totals(sch, st.U), t0, atol=2e-14 * scale * n ** dim)


def test_skipping_the_flux_correction_breaks_conservation(monkeypatch):
    """Planted mistake: without the neighbour flux correction the limited step
    is no longer conservative (so the conservation pin guards it)."""
    w = _periodic_explosion(12, 2)
    sch, st = _setup(w)
    for _ in range(2):
        st, _ = step(sch, st, stable_dt(sch, st, 0.5 * w["cfl"]))
    dt = stable_dt(sch, st, 0.5 * w["cfl"])
    _, info = step(sch, st, dt)
    assert info["fixed"] > 0
    t0 = _totals(sch, st.U)
    monkeypatch.setattr(ostep, "neighbour", lambda *a: None)
    st, info = step(sch, st, dt)
    assert info["troubled"] > 0
    assert np.max(np.abs(_totals(sch, st.U) - t0)) > 1e-8


@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("dim", [2, 3])
def test_free_stream(force, dim):
    N = 2
    n = 4
    g = Grid((n,) * dim, (0.0,) * dim, (0.25,) * dim, (0,) * (2 * dim))
    sch = Scheme(g, N, GAMMA)
    Q = euler.prim_to_cons(np.array(0.7), [np.array(0.3 - 0.1 * k) for k in range(dim)],
                           np.array(1.3), GAMMA)
    U = np.broadcast_to(Q.reshape((dim + 2,) + (1,) * (2 * dim)),
                        (dim + 2,) + (n,) * dim + (N + 1,) * dim).copy()
    Vs = np.broadcast_to(Q.reshape((dim + 2,) + (1,) * (2 * dim)),
                         (dim + 2,) + (n,) * dim + (2 * N + 1,) * dim).copy()
    st = State(U, np.full((n,) * dim, 1 if force else 0, dtype=np.int32), Vs)
    for _ in range(2):
        st, info = step(sch, st, 0.01, force_all=force)
        assert info["troubled"] == (n ** dim if force else 0)
    np.testing.assert_allclose(st.U, U, rtol=2e-14, atol=2e-15)


def test_vortex_design_order_and_quiet_limiter():
    """Sec. 2.4 / Sec. 5.2: order about N+1 on the smooth vortex and no troubled
    cells on the finer grid (N = 3, 12^2 -> 24^2 on [-5, 5]^2, t = 0.2,
    half the configured CFL number)."""
    errs = []
    flags = []
    for n in (12, 24):
        w = inputs.vortex_2d(n, 3)
        sch, st = _setup(w)
        t, T, nflag = 0.0, 0.2, int(st.beta.sum())
        while t < T - 1e-14:
            dt = min(stable_dt(sch, st, 0.5 * w["cfl"]), T - t)
            st, info = step(sch, st, dt)
            t += dt
            nflag += info["troubled"]
        moved = dict(w["problem"])
        moved["vortex"] = dict(center=(t, t), strength=5.0)
        Ue, _ = project_problem(sch, moved)
        b = sch.basis
        errs.append(np.einsum("ijab,a,b->", np.abs(st.U[0] - Ue[0]), b.w, b.w) * sch.grid.dx[0] ** 2)
        flags.append(nflag)
    assert flags[1] == 0, flags
    assert np.log2(errs[0] / errs[1]) > 3.5, errs


def test_explosion_symmetry():
    """The circular explosion is symmetric under x -> -x and x <-> y.  The
    flags, the candidate and every DOF keep the mirror symmetry; the diagonal
    symmetry holds for the flags and the DG candidate (the dimension-by-
    dimension WENO sweeps x before y, so limited cells keep it only approximately)."""
    w = inputs.explosion_2d(n=12, N=2)
    sch, st = _setup(w)
    for it in range(2):
        dt = stable_dt(sch, st, 0.5 * w["cfl"])
        st, info = step(sch, st, dt)
        beta = info["beta"]
        assert beta.sum() > 0
        np.testing.assert_array_equal(beta, beta[::-1, :])
        if it == 0:       # before any limited cell has fed back into the DG data
            np.testing.assert_array_equal(beta, beta.T)
            us = info["Ustar"][0]
            np.testing.assert_allclose(us, np.transpose(us, (1, 0, 3, 2)), atol=1e-12)
        rho = st.U[0]
        np.testing.assert_allclose(rho, rho[::-1, :, ::-1, :], atol=1e-12)
        np.testing.assert_allclose(rho, np.transpose(rho, (1, 0, 3, 2)), atol=1e-2)


def test_initial_detection_marks_only_the_discontinuity():
    """Sec. 4.4: cells cut by the initial circle are flagged at t = 0, cells
    of constant data are not, and flagged cells start from their exact averages."""
    w = inputs.explosion_2d(n=16, N=3)
    sch, st = _setup(w)
    g = sch.grid
    xc = g.x0[0] + (np.arange(16) + 0.5) * g.dx[0]
    r = np.hypot(xc[:, None], xc[None, :])
    far = np.abs(r - 0.5) > 2.0 * g.dx[0] * np.sqrt(2)
    assert st.beta.sum() > 0
    assert st.beta[far].sum() == 0
    cut = np.abs(r - 0.5) < 0.5 * g.dx[0]
    assert st.beta[cut].all()
    np.testing.assert_allclose(sch.P(st.U)[:, st.beta == 1].shape, st.Vs[:, st.beta == 1].shape)
