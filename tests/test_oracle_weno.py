"""Pins of the oracle's subcell ADER-WENO3 operator (Sec. 4.3 Eq. aderweno).

The paper defers the operator's formulas to the cited literature, so these pins
check the reading by mathematics: exactness for quadratics, the smoothness
indicator's closed form, the ENO property, constant preservation, conservation
and third-order convergence of the full subgrid scheme."""
import numpy as np
import pytest

from oracle import euler
from oracle.dg import Grid
from oracle.ic import initial_state, project_problem
from oracle.step import Scheme, step, stable_dt
from oracle.weno import Weno3, ader_weno
from paper_1406_7416_gb300 import inputs

GAMMA = 1.4


def _averages(F, lo, hi):
    return (F(hi) - F(lo)) / (hi - lo)


def test_quadratic_reconstructed_exactly():
    """All three stencils reproduce a quadratic, so any weights give its point
    values at the subcell GL nodes."""
    wn = Weno3()
    L = 9
    c = (0.3, -1.1, 0.7)
    P = lambda x: c[0] * x + c[1] * x ** 2 / 2 + c[2] * x ** 3 / 3   # antiderivative
    f = lambda x: c[0] + c[1] * x + c[2] * x ** 2
    j = np.arange(L)
    avg = _averages(P, j, j + 1.0)
    out = wn.line(avg, 0)                                           # subcells 2..L-3
    for i, s in enumerate(range(2, L - 2)):
        np.testing.assert_allclose(out[i], f(s + wn.xi), rtol=1e-12, atol=1e-12)


def test_smoothness_indicator_closed_form():
    """sigma = c1^2 + 2 c1 c2 + 16/3 c2^2 for p = c0 + c1 xi + c2 xi^2."""
    wn = Weno3()
    rng = np.random.default_rng(0)
    c = rng.uniform(-2, 2, size=(20, 3))
    np.testing.assert_allclose(wn.smoothness(c),
                               c[:, 1] ** 2 + 2 * c[:, 1] * c[:, 2] + 16.0 / 3.0 * c[:, 2] ** 2,
                               rtol=1e-13)


def test_eno_property_at_a_jump():
    """Next to a jump the stencil that does not cross it dominates: the
    reconstruction of constant data left of the jump stays constant."""
    wn = Weno3()
    u = np.array([1.0] * 6 + [5.0] * 6)
    out = wn.line(u, 0)          # subcells 2..9
    # subcell 5 (last of the left plateau): left stencil {3,4,5} is constant
    np.testing.assert_allclose(out[5 - 2], 1.0, atol=1e-9)
    np.testing.assert_allclose(out[6 - 2], 5.0, atol=1e-9)


def _euler_patch(Q, Ns, d, T=2):
    L = Ns + 6
    return np.broadcast_to(np.asarray(Q).reshape((d + 2,) + (1,) * (1 + d)),
                           (d + 2, T) + (L,) * d).copy()


@pytest.mark.parametrize("d", [2, 3])
def test_constant_state_preserved(d):
    Q = euler.prim_to_cons(np.array(0.9), [np.array(0.4)] * d, np.array(0.7), GAMMA)
    Ns = 5
    patch = _euler_patch(Q, Ns, d)
    vnew, faces = ader_weno(patch, 0.01, [0.1] * d, GAMMA, d)
    np.testing.assert_allclose(vnew, patch[(slice(None), slice(None)) + (slice(3, 3 + Ns),) * d],
                               rtol=1e-14, atol=1e-14)


def test_conservation_on_the_patch():
    """sum(v_new - v_old) h^d = -dt sum over the patch boundary of sub-face fluxes."""
    d, Ns = 2, 7
    rng = np.random.default_rng(4)
    L = Ns + 6
    rho = rng.uniform(0.5, 1.5, size=(1, L, L))
    u = rng.uniform(-0.5, 0.5, size=(1, L, L))
    v = rng.uniform(-0.5, 0.5, size=(1, L, L))
    p = rng.uniform(0.5, 1.5, size=(1, L, L))
    patch = euler.prim_to_cons(rho, [u, v], p, GAMMA)
    dt, h = 0.002, [0.05, 0.05]
    vnew, faces = ader_weno(patch, dt, h, GAMMA, d)
    vold = patch[:, :, 3:3 + Ns, 3:3 + Ns]
    change = (vnew - vold).sum(axis=(2, 3))
    boundary = sum(-(dt / h[k]) * (faces[k][1].sum(axis=2) - faces[k][0].sum(axis=2))
                   for k in range(d))
    np.testing.assert_allclose(change, boundary, atol=1e-13)


def test_subgrid_scheme_third_order():
    """With every cell forced onto the subgrid the step is the pure ADER-WENO3
    finite volume scheme on the N_s-refined grid; on the smooth vortex its
    subcell-average density error drops at third order (exact averages: the
    vortex translated with the ambient velocity (1, 1))."""
    errs = []
    t_end = 0.1
    for n in (12, 24):
        w = inputs.vortex_2d(n, 1)
        g = Grid(w["ncell"], w["x0"], w["dx"], w["bc"])
        sch = Scheme(g, 1, GAMMA)
        U0, V0 = project_problem(sch, w["problem"])
        st = initial_state(sch, U0, V0, detect_ic=False)
        st.beta[...] = 1
        st.Vs = V0.copy()
        t = 0.0
        while t < t_end - 1e-14:
            dt = min(stable_dt(sch, st, w["cfl"]), t_end - t)
            st, _ = step(sch, st, dt, force_all=True)
            t += dt
        moved = dict(w["problem"])
        moved["vortex"] = dict(center=(t, t), strength=5.0)
        _, Vexact = project_problem(sch, moved)
        errs.append(np.abs(st.Vs[0] - Vexact[0]).sum() * (g.dx[0] / sch.Ns) ** 2)
    rate = np.log2(errs[0] / errs[1])
    assert rate > 2.7, (errs, rate)
