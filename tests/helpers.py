"""Test glue: layout conversion between the oracle's arrays and the C ABI's
host arrays, oracle set-up from a workload dict, and comparison helpers."""
import numpy as np

from oracle import detect as odet
from oracle.dg import Grid
from oracle.ic import initial_state, project_problem
from oracle.step import Scheme, State, stable_dt, step


def to_abi(U, dim):
    """Oracle (nvar, cells..., nodes...) -> ABI [cell][var][node], x fastest."""
    cells = list(range(1, 1 + dim))[::-1]
    nodes = list(range(1 + dim, 1 + 2 * dim))[::-1]
    A = np.transpose(U, cells + [0] + nodes)
    nv = U.shape[0]
    ncell = int(np.prod(U.shape[1:1 + dim]))
    return np.ascontiguousarray(A).reshape(ncell, nv, -1)


def from_abi(A, dim, ncell, nper):
    """ABI [cell][var][node] -> oracle (nvar, cells..., nodes...)."""
    nv = A.shape[1]
    shp = tuple(ncell[::-1]) + (nv,) + (nper,) * dim
    X = A.reshape(shp)
    cells = list(range(dim))[::-1]
    nodes = list(range(dim + 1, 2 * dim + 1))[::-1]
    return np.ascontiguousarray(np.transpose(X, [dim] + cells + nodes))


def beta_to_abi(beta):
    return np.ascontiguousarray(np.transpose(beta)).ravel().astype(np.uint8)


def beta_from_abi(b, ncell):
    return np.transpose(b.reshape(tuple(ncell[::-1]))).astype(np.int32)


def oracle_setup(w, detect_ic=True, **kw):
    g = Grid(w["ncell"], w["x0"], w["dx"], w["bc"], w.get("bc_states"), w.get("bc_fronts"))
    sch = Scheme(g, w["N"], w["gamma"], **kw)
    U0, V0 = project_problem(sch, w["problem"])
    return sch, initial_state(sch, U0, V0, detect_ic=detect_ic), U0, V0


def advance(sch, st, nsteps, cfl, force=False):
    for _ in range(nsteps):
        st, _ = step(sch, st, stable_dt(sch, st, cfl), force_all=force)
    return st


def sub_to_abi(sch, st):
    Vs = np.where(np.isnan(st.Vs), 0.0, st.Vs)
    return to_abi(Vs, sch.dim)


def load_state(solver, sch, st):
    solver.load_full(to_abi(st.U, sch.dim), beta_to_abi(st.beta), sub_to_abi(sch, st))


def scale_per_var(U):
    """max |U_v| per variable, broadcastable against U; a variable that
    vanishes identically (e.g. the transverse momentum of a planar problem,
    zero up to round-off) is measured against 1e-3 of the largest variable's
    scale instead of its own round-off."""
    ax = tuple(range(1, U.ndim))
    s = np.max(np.abs(U), axis=ax)
    s = np.maximum(s, 1e-3 * np.max(s))
    return np.maximum(s, 1e-300).reshape((-1,) + (1,) * (U.ndim - 1))


def assert_close_rel(got, ref, rtol, what=""):
    """|got - ref| <= rtol * max_v |ref_v| per variable (relative to the
    variable's magnitude over the grid, so components through zero are fine)."""
    if ref.size == 0:
        assert got.size == 0, f"{what}: size differs"
        return 0.0
    err = np.abs(got - ref) / scale_per_var(ref)
    worst = float(np.nanmax(err))
    assert np.all(np.isfinite(got) == np.isfinite(ref)), f"{what}: finiteness differs"
    assert worst <= rtol, f"{what}: max relative error {worst:.3e} > {rtol:.1e}"
    return worst


def near_threshold_cells(sch, info, margin=1e-10):
    marg = odet.detector_margin(info["vstar"], info["m"], info["M"], sch.gamma, sch.dim,
                                sch.eps, sch.floor)
    return marg < margin


def neighbourhood_mask(mask, layers, periodic):
    """Dilate a boolean cell mask by `layers` cells along every axis."""
    out = mask.copy()
    for _ in range(layers):
        grown = out.copy()
        for ax in range(mask.ndim):
            for sh in (-1, 1):
                r = np.roll(out, sh, axis=ax)
                if not periodic[ax]:
                    idx = [slice(None)] * mask.ndim
                    idx[ax] = 0 if sh == 1 else -1
                    r[tuple(idx)] = False
                grown |= r
        out = grown
    return out


def state_copy(st):
    return State(st.U.copy(), st.beta.copy(), st.Vs.copy())


def rough_conserved(shape, d, rng, mach=3.0, gamma=1.4, rho=(0.02, 5.0), p=(0.005, 5.0)):
    """Admissible conserved states with strong contrasts over `shape`: rho and
    p log-uniform over the given ranges (by default two to three decades),
    velocities up to `mach` (nvar first in the result)."""
    from oracle import euler
    rho = np.exp(rng.uniform(np.log(rho[0]), np.log(rho[1]), size=shape))
    p = np.exp(rng.uniform(np.log(p[0]), np.log(p[1]), size=shape))
    vel = [rng.uniform(-mach, mach, size=shape) for _ in range(d)]
    return euler.prim_to_cons(rho, vel, p, gamma)


def rough_forced_state(sch, rng, rough_cells, mild=False):
    """Every cell flagged (beta = 1, subcell data stored): per-cell states with
    strong jumps between cells (mild: within a factor 2, Mach 0.5) and 5%
    variation between subcells, plus cells whose subcells are rough on their
    own -- WENO3 fails the admissibility test in some cells and passes in
    others."""
    d = sch.dim
    nc = tuple(sch.grid.ncell)
    if mild:
        Vc = rough_conserved(nc, d, rng, mach=0.5, rho=(0.7, 1.4), p=(0.7, 1.4))
    else:
        Vc = rough_conserved(nc, d, rng)
    Vs = np.broadcast_to(Vc[(Ellipsis,) + (None,) * d], Vc.shape + (sch.Ns,) * d).copy()
    Vs *= 1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=Vs.shape[1:])
    for c in rough_cells:
        Vs[(slice(None),) + tuple(c)] = rough_conserved((sch.Ns,) * d, d, rng)
    return State(sch.R(Vs), np.ones(nc, dtype=np.int32), Vs)


def rough_island_state(sch, rng, rough_cells, gamma=1.4):
    """A uniform flow (rho = p = 1, velocity 0.3 per axis) with a few flagged
    cells holding rough subcell data: the limiter runs in and around them
    while their unlimited neighbours take the flux correction."""
    from oracle import euler
    d, Ns = sch.dim, sch.Ns
    nc = tuple(sch.grid.ncell)
    base = euler.prim_to_cons(np.array(1.0), [np.array(0.3)] * d, np.array(1.0), gamma)
    Vs = np.broadcast_to(base.reshape((d + 2,) + (1,) * (2 * d)), (d + 2,) + nc + (Ns,) * d).copy()
    beta = np.zeros(nc, dtype=np.int32)
    for c in rough_cells:
        Vs[(slice(None),) + tuple(c)] = rough_conserved((Ns,) * d, d, rng, mach=2.0)
        beta[tuple(c)] = 1
    U = sch.R(Vs)
    stored = np.where(beta[(None, Ellipsis) + (None,) * d] == 1, Vs, np.nan)
    return State(U, beta, stored)
