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
    g = Grid(w["ncell"], w["x0"], w["dx"], w["bc"])
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
    """max |U_v| per variable, broadcastable against U."""
    ax = tuple(range(1, U.ndim))
    s = np.max(np.abs(U), axis=ax)
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
