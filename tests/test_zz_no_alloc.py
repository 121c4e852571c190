"""GPU test of adg_subcell_update_noalloc, the entry point for callers that
cannot allocate device memory (it keeps its scratch in a static device array).

Its output must equal the subcell data that adg_step produces when every cell
is limited: with all cells flagged before and during the step, adg_step
recomputes each cell from the stored subcell averages of its 3 x 3 (x 3)
neighbourhood, i.e. from exactly the patches this test gathers and hands to the
no-allocation entry point.  Two calls in a row cover the reuse of the shared
static scratch.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1406_7416_gb300 import adg, build_lib

from helpers import beta_to_abi, from_abi, to_abi

pytestmark = pytest.mark.gpu
RTOL = 1e-12
GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def _random_subcells(dim, N, ncell, seed):
    """Random subcell averages within 10% of a rest state, oracle layout
    (nvar, cells..., Ns...): rough enough to engage the WENO weights, mild
    enough that every reconstruction stays admissible."""
    Ns = 2 * N + 1
    rng = np.random.default_rng(seed)
    shape = tuple(ncell) + (Ns,) * dim
    rho = rng.uniform(0.9, 1.1, size=shape)
    vel = [rng.uniform(-0.1, 0.1, size=shape) for _ in range(dim)]
    p = rng.uniform(0.9, 1.1, size=shape)
    V = np.empty((dim + 2,) + shape)
    V[0] = rho
    for k in range(dim):
        V[1 + k] = rho * vel[k]
    V[-1] = p / (GAMMA - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    return V


def _patches(V, dim, N):
    """Periodic gather of the (Ns+6)^d subcell patch of every cell, ABI layout
    [cell][var][L^d] with the cell index and the patch index x fastest."""
    Ns = 2 * N + 1
    L = Ns + 6
    ncell = V.shape[1:1 + dim]
    order = [0]
    for k in range(dim):
        order += [1 + k, 1 + dim + k]
    G = np.transpose(V, order).reshape((V.shape[0],) + tuple(c * Ns for c in ncell))
    out = []
    for cell in np.ndindex(*ncell[::-1]):          # ABI order: last axis slowest
        cell = cell[::-1]
        idx = [np.mod(cell[k] * Ns - 3 + np.arange(L), ncell[k] * Ns) for k in range(dim)]
        P = G[(slice(None),) + np.ix_(*idx)]          # (nvar, L, .., L), x first
        out.append(np.transpose(P, [0] + list(range(dim, 0, -1))).reshape(V.shape[0], -1))
    return np.ascontiguousarray(np.stack(out))


@pytest.mark.parametrize("dim,N,ncell", [(2, 2, (6, 5)), (2, 5, (4, 4)), (3, 1, (3, 3, 3))])
def test_noalloc_equals_adg_step_subcell_update(dim, N, ncell):
    import torch

    Ns = 2 * N + 1
    V = _random_subcells(dim, N, ncell, seed=7 + N)
    cells = int(np.prod(ncell))
    dx = (0.1,) * dim
    h = [d / Ns for d in dx]
    dt = 0.05 * min(h)
    s = adg.Solver(dim, ncell, (0.0,) * dim, dx, (0,) * (2 * dim), N, GAMMA)
    s.set_option(adg.OPT_FORCE_LIMITER, 1)
    nv = dim + 2
    dofs = np.zeros((cells, nv, (N + 1) ** dim))
    dofs[:, 0] = 1.0
    dofs[:, -1] = 2.5
    s.load_full(dofs, np.ones(cells, dtype=np.uint8), to_abi(V, dim))
    s.step(dt)
    _, beta, sub_ref = s.read_full()
    assert beta.all() and np.isfinite(sub_ref).all()
    s.close()

    patches = torch.from_numpy(_patches(V, dim, N)).cuda()
    vnew = torch.full((cells, nv, Ns ** dim), float("nan"), dtype=torch.float64, device="cuda")
    faces = torch.zeros((cells, dim, 2, nv, Ns ** (dim - 1)), dtype=torch.float64, device="cuda")
    half = cells // 2
    calls = [(0, half), (half, cells)]                 # two calls in a row, shared scratch
    for lo, hi in calls:
        rc, msg = adg.subcell_update_noalloc(
            dim, N, GAMMA, h, dt, patches[lo:].data_ptr(), hi - lo, vnew[lo:].data_ptr(),
            faces[lo:].data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == adg.OK, msg
    torch.cuda.synchronize()
    got = vnew.cpu().numpy()
    scale = np.abs(sub_ref).max(axis=(0, 2))[None, :, None]
    err = float(np.max(np.abs(got - sub_ref) / scale))
    assert err <= RTOL, err
    # the returned cell-face fluxes close the balance of every cell:
    # sum_s (vnew - v) h^d = -dt sum_k h^(d-1) (F_high - F_low)
    P = _patches(V, dim, N).reshape((cells, nv) + (Ns + 6,) * dim)
    inner = (slice(None), slice(None)) + (slice(3, 3 + Ns),) * dim
    change = (got.reshape((cells, nv) + (Ns,) * dim) - P[inner]).sum(axis=tuple(range(2, 2 + dim)))
    F = faces.cpu().numpy()
    flux = sum((dt / h[k]) * (F[:, k, 1].sum(axis=-1) - F[:, k, 0].sum(axis=-1)) for k in range(dim))
    np.testing.assert_allclose(change, -flux, atol=1e-12 * np.abs(P).max() * Ns ** dim)


def test_noalloc_rejects_counts_beyond_its_static_scratch():
    rc, msg = adg.subcell_update_noalloc(2, 5, GAMMA, [0.01, 0.01], 1e-4, 1, 100000, 1)
    assert rc == adg.ERR_CAPACITY
    assert "static" in msg and "at most" in msg
    rc, msg = adg.subcell_update_noalloc(4, 5, GAMMA, [0.01, 0.01], 1e-4, 1, 1, 1)
    assert rc == adg.ERR_ARG and "dim" in msg


def _advertised_limit(dim, N):
    """The largest count the static scratch takes, as the capacity error states it."""
    h = [0.01] * dim
    rc, msg = adg.subcell_update_noalloc(dim, N, GAMMA, h, 1e-4, 1, 10 ** 7, 1)
    assert rc == adg.ERR_CAPACITY
    return int(msg.split("at most ")[1].split()[0])


def test_noalloc_at_its_largest_count_without_faces():
    """The largest advertised count (2D, N = 5) runs and equals adg_step on a
    one-row periodic grid of that many cells, with the faces output left out
    (NULL); one patch more is refused with ADG_ERR_CAPACITY."""
    import torch

    dim, N = 2, 5
    Ns = 2 * N + 1
    M = _advertised_limit(dim, N)
    assert M >= 16
    ncell = (M, 1)
    V = _random_subcells(dim, N, ncell, seed=11)
    dx = (0.1, 0.1)
    h = [d / Ns for d in dx]
    dt = 0.05 * min(h)
    s = adg.Solver(dim, ncell, (0.0, 0.0), dx, (0, 0, 0, 0), N, GAMMA)
    s.set_option(adg.OPT_FORCE_LIMITER, 1)
    nv = dim + 2
    dofs = np.zeros((M, nv, (N + 1) ** dim))
    dofs[:, 0] = 1.0
    dofs[:, -1] = 2.5
    s.load_full(dofs, np.ones(M, dtype=np.uint8), to_abi(V, dim))
    s.step(dt)
    _, beta, sub_ref = s.read_full()
    assert beta.all()
    s.close()
    patches = torch.from_numpy(_patches(V, dim, N)).cuda()
    vnew = torch.full((M, nv, Ns ** dim), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc, msg = adg.subcell_update_noalloc(dim, N, GAMMA, h, dt, patches.data_ptr(), M,
                                         vnew.data_ptr(), 0, stream)
    assert rc == adg.OK, msg
    torch.cuda.synchronize()
    got = vnew.cpu().numpy()
    scale = np.abs(sub_ref).max(axis=(0, 2))[None, :, None]
    assert float(np.max(np.abs(got - sub_ref) / scale)) <= RTOL
    extra = torch.zeros((M + 1, nv, (Ns + 6) ** dim), dtype=torch.float64, device="cuda")
    out = torch.zeros((M + 1, nv, Ns ** dim), dtype=torch.float64, device="cuda")
    rc, msg = adg.subcell_update_noalloc(dim, N, GAMMA, h, dt, extra.data_ptr(), M + 1,
                                         out.data_ptr(), 0, stream)
    assert rc == adg.ERR_CAPACITY and f"at most {M} " in msg
