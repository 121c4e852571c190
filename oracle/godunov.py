"""First-order Godunov-type finite volume update on the subgrid (oracle).

Test infrastructure only: imported by the tests, by the checker in
__graft_entry__.smoke() and by the CPU-baseline leg of bench.py, never by the
product path.

Sec. 6 (Fig. algo2) names one more MOOD layer after the subcell ADER-WENO3
scheme: where the WENO3 result is still not acceptable, the troubled cell is
recomputed on its subgrid with a more dissipative first-order Godunov-type
scheme.  The paper prints no formulas for it; the reading here:
  * data: the subcell averages v^n of the cell and the first ghost layer of its
    face neighbours, built from Eq. (ader.icbc) exactly as for the WENO3 patch;
  * flux: the Rusanov flux of Sec. 2.3 between the two piecewise-constant
    states of every sub-face (no reconstruction, no predictor);
  * update: one forward-Euler step,
        v^{n+1}_s = v^n_s - sum_d (dt/h_d) (F_{s+1/2 e_d} - F_{s-1/2 e_d}).
With alpha >= |u| + c on both sides of a sub-face, each updated subcell is a
convex combination of v_s and the states v -/+ f(v)/alpha of its neighbours
whenever sum_d alpha dt/h_d <= 1, which the time step of Eq. (cfl.fv) (with
a safety factor below one) guarantees; those states are admissible for the
Euler equations, so the layer preserves rho > 0 and p > 0.

Parity unpinned by the paper (no formulas).  Pins (tests/test_oracle_godunov.py):
constant and contact preservation, conservation, positivity on rough data at
the CFL bound, first-order convergence on the smooth vortex.
"""
import numpy as np

from . import euler


def godunov1(patch, dt, h, gamma, dim):
    """One first-order Rusanov step on a batch of subcell patches.

    patch: (nvar, T, L, .., L) with L = N_s + 6 (local index -3..N_s+2, the
    layout of the WENO3 patch; only local -1..N_s is read).  Returns (v_new,
    faces) like weno.ader_weno: v_new (nvar, T, N_s, .., N_s) and faces[k] =
    (low, high) sub-face fluxes on the cell faces normal to axis k, each over
    the d-1 tangential subcell axes."""
    L = patch.shape[2]
    Ns = L - 6
    lead = (slice(None), slice(None))
    core = patch[lead + (slice(2, Ns + 4),) * dim]           # local -1..Ns
    vnew = patch[lead + (slice(3, 3 + Ns),) * dim].copy()
    faces = []
    for k in range(dim):
        left = list(lead) + [slice(1, Ns + 1)] * dim
        right = list(left)
        left[2 + k] = slice(0, Ns + 1)                         # local -1..Ns-1
        right[2 + k] = slice(1, Ns + 2)                        # local 0..Ns
        G = euler.rusanov(core[tuple(left)], core[tuple(right)], gamma, k)
        hi = np.take(G, np.arange(1, Ns + 1), axis=2 + k)
        lo = np.take(G, np.arange(0, Ns), axis=2 + k)
        vnew = vnew - (dt / h[k]) * (hi - lo)
        faces.append((np.take(G, 0, axis=2 + k), np.take(G, Ns, axis=2 + k)))
    return vnew, faces
