"""Seeded synthetic workloads (problem parameters only, no scheme arithmetic).

Both the CUDA library (through the binding) and the test-side CPU checker
consume these descriptions; each side evaluates and projects the initial data
with its own code.  Shapes follow the paper's test problems:
  * circular / spherical explosion (Sec. 5.8, radius and the Sod states),
  * four-quadrant 2D Riemann data (Sec. 5.6 quadrant convention), with seeded
    states rho ~ U[0.1, 1.5], p ~ U[0.02, 1.5], u, v ~ U[-1, 1],
  * the five 2D Riemann problems of Sec. 5.6 (the serving runs draw from
    them, densities and pressures jittered by 2%),
  * isentropic vortex (Sec. 5.2, strength 5), alone or superposed.
Seeds are 1406 + workload index with numpy's default_rng.

A workload dict carries:
  dim, ncell, x0, dx, bc (per face: 0 periodic, 1 transmissive, 2 reflective,
  3 inflow, 4 front), bc_states (conserved state of each inflow face),
  bc_fronts (per front face: axis, a, b, before / after = (kind, state)), N,
  gamma, cfl, steps, problem (see below), name.
Problem dicts: {"kind": "radial", "center", "radius", "inner", "outer",
"cell_rho_factor"} with states (rho, vel..., p); {"kind": "quadrant", "center",
"states" (4 x (rho, u, v, p)), "vortex": None | {"center", "strength"}}.
"""
import numpy as np

GAMMA = 1.4
PERIODIC = 0
TRANSMISSIVE = 1


def seed_of(index):
    return 1406 + index


def _grid(lo, hi, n, dim, bc):
    return dict(dim=dim, ncell=(n,) * dim, x0=(lo,) * dim, dx=((hi - lo) / n,) * dim,
                bc=(bc,) * (2 * dim))


def random_quadrants(rng):
    """Four primitive 2D states (rho, u, v, p)."""
    states = []
    for _ in range(4):
        rho = rng.uniform(0.1, 1.5)
        u = rng.uniform(-1.0, 1.0)
        v = rng.uniform(-1.0, 1.0)
        p = rng.uniform(0.02, 1.5)
        states.append((rho, u, v, p))
    return states


def explosion_2d(n=32, N=3, steps=20):
    """Circular explosion on [-1,1]^2, transmissive (r < 0.5: rho=1, p=1)."""
    w = _grid(-1.0, 1.0, n, 2, TRANSMISSIVE)
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (2 * (2 * N + 1)), steps=steps,
             name=f"2D explosion N={N} {n}x{n} transmissive")
    w["problem"] = dict(kind="radial", center=(0.0, 0.0), radius=0.5,
                        inner=(1.0, 0.0, 0.0, 1.0), outer=(0.125, 0.0, 0.0, 0.1),
                        cell_rho_factor=None)
    return w


def quadrants_vortex_2d(n=512, N=5, steps=10, index=1):
    """Seeded four-quadrant Riemann data + vortex (strength 5) on [-5,5]^2, periodic."""
    rng = np.random.default_rng(seed_of(index))
    w = _grid(-5.0, 5.0, n, 2, PERIODIC)
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (2 * (2 * N + 1)), steps=steps,
             name=f"2D quadrant Riemann + vortex N={N} {n}x{n} periodic")
    w["problem"] = dict(kind="quadrant", center=(0.0, 0.0), states=random_quadrants(rng),
                        vortex=dict(center=(0.0, 0.0), strength=5.0))
    return w


def explosion_3d(n=128, N=3, steps=20, index=2):
    """Spherical explosion on [-1,1]^3 (r < 0.4) with seeded +-1% per-cell density noise."""
    rng = np.random.default_rng(seed_of(index))
    w = _grid(-1.0, 1.0, n, 3, TRANSMISSIVE)
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (3 * (2 * N + 1)), steps=steps,
             name=f"3D explosion N={N} {n}^3 transmissive, 1% density noise")
    fac = 1.0 + 0.01 * rng.uniform(-1.0, 1.0, size=(n, n, n))
    w["problem"] = dict(kind="radial", center=(0.0, 0.0, 0.0), radius=0.4,
                        inner=(1.0, 0.0, 0.0, 0.0, 1.0), outer=(0.125, 0.0, 0.0, 0.0, 0.1),
                        cell_rho_factor=fac)
    return w


def quadrants_2d(n=200, N=9, steps=10, index=3, lo=-0.5, hi=0.5):
    """Seeded four-quadrant Riemann data on [lo,hi]^2, periodic."""
    rng = np.random.default_rng(seed_of(index))
    w = _grid(lo, hi, n, 2, PERIODIC)
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (2 * (2 * N + 1)), steps=steps,
             name=f"2D quadrant Riemann N={N} {n}x{n} periodic")
    w["problem"] = dict(kind="quadrant", center=(0.5 * (lo + hi),) * 2,
                        states=random_quadrants(rng), vortex=None)
    return w


def vortex_2d(n, N, steps=None):
    """Pure isentropic vortex of Sec. 5.2 on [-5,5]^2 (ambient rho=u=v=p=1), periodic."""
    w = _grid(-5.0, 5.0, n, 2, PERIODIC)
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (2 * (2 * N + 1)), steps=steps,
             name=f"2D isentropic vortex N={N} {n}x{n}")
    amb = (1.0, 1.0, 1.0, 1.0)
    w["problem"] = dict(kind="quadrant", center=(0.0, 0.0), states=[amb] * 4,
                        vortex=dict(center=(0.0, 0.0), strength=5.0))
    return w


# Sec. 5.6, the initial states of the five 2D Riemann problems RP1..RP5 as
# (rho, u, v, p) in quadrant order (1: x>0,y>0; 2: x<=0,y>0; 3: x<=0,y<=0;
# 4: x>0,y<=0), each with its final time.
RP2D = (
    (((1.5, 0.0, 0.0, 1.5), (0.5323, 1.206, 0.0, 0.3),
      (0.138, 1.206, 1.206, 0.029), (0.5323, 0.0, 1.206, 0.3)), 0.25),
    (((1.1, 0.0, 0.0, 1.1), (0.5065, 0.8939, 0.0, 0.35),
      (1.1, 0.8939, 0.8939, 1.1), (0.5065, 0.0, 0.8939, 0.35)), 0.25),
    (((1.0, 0.75, -0.5, 1.0), (2.0, 0.75, 0.5, 1.0),
      (1.0, -0.75, 0.5, 1.0), (3.0, -0.75, -0.5, 1.0)), 0.30),
    (((0.5197, 0.1, 0.1, 0.4), (1.0, -0.6259, 0.1, 1.0),
      (0.8, 0.1, 0.1, 1.0), (1.0, 0.1, -0.6259, 1.0)), 0.25),
    (((0.5313, 0.0, 0.0, 0.4), (1.0, 0.7276, 0.0, 1.0),
      (0.8, 0.0, 0.0, 1.0), (1.0, 0.0, 0.7276, 1.0)), 0.25),
)


def riemann_2d(n, N, config, jitter=0.0, rng=None, bc=TRANSMISSIVE):
    """One of the five 2D Riemann problems of Sec. 5.6 on [-0.5,0.5]^2
    (config 0..4 = RP1..RP5).  With jitter > 0 every density and pressure is
    scaled by a seeded factor in [1 - jitter, 1 + jitter]."""
    states, t_final = RP2D[config]
    states = [list(s) for s in states]
    if jitter > 0.0:
        for s in states:
            s[0] *= 1.0 + rng.uniform(-jitter, jitter)
            s[3] *= 1.0 + rng.uniform(-jitter, jitter)
    w = _grid(-0.5, 0.5, n, 2, bc)
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (2 * (2 * N + 1)), steps=None, t_end=t_final,
             name=f"2D Riemann problem RP{config + 1} N={N} {n}x{n}")
    w["problem"] = dict(kind="quadrant", center=(0.0, 0.0),
                        states=[tuple(s) for s in states], vortex=None)
    return w


def serving_runs(count=256, index=4, sizes=(32, 64, 128, 256), orders=(3, 5), t_end=None):
    """Independent runs of the 2D Riemann problems of Sec. 5.6: per run a
    seeded configuration RP1..RP5 (densities and pressures jittered by 2%),
    grid size and order drawn uniformly; each run goes to t_end (default: the
    configuration's final time)."""
    rng = np.random.default_rng(seed_of(index))
    runs = []
    for r in range(count):
        n = int(rng.choice(sizes))
        N = int(rng.choice(orders))
        cfg = int(rng.integers(len(RP2D)))
        w = riemann_2d(n, N, cfg, jitter=0.02, rng=rng)
        if t_end is not None:
            w["t_end"] = float(t_end)
        w["name"] = f"serving run {r}: " + w["name"]
        runs.append(w)
    return runs


REFLECTIVE = 2
INFLOW = 3


def conserved_state(rho, vel, p, gamma=GAMMA):
    """Conserved vector (rho, rho v, rho E) of one primitive state."""
    kin = 0.5 * rho * sum(v * v for v in vel)
    return [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + kin]


# Sec. 5.1 table: left / right primitive states (rho, u, p) and final times of
# the Sod and Lax shock tubes (initial discontinuity at x = 0.5, v = 0)
SHOCK_TUBES = {"sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.2),
               "lax": ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.14)}


def shock_tube(name, nx=20, ny=5, N=9):
    """Sod or Lax shock tube of Sec. 5.1 on [0,1] x [-0.5,0.5]: Dirichlet
    (inflow with the initial left / right state) in x, periodic in y; the
    paper's mesh is 20 x 5 cells at N = 9."""
    left, right, t_final = SHOCK_TUBES[name]
    w = dict(dim=2, ncell=(nx, ny), x0=(0.0, -0.5), dx=(1.0 / nx, 1.0 / ny),
             bc=(INFLOW, INFLOW, PERIODIC, PERIODIC))
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (2 * (2 * N + 1)), steps=None, t_end=t_final,
             name=f"{name} shock tube N={N} {nx}x{ny}")
    lp = (left[0], left[1], 0.0, left[2])
    rp = (right[0], right[1], 0.0, right[2])
    w["bc_states"] = {0: conserved_state(left[0], (left[1], 0.0), left[2]),
                      1: conserved_state(right[0], (right[1], 0.0), right[2])}
    w["problem"] = dict(kind="quadrant", center=(0.5, 0.0), states=[rp, lp, lp, rp], vortex=None)
    return w


FRONT = 4


def oblique_shock_states(gamma=GAMMA):
    """Sec. 5.4: the Mach 10 shock of the double-Mach problem in the rotated
    frame (x' along the shock normal): behind it (rho, u', v', p) =
    (8/gamma, 8.25, 0, 116.5/gamma), ahead (1, 0, 0, 1/gamma).  Reading: the
    printed factor 1/gamma scales density and pressure only -- with it on the
    velocity too the pair would not satisfy the Rankine-Hugoniot conditions of
    a shock moving at Mach 10 into the state ahead (sound speed 1)."""
    return (8.0 / gamma, 8.25, 0.0, 116.5 / gamma), (1.0, 0.0, 0.0, 1.0 / gamma)


def double_mach(nx=350, ny=100, N=5, length=3.5, shock_x=0.1, angle_deg=30.0, height=1.0):
    """Double Mach reflection of Sec. 5.4 on [0, length] x [0, 1]: the shock
    x' = x cos(angle) - y sin(angle) = shock_x (60 degrees to the wall),
    moving along x' at speed 10.  Boundaries: post-shock inflow on the left,
    outflow on the right; the bottom is post-shock inflow before the shock's
    foot x = shock_x / cos(angle) and a reflecting wall after it; the top
    follows the exact moving shock (post-shock state behind it, pre-shock
    state ahead).  The paper's mesh is 350 x 100 (h = 1/100), N = 1, 2, 5, 9,
    t_final = 0.2, Rusanov flux."""
    a = np.radians(angle_deg)
    c, s = np.cos(a), np.sin(a)
    post_rot, pre = oblique_shock_states()
    post = (post_rot[0], post_rot[1] * c, -post_rot[1] * s, post_rot[3])
    qpost = conserved_state(post[0], (post[1], post[2]), post[3])
    qpre = conserved_state(pre[0], (pre[1], pre[2]), pre[3])
    w = dict(dim=2, ncell=(nx, ny), x0=(0.0, 0.0), dx=(length / nx, height / ny),
             bc=(INFLOW, TRANSMISSIVE, FRONT, FRONT))
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (2 * (2 * N + 1)), steps=None, t_end=0.2,
             name=f"double Mach reflection N={N} {nx}x{ny}")
    w["bc_states"] = {0: qpost}
    w["bc_fronts"] = {
        # bottom: post-shock inflow before the foot of the shock, wall after it
        2: dict(axis=0, a=shock_x / c, b=0.0, before=(INFLOW, qpost), after=(REFLECTIVE, None)),
        # top (y = height): x'(x, height) = shock_x + 10 t <=> x = (shock_x + height s + 10 t) / c
        3: dict(axis=0, a=(shock_x + height * s) / c, b=10.0 / c, before=(INFLOW, qpost),
                after=(INFLOW, qpre)),
    }
    w["problem"] = dict(kind="planar", normal=(c, -s), offset=shock_x, inner=post, outer=pre)
    return w


def closed_box(n=32, N=3, dim=2):
    """Off-centre explosion in the unit box with reflecting walls everywhere
    (mass and energy stay constant)."""
    w = _grid(0.0, 1.0, n, dim, REFLECTIVE)
    w.update(N=N, gamma=GAMMA, cfl=0.9 / (dim * (2 * N + 1)), steps=None,
             name=f"{dim}D explosion in a closed box N={N} {n}^{dim}")
    c = (0.31, 0.42, 0.55)[:dim]
    w["problem"] = dict(kind="radial", center=c, radius=0.3, inner=(1.0,) + (0.0,) * dim + (1.0,),
                        outer=(0.125,) + (0.0,) * dim + (0.1,), cell_rho_factor=None)
    return w


def random_state_perturbation(shape, seed, scale=1e-3):
    """Seeded uniform numbers in [-scale, scale] (used to jitter test data)."""
    return np.random.default_rng(seed).uniform(-scale, scale, size=shape)
