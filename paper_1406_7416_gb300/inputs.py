"""Seeded synthetic workloads (problem parameters only, no scheme arithmetic).

Both the CUDA library (through the binding) and the test-side CPU checker
consume these descriptions; each side evaluates and projects the initial data
with its own code.  Shapes follow the paper's test problems:
  * circular / spherical explosion (Sec. 5.8, radius and the Sod states),
  * four-quadrant 2D Riemann data (Sec. 5.6 quadrant convention), with seeded
    states rho ~ U[0.1, 1.5], p ~ U[0.02, 1.5], u, v ~ U[-1, 1],
  * isentropic vortex (Sec. 5.2, strength 5), alone or superposed.
Seeds are 1406 + workload index with numpy's default_rng.

A workload dict carries:
  dim, ncell, x0, dx, bc (per face: 0 periodic, 1 transmissive), N, gamma,
  cfl, steps, problem (see below), name.
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


def serving_runs(count=256, index=4, sizes=(32, 64, 128, 256), orders=(3, 5), t_end=0.2):
    """Independent 2D runs with grid sizes and orders drawn uniformly; seeded
    quadrant states on [-0.5,0.5]^2; each run goes to t_end."""
    rng = np.random.default_rng(seed_of(index))
    runs = []
    for r in range(count):
        n = int(rng.choice(sizes))
        N = int(rng.choice(orders))
        w = _grid(-0.5, 0.5, n, 2, PERIODIC)
        w.update(N=N, gamma=GAMMA, cfl=0.9 / (2 * (2 * N + 1)), steps=None, t_end=t_end,
                 name=f"serving run {r}: N={N} {n}x{n}")
        w["problem"] = dict(kind="quadrant", center=(0.0, 0.0),
                            states=random_quadrants(rng), vortex=None)
        runs.append(w)
    return runs


def random_state_perturbation(shape, seed, scale=1e-3):
    """Seeded uniform numbers in [-scale, scale] (used to jitter test data)."""
    return np.random.default_rng(seed).uniform(-scale, scale, size=shape)
