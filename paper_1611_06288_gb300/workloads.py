"""Seeded synthetic inputs for the periodic 3D PFC solver.

This module only draws random numbers and samples closed-form initial fields
at cell centres; it holds none of the scheme's arithmetic.  Both the CUDA path
and the CPU oracle are fed from here.

Every generator returns a C-contiguous float64 numpy array of shape (n, n, n)
indexed [k, j, i] (z, y, x); cell (i, j, k) has centre ((i+1/2)h, (j+1/2)h,
(k+1/2)h) with h = L/n.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DEFAULT_SEED = 1234


def cell_centres(n: int, L: float):
    """Cell-centre coordinates (z, y, x) as broadcastable 1-D arrays."""
    h = L / n
    c = (np.arange(n) + 0.5) * h
    return c[:, None, None], c[None, :, None], c[None, None, :]


def uniform_noise(n: int, mean: float, amp: float, seed: int = DEFAULT_SEED):
    """phi = mean + amp * U(-1, 1) per cell (the small random-start case:
    n = 16, L = 32, eps = 0.025, mean = amp = 0.07)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(mean + amp * rng.uniform(-1.0, 1.0, (n, n, n)))


def smooth_mode(n: int, L: float, amp: float = 0.1):
    """phi = amp sin(2 pi x/L) cos(2 pi y/L) sin(2 pi z/L) (the smooth
    convergence-sweep workload on L = 32)."""
    z, y, x = cell_centres(n, L)
    k = 2.0 * math.pi / L
    return np.ascontiguousarray(
        amp * np.sin(k * x) * np.cos(k * y) * np.sin(k * z))


def cosine_bump(n: int, L: float = 3.2, mean: float = 0.2, amp: float = 0.05):
    """phi = mean + amp cos(2 pi x/L) cos(2 pi y/L) cos(2 pi z/L) on [0, L]^3
    (the initial data of the paper's accuracy and multigrid-complexity tests,
    Section 6.1)."""
    z, y, x = cell_centres(n, L)
    k = 2.0 * math.pi / L
    return np.ascontiguousarray(
        mean + amp * np.cos(k * x) * np.cos(k * y) * np.cos(k * z))


def uniform_01_start(n: int, mean: float = 0.2, amp: float = 0.005,
                     seed: int = DEFAULT_SEED):
    """phi = mean + amp * U[0, 1] per cell (Section 6.2 polycrystal start)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(mean + amp * rng.uniform(0.0, 1.0, (n, n, n)))


def _random_rotation(rng):
    """Uniform random rotation matrix from a normalised Gaussian quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


# The six {110} wave vectors of a one-mode BCC density field, |q| = 1.
BCC_Q = np.array([[1, 1, 0], [1, -1, 0], [1, 0, 1],
                  [1, 0, -1], [0, 1, 1], [0, 1, -1]], dtype=float) / math.sqrt(2)


def polycrystal_seeds(n: int, L: float | None = None, n_seeds: int = 6,
                      liquid: float = -0.25, noise: float = 0.01,
                      crystal_amp: float = 0.3, radius_cells: float = 10.0,
                      seed: int = DEFAULT_SEED):
    """Liquid phi = liquid + noise * N(0,1) with ``n_seeds`` spherical seeds
    (radius ``radius_cells`` * h, uniform random centres, periodic distance),
    each adding a one-mode BCC field crystal_amp * sum_q cos(q . R (r - c))
    with a random rotation R per seed.  Default L = n * pi / 4 (h = pi/4)."""
    if L is None:
        L = n * math.pi / 4.0
    h = L / n
    rng = np.random.default_rng(seed)
    phi = liquid + noise * rng.normal(size=(n, n, n))
    z, y, x = cell_centres(n, L)
    X = np.broadcast_to(x, (n, n, n))
    Y = np.broadcast_to(y, (n, n, n))
    Z = np.broadcast_to(z, (n, n, n))
    radius = radius_cells * h
    for _ in range(n_seeds):
        centre = rng.uniform(0.0, L, 3)
        R = _random_rotation(rng)
        # periodic displacement from the centre
        dx = (X - centre[0] + 0.5 * L) % L - 0.5 * L
        dy = (Y - centre[1] + 0.5 * L) % L - 0.5 * L
        dz = (Z - centre[2] + 0.5 * L) % L - 0.5 * L
        inside = dx * dx + dy * dy + dz * dz <= radius * radius
        qs = BCC_Q @ R.T
        field = sum(np.cos(q[0] * dx + q[1] * dy + q[2] * dz) for q in qs)
        phi = np.where(inside, phi + crystal_amp * field, phi)
    return np.ascontiguousarray(phi)


@dataclass(frozen=True)
class Workload:
    """One named workload: grid, model parameters, the initial field, and the
    mixed-path solver settings measured fastest for it on GB300 (every setting
    converges to the same tolerance; they differ only in cost)."""
    name: str
    n: int
    L: float
    eps: float
    dt: float
    steps: int
    tol: float
    mixed_settings: tuple = ()
    guess: str = "previous"
    fp64_settings: tuple = ()

    @property
    def h(self) -> float:
        return self.L / self.n

    def mixed(self) -> dict:
        """Keyword arguments of PFCSolver for the mixed path on this workload
        (the multigrid settings; the initial iterate stays the default)."""
        return dict(self.mixed_settings)

    def settings(self, precision: str = "mixed") -> dict:
        """Keyword arguments of PFCSolver for this workload's timed runs at a
        precision: the mixed settings, or on the FP64 FAS path its own
        measured ones, and the initial iterate of a step.  The double-float
        state has no three-field extrapolation and starts from phi^k."""
        kw = self.mixed() if precision != "fp64" else dict(self.fp64_settings)
        guess = self.guess
        if guess == "extrapolate_all" and precision == "mixed_df":
            guess = "previous"
        kw["guess"] = guess
        return kw

    def phi0(self, seed: int = DEFAULT_SEED):
        if self.name.startswith("random16"):
            return uniform_noise(self.n, 0.07, 0.07, seed)
        if self.name.startswith("smooth"):
            return smooth_mode(self.n, self.L)
        if self.name.startswith("polycrystal"):
            return polycrystal_seeds(self.n, self.L, seed=seed)
        if self.name.startswith("growth"):
            return uniform_01_start(self.n, seed=seed)
        if self.name.startswith("cosine"):
            return cosine_bump(self.n, self.L)
        raise KeyError(self.name)


def random16():
    """16^3, L = 32, eps = 0.025, phi0 = 0.07 + 0.07 U(-1,1), dt = 0.01,
    10 steps, tolerance 1e-10."""
    return Workload("random16", 16, 32.0, 0.025, 0.01, 10, 1e-10)


def smooth_sweep(n: int, dt: float = 0.0125, tol: float = 1e-9):
    """Smooth mode on L = 32, eps = 0.025, to T = 1 (steps = 1/dt).

    Mixed-path settings: at n >= 64 the finest level is stiff (red-black) and
    V(0,1) cycles are fastest, two per correction with 4 Jacobi sweeps per
    requested sweep on the intermediate levels; at 32^3 V(1,2).  Below 256^3
    the 16^3 coarsest level runs on an 8-CTA cluster (cluster_tail 2: 1464
    against 1425 steps/s at 128^3 when a step took two corrections; no
    change at 256^3).

    Timed runs start each step from u^{k+1} := 2 u^k - u^{k-1} in phi, mu and
    omega (guess extrapolate_all): the first defect falls from 2.3e-5 to
    2.6e-8 and a step takes one correction instead of two.  Whole runs to
    T = 1 (steps/s, corrections): 128^3 2510 at a Jacobi factor of 4 (2485 at
    2, 2390 at 5, and 1626 at 3, where every step takes two corrections);
    256^3 455 with two cycles per correction and a factor of 4 (461 at 2, 342
    at 3), against 321 with the five cycles and factor 3 that three
    corrections per step needed from phi^k."""
    if n >= 64:
        kw = (("nu1", 0), ("nu2", 1), ("inner_cycles", 2), ("jacobi_factor", 4),
              ("coarse_sweeps", 2)) + ((("cluster_tail", 2),) if n < 256 else ())
    else:
        kw = (("nu1", 1), ("nu2", 2), ("inner_cycles", 2), ("jacobi_factor", 3),
              ("coarse_sweeps", 2))
    # FP64 FAS: V(0,1) with a Jacobi factor of 2, the fastest of a measured
    # sweep of cycle shapes and factors from the extrapolated start (128^3 /
    # 256^3 steps/s: 514 / 81.8 with 2 cycles a step; V(1,1) factor 2 402 /
    # 64.0; the library's V(2,2) 165 / 29.8 with 3)
    fp64 = (("nu1", 0), ("nu2", 1), ("jacobi_factor", 2))
    return Workload(f"smooth{n}", n, 32.0, 0.025, dt, int(round(1.0 / dt)), tol, kw,
                    "extrapolate_all", fp64)


def polycrystal(n: int = 256, steps: int = 2000, tol: float = 1e-9):
    """Polycrystal growth: h = pi/4, eps = 0.25, dt = 0.1.

    Mixed-path settings: the finest level is in the damped-Jacobi regime, so
    V(1,2) with three cycles per correction; timed runs start from the
    three-field extrapolation (128^3, 200 steps: 3.07 corrections per step
    and 470 steps/s, against 4.0 and 372 from phi^k)."""
    kw = (("nu1", 1), ("nu2", 2), ("inner_cycles", 3), ("jacobi_factor", 3),
          ("coarse_sweeps", 2))
    return Workload(f"polycrystal{n}", n, n * math.pi / 4.0, 0.25, 0.1, steps, tol, kw,
                    "extrapolate_all")


def growth(n: int = 128, steps: int = 10000, tol: float = 1e-9):
    """Section 6.2 growth of a polycrystal: Omega = [0, 64]^3, eps = 0.25,
    dt = 0.01, phi0 = 0.2 + 0.005 U[0, 1] (the grid is not stated; n = 128
    gives h = 0.5).  Long runs of it are the energy/mass soak test.

    Mixed-path settings: the finest level is in the damped-Jacobi regime
    (108 tau/h^6 = 69 at h = 0.5), so V(1,2) with three cycles per
    correction; timed runs start from the three-field extrapolation (128^3,
    10^4 steps: 1.24 corrections per step and 1063 steps/s; two cycles 1.89
    and 978, though faster over the first 600 steps; from phi^k 2.6 and
    549)."""
    kw = (("nu1", 1), ("nu2", 2), ("inner_cycles", 3), ("jacobi_factor", 3),
          ("coarse_sweeps", 2))
    return Workload(f"growth{n}", n, 64.0, 0.25, 0.01, steps, tol, kw, "extrapolate_all")


def cosine_table(n: int, dt: float = 1e-3, steps: int = 10, tol: float = 1e-8):
    """Section 6.1 multigrid-complexity setting: [0, 3.2]^3, eps = 0.025."""
    return Workload(f"cosine{n}", n, 3.2, 0.025, dt, steps, tol)


def ensemble(count: int = 96, sizes=(32, 48, 64), L: float = 32.0, dt: float = 0.05,
             steps: int = 100, seed: int = DEFAULT_SEED):
    """Batched-ensemble workload: `count` independent runs with grids drawn
    from `sizes`, eps ~ U[0.02, 0.3], phi0 = m + 0.05 U(-1, 1) per cell with
    the mean m ~ U[-0.3, 0.1], dt = 0.05, `steps` steps, on a box of side L
    (the same for every size).  Returns {n: (eps list, phi0 array of shape
    (members, n, n, n))} grouped by grid size, members in draw order.

    Mixed-path settings (finest levels in the damped-Jacobi regime at
    dt = 0.05, 108 dt/h^6 = 5.4-346): V(1,2), three cycles per correction;
    timed runs start from the three-field extrapolation (ENSEMBLE_GUESS:
    2.52 corrections per step and group against 3.24 from phi^k)."""
    rng = np.random.default_rng(seed)
    picks = rng.choice(len(sizes), size=count)
    eps = rng.uniform(0.02, 0.3, count)
    means = rng.uniform(-0.3, 0.1, count)
    groups = {}
    for m in range(count):
        n = int(sizes[picks[m]])
        phi = means[m] + 0.05 * rng.uniform(-1.0, 1.0, (n, n, n))
        groups.setdefault(n, ([], []))
        groups[n][0].append(float(eps[m]))
        groups[n][1].append(phi)
    return {n: (e, np.ascontiguousarray(np.stack(f))) for n, (e, f) in sorted(groups.items())}


ENSEMBLE_SETTINGS = {"nu1": 1, "nu2": 2, "inner_cycles": 3, "jacobi_factor": 3,
                     "coarse_sweeps": 2}
# initial iterate of the ensemble workload's timed runs (9938 member-steps/s
# against 8679 from phi^k)
ENSEMBLE_GUESS = "extrapolate_all"
