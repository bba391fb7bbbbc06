"""Autotuner of the mixed-path cycle settings and the FP64 defect's tile.

The cost of a converged step depends on the cycle shape (pre/post sweeps),
the FP32 V-cycles per correction, the Jacobi sweeps per requested sweep on
the intermediate levels and the coarsest-level sweeps, and the best choice
differs between workloads (a stiff finest level favours V(0,1) cycles, a
finest level in the damped-Jacobi regime V(1,2)).  tune() times every
candidate on the caller's own problem (a single run or an ensemble) for a
few graph-launched steps after warm-up and returns the fastest one that
converged within the cycle budget; all candidates reach the same tolerance.

A second stage sizes the tile of the finest-level FP64 defect: its thread
blocks own 32 x 8 cells over a column of `defect_planes` planes, which sets
the grid (blocks per SM wave), the halo share (the first plane's neighbours
are loaded once per column) and the pipeline depth.  The tile changes the
rounding order of the residual norm only, not the iteration, so it is
timed on the best cycle settings alone rather than crossed with them.
"""

from __future__ import annotations

import itertools

import torch

from . import binding as B
from .solver import PFCBatch, PFCSolver

# (nu1, nu2) x inner cycles x Jacobi factor; two coarsest sweeps.  Then the
# defect's planes per block (0: the SM-count heuristic's choice).
DEFAULT_SPACE = {"nu": [(0, 1), (1, 1), (1, 2), (2, 2)], "inner_cycles": [2, 3, 5],
                 "jacobi_factor": [3, 4], "coarse_sweeps": [2],
                 "defect_planes": [0, 4, 8, 16, 32]}


def candidates(space=None):
    """Every combination of the cycle settings of the search space as a
    PFCSolver keyword dict (the first stage)."""
    space = space or DEFAULT_SPACE
    out = []
    for (nu1, nu2), inner, jf, cs in itertools.product(space["nu"], space["inner_cycles"],
                                                       space["jacobi_factor"],
                                                       space["coarse_sweeps"]):
        out.append({"nu1": nu1, "nu2": nu2, "inner_cycles": inner, "jacobi_factor": jf,
                    "coarse_sweeps": cs})
    return out


def tile_candidates(best, space=None):
    """The second stage: the best cycle settings with each defect tile depth
    of the space (none when the space has no "defect_planes" entry)."""
    space = space or DEFAULT_SPACE
    return [dict(best, defect_planes=int(z)) for z in space.get("defect_planes", [])]


def select(results):
    """The fastest candidate among those that converged: results is a list of
    (settings, ms_per_step or None when the candidate failed)."""
    ok = [(ms, i) for i, (_, ms) in enumerate(results) if ms is not None]
    if not ok:
        raise RuntimeError("no candidate setting converged")
    return results[min(ok)[1]][0]


def _time_steps(solver, steps):
    st = solver.stream
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(steps):
        solver.step(1)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / steps


def tune(n, L, eps, dt, phi0, tol=1e-9, steps=4, warmup=2, space=None, max_cycles=40,
         precision="mixed"):
    """Time each candidate on the problem (eps a number and phi0 one field, or
    eps a list and phi0 the ensemble's fields) and return (best settings,
    [(settings, ms per step or None), ...]) over both stages."""
    batch = not isinstance(eps, (int, float))

    def time_one(kw):
        try:
            if batch:
                s = PFCBatch(n, L, eps, dt, phi0, tol=tol, max_cycles=max_cycles,
                             precision=precision, **kw)
            else:
                s = PFCSolver(n, L, eps, dt, phi0, tol=tol, max_cycles=max_cycles,
                              precision=precision, **kw)
        except B.PFCError:
            return None
        try:
            for _ in range(warmup):
                s.step(1)
            return _time_steps(s, steps)
        except B.PFCError:
            return None
        finally:
            s.close()

    results = [(kw, time_one(kw)) for kw in candidates(space)]
    best = select(results)
    tiles = [(kw, time_one(kw)) for kw in tile_candidates(best, space)]
    results += tiles
    return (select(tiles) if tiles else best), results
