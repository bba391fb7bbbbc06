"""Ensembles (pfc_batch_*): independent runs of one grid size with their own
eps and initial fields advanced together.  Every member must match the
oracle run of that member alone, and the batch must match the same runs
made one at a time through pfc_init."""

import numpy as np
import pytest
import torch

from gpu_helpers import host, rel_l2
from oracle import pfc_oracle as O
from paper_1611_06288_gb300 import binding as B
from paper_1611_06288_gb300 import workloads as W
from paper_1611_06288_gb300.solver import PFCBatch, PFCSolver

pytestmark = pytest.mark.gpu

PARITY_RTOL = 1e-10


def members(n, count, seed):
    rng = np.random.default_rng(seed)
    eps = list(rng.uniform(0.02, 0.3, count))
    phi0 = np.stack([m + 0.05 * rng.uniform(-1, 1, (n, n, n))
                     for m in rng.uniform(-0.3, 0.1, count)])
    return eps, phi0


@pytest.mark.parametrize("graphs", [True, False])
def test_batch_matches_oracle(graphs):
    """Three 16^3 members, L = 32, dt = 0.05, 3 steps to 1e-12: each member's
    phi, mu and energies equal the oracle's run of that member."""
    n, L, dt = 16, 32.0, 0.05
    eps, phi0 = members(n, 3, 5)
    b = PFCBatch(n, L, eps, dt, phi0, tol=1e-12, max_cycles=80, **W.ENSEMBLE_SETTINGS)
    b.use_graphs(graphs)
    b.step(3)
    phi, mu = host(b.phi()), host(b.mu())
    its, res, _ = b.status()
    diag = b.diagnostics()
    for m in range(3):
        ref = O.run(phi0[m], 3, L / n, O.Params(eps=eps[m], tau=dt), tol=1e-12)
        assert res[m] <= 1e-12 and its[m] >= 1
        assert rel_l2(phi[m], ref[0]) <= PARITY_RTOL, m
        assert rel_l2(mu[m], ref[2]) <= PARITY_RTOL, m
        assert diag[m]["energy"] == pytest.approx(O.energy(ref[0], L / n, eps[m]), rel=1e-10)
        assert diag[m]["mass"] == pytest.approx(O.mass(phi0[m], L / n), rel=1e-12)
    b.close()


@pytest.mark.parametrize("n", [32, 48])
def test_batch_matches_single_runs(n):
    """Five members at 32^3 or 48^3 (levels 48, 24, 12): the batch equals the
    five runs made one at a time through pfc_init, step by step."""
    L, dt = 32.0, 0.05
    eps, phi0 = members(n, 5, n)
    kw = dict(tol=1e-11, max_cycles=80, **W.ENSEMBLE_SETTINGS)
    b = PFCBatch(n, L, eps, dt, phi0, **kw)
    singles = [PFCSolver(n, L, eps[m], dt, phi0[m], precision="mixed", **kw) for m in range(5)]
    for _ in range(4):
        b.step(1)
        for s in singles:
            s.step(1)
        got = host(b.phi())
        for m, s in enumerate(singles):
            assert rel_l2(got[m], host(s.phi())) <= PARITY_RTOL, m
    _, res, _ = b.status()
    assert max(res) <= 1e-11
    b.close()
    for s in singles:
        s.close()


@pytest.mark.parametrize("n", [64, 128])
def test_batch_without_presmoothing_matches_single_runs(n):
    """Two members on the V(0,1) settings of the smooth-mode workload, where
    the V-cycle's descent runs in one launch (64^3: 32^3 and 16^3 from the
    first restriction; 128^3: 64^3, 32^3, 16^3) and the prolongation skips
    the colour-0 children: the batch equals the members run alone."""
    L, dt = 32.0, 0.05
    eps, phi0 = members(n, 2, n + 1)
    kw = dict(tol=1e-11, max_cycles=80, nu1=0, nu2=1, inner_cycles=2, jacobi_factor=4,
              coarse_sweeps=2)
    b = PFCBatch(n, L, eps, dt, phi0, **kw)
    singles = [PFCSolver(n, L, eps[m], dt, phi0[m], precision="mixed", **kw) for m in range(2)]
    for _ in range(3):
        b.step(1)
        for s in singles:
            s.step(1)
        got = host(b.phi())
        for m, s in enumerate(singles):
            assert rel_l2(got[m], host(s.phi())) <= PARITY_RTOL, m
    _, res, _ = b.status()
    assert max(res) <= 1e-11
    b.close()
    for s in singles:
        s.close()


def test_batch_validation():
    eps, phi0 = members(16, 2, 1)
    with pytest.raises(B.PFCError):
        PFCBatch(16, 32.0, eps, 0.05, phi0, precision="fp64")
    with pytest.raises(B.PFCError):
        PFCBatch(16, 32.0, [0.1, 1.5], 0.05, phi0)          # eps >= 1
    with pytest.raises(ValueError):
        PFCBatch(16, 32.0, eps, 0.05, phi0[:1])


def test_autotune_picks_a_converging_setting():
    """The autotuner on a 32^3 ensemble returns one of its candidates, and a
    batch built with it converges."""
    from paper_1611_06288_gb300.autotune import tune
    eps, phi0 = members(32, 3, 7)
    space = {"nu": [(0, 1), (1, 2)], "inner_cycles": [2], "jacobi_factor": [3],
             "coarse_sweeps": [2], "defect_planes": [0, 8]}
    best, table = tune(32, 32.0, eps, 0.05, phi0, space=space, steps=2, warmup=1)
    assert best in [kw for kw, _ in table] and len(table) == 4
    assert best["defect_planes"] in (0, 8)
    b = PFCBatch(32, 32.0, eps, 0.05, phi0, tol=1e-9, **best)
    b.step(2)
    _, res, _ = b.status()
    assert max(res) <= 1e-9
    b.close()
