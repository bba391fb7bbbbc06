"""Groups of ensembles of different grid sizes (pfc_group_*): one CUDA graph
launch per time step advances every context under one device-side loop.
Every member must match the oracle run of that member alone, and the group
must match its ensembles stepped on their own."""

import numpy as np
import pytest

from gpu_helpers import host, rel_l2
from oracle import pfc_oracle as O
from paper_1611_06288_gb300 import binding as B
from paper_1611_06288_gb300 import workloads as W
from paper_1611_06288_gb300.solver import PFCBatch, PFCGroup, PFCSolver

pytestmark = pytest.mark.gpu

PARITY_RTOL = 1e-10
L, DT = 32.0, 0.05


def members(n, count, seed):
    rng = np.random.default_rng(seed)
    eps = list(rng.uniform(0.02, 0.3, count))
    phi0 = np.stack([m + 0.05 * rng.uniform(-1, 1, (n, n, n))
                     for m in rng.uniform(-0.3, 0.1, count)])
    return eps, phi0


@pytest.mark.parametrize("graphs", [True, False])
def test_group_of_two_sizes_matches_oracle(graphs):
    """Two 16^3 and two 24^3 members (levels 16, 8 and 24, 12), their own eps,
    3 steps to 1e-12 in one group: each member's phi and mu equal the
    oracle's run of that member; one graph launch per group step (none when
    the contexts are host-driven: they are then stepped one after another)."""
    steps = 3
    spec = {16: members(16, 2, 3), 24: members(24, 2, 4)}
    batches = [PFCBatch(n, L, eps, DT, phi0, tol=1e-12, max_cycles=80, **W.ENSEMBLE_SETTINGS)
               for n, (eps, phi0) in spec.items()]
    for b in batches:
        b.use_graphs(graphs)
    g = PFCGroup(batches)
    stats = g.step(steps)
    assert g.graph_launches == (steps if graphs else 0)
    for b, st, (n, (eps, phi0)) in zip(batches, stats, spec.items()):
        assert st.steps == steps and st.residual <= 1e-12
        phi, mu = host(b.phi()), host(b.mu())
        its, res, _ = b.status()
        for m in range(len(eps)):
            ref = O.run(phi0[m], steps, L / n, O.Params(eps=eps[m], tau=DT), tol=1e-12)
            assert res[m] <= 1e-12 and its[m] >= 1
            assert rel_l2(phi[m], ref[0]) <= PARITY_RTOL, (n, m)
            assert rel_l2(mu[m], ref[2]) <= PARITY_RTOL, (n, m)
    g.close()
    for b in batches:
        b.close()


def test_group_matches_its_ensembles_alone():
    """32^3 (3 members) and 48^3 (2 members, levels 48, 24, 12) to 1e-11:
    4 group steps equal 4 steps of each ensemble on its own, bit for bit,
    with the same corrections per step (a context whose members have all
    converged takes no further loop body while the other runs)."""
    kw = dict(tol=1e-11, max_cycles=80, **W.ENSEMBLE_SETTINGS)
    spec = {32: members(32, 3, 32), 48: members(48, 2, 48)}
    grouped = [PFCBatch(n, L, eps, DT, phi0, **kw) for n, (eps, phi0) in spec.items()]
    alone = [PFCBatch(n, L, eps, DT, phi0, **kw) for n, (eps, phi0) in spec.items()]
    g = PFCGroup(grouped)
    for _ in range(4):
        gst = g.step(1)
        for b, st in zip(alone, gst):
            assert b.step(1).cycles_last == st.cycles_last
    assert g.graph_launches == 4
    for a, b in zip(grouped, alone):
        assert B.pfc_step_index(a.ctx) == B.pfc_step_index(b.ctx) == 4
        assert np.array_equal(host(a.phi()), host(b.phi()))
        assert np.array_equal(host(a.mu()), host(b.mu()))
        _, res, _ = a.status()
        assert max(res) <= 1e-11
        assert a.diagnostics() == b.diagnostics()
    g.close()
    for b in grouped + alone:
        b.close()


def test_group_with_extrapolated_guesses_matches_alone():
    """Ensembles whose steps start from 2 u^k - u^{k-1} (guess
    extrapolate_all; the graph of a step depends on which mu, omega slot it
    writes): 5 group steps equal 5 steps of each ensemble alone, bit for
    bit, and the members match the oracle."""
    kw = dict(tol=1e-12, max_cycles=80, guess="extrapolate_all", **W.ENSEMBLE_SETTINGS)
    spec = {16: members(16, 2, 5), 24: members(24, 2, 6)}
    grouped = [PFCBatch(n, L, eps, DT, phi0, **kw) for n, (eps, phi0) in spec.items()]
    alone = [PFCBatch(n, L, eps, DT, phi0, **kw) for n, (eps, phi0) in spec.items()]
    g = PFCGroup(grouped)
    for _ in range(5):
        gst = g.step(1)
        for b, st in zip(alone, gst):
            assert b.step(1).cycles_last == st.cycles_last
    for a, b, (n, (eps, phi0)) in zip(grouped, alone, spec.items()):
        assert np.array_equal(host(a.phi()), host(b.phi()))
        assert np.array_equal(host(a.mu()), host(b.mu()))
        phi = host(a.phi())
        for m in range(len(eps)):
            ref = O.run(phi0[m], 5, L / n, O.Params(eps=eps[m], tau=DT), tol=1e-12)
            assert rel_l2(phi[m], ref[0]) <= PARITY_RTOL, (n, m)
    g.close()
    for b in grouped + alone:
        b.close()


def test_group_of_a_single_run_and_an_ensemble():
    """A pfc_init context (16^3, random start) grouped with a 24^3 ensemble:
    the single run equals its oracle run."""
    wl = W.random16()
    phi0 = wl.phi0()
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=1e-12, precision="mixed",
                  **W.ENSEMBLE_SETTINGS)
    eps, p24 = members(24, 2, 9)
    b = PFCBatch(24, L, eps, DT, p24, tol=1e-12, max_cycles=80, **W.ENSEMBLE_SETTINGS)
    g = PFCGroup([s, b])
    g.step(2)
    ref, *_ = O.run(phi0, 2, wl.h, O.Params(eps=wl.eps, tau=wl.dt), tol=1e-12)
    assert rel_l2(s.phi().cpu().numpy(), ref) <= PARITY_RTOL
    g.close()
    s.close()
    b.close()


def test_group_failure_keeps_the_converged_contexts_step():
    """One context cannot converge within its cycle budget (max_cycles 3 at
    an unreachable tol 1e-20) while the other converges in fewer: the group
    step reports PFC_ENOCONV, the context that converged has taken its step,
    the failing one has not."""
    e1, p1 = members(16, 2, 11)
    e2, p2 = members(16, 1, 12)
    good = PFCBatch(16, L, e1, DT, p1, tol=1e-9, max_cycles=80, **W.ENSEMBLE_SETTINGS)
    bad = PFCBatch(16, L, e2, DT, p2, tol=1e-20, max_cycles=3, **W.ENSEMBLE_SETTINGS)
    g = PFCGroup([good, bad])
    with pytest.raises(B.PFCError) as err:
        g.step(1)
    assert err.value.code == B.PFC_ENOCONV
    assert B.pfc_step_index(good.ctx) == 1
    assert B.pfc_step_index(bad.ctx) == 0
    g.close()
    good.close()
    bad.close()
