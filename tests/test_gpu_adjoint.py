"""Gradients through the time stepper (adjoint.rollout / pfc_adjoint_step):
against the oracle's FP64 adjoint (8^3, dense transposed solves) and against
central finite differences of the GPU forward solve (32^3, and the gradient
workload's 64^3 shape with checkpoints every 20 steps)."""

import numpy as np
import pytest
import torch

from gpu_helpers import host, rel_l2
from oracle import pfc_adjoint as A
from oracle import pfc_oracle as O
from paper_1611_06288_gb300.adjoint import rollout
from paper_1611_06288_gb300.solver import PFCSolver

pytestmark = pytest.mark.gpu


def loss_and_grads(phi0, eps, target, **kw):
    x = torch.tensor(phi0, dtype=torch.float64, device="cuda", requires_grad=True)
    e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
    h = kw["L"] / kw["n"]
    phiK = rollout(x, e, **kw)
    t = torch.as_tensor(target, dtype=torch.float64, device="cuda")
    loss = 0.5 * h ** 3 * ((phiK - t) ** 2).sum()
    loss.backward()
    return float(loss.detach()), host(x.grad), float(e.grad)


def test_adjoint_matches_oracle_adjoint():
    """8^3, L = 8, dt = 0.05, 4 steps with checkpoints every 2: dL/dphi0 and
    dL/deps equal the oracle's dense FP64 adjoint of the same trajectory.
    The agreement follows the solver tolerances: forward residual 1e-13 and
    adjoint residual 1e-12 of its initial value give about 6e-12 (measured on
    GB300; 5e-11 at 1e-12 / 1e-11), so the bound is 1e-10."""
    n, L, dt, steps = 8, 8.0, 0.05, 4
    h = L / n
    rng = np.random.default_rng(3)
    phi0 = 0.1 + 0.05 * rng.uniform(-1, 1, (n,) * 3)
    target = A.forward(0.1 + 0.05 * rng.uniform(-1, 1, (n,) * 3), steps, h,
                       O.Params(eps=0.1, tau=dt), 1e-13)[-1]
    eps = 0.15
    _, g0, geps = loss_and_grads(phi0, eps, target, n=n, L=L, dt=dt, steps=steps, every=2,
                                 tol=1e-13, adj_rtol=1e-12)
    prm = O.Params(eps=eps, tau=dt)
    phis = A.forward(phi0, steps, h, prm, 1e-14)
    r0, reps = A.adjoint(phis, h, prm, h ** 3 * (phis[-1] - target))
    assert rel_l2(g0, r0) <= 1e-10
    assert geps == pytest.approx(reps, rel=1e-10)


def test_adjoint_against_finite_differences():
    """32^3, L = 16, dt = 0.05, 40 steps, checkpoints every 10: dL/deps and a
    directional derivative of dL/dphi0 equal central differences (step 1e-6)
    of the forward solve converged to 1e-12."""
    n, L, dt, steps = 32, 16.0, 0.05, 40
    h = L / n
    rng = np.random.default_rng(8)
    phi0 = 0.1 + 0.05 * rng.uniform(-1, 1, (n,) * 3)
    kw = dict(precision="mixed", tol=1e-12, max_cycles=80, nu1=1, nu2=2, inner_cycles=3,
              jacobi_factor=3, coarse_sweeps=2)

    def forward(p0, eps):
        s = PFCSolver(n, L, eps, dt, p0, **kw)
        s.step(steps)
        out = host(s.phi())
        s.close()
        return out

    target = forward(0.1 + 0.05 * rng.uniform(-1, 1, (n,) * 3), 0.1)
    eps = 0.15

    def loss(p0, e):
        return 0.5 * h ** 3 * float(np.sum((forward(p0, e) - target) ** 2))

    _, g0, geps = loss_and_grads(phi0, eps, target, n=n, L=L, dt=dt, steps=steps, every=10,
                                 tol=1e-12, adj_rtol=1e-11)
    d = 1e-6
    fd = (loss(phi0, eps + d) - loss(phi0, eps - d)) / (2 * d)
    assert geps == pytest.approx(fd, rel=1e-4)
    v = rng.standard_normal((n,) * 3)
    fdv = (loss(phi0 + d * v, eps) - loss(phi0 - d * v, eps)) / (2 * d)
    assert float(np.sum(g0 * v)) == pytest.approx(fdv, rel=1e-4)


def test_gradient_workload_shape_against_finite_differences():
    """The gradient workload's shape at 40 of its 200 steps: 64^3, L = 32,
    dt = 0.05, forward checkpoints every 20 steps (two recomputed segments),
    target from a seeded run at eps = 0.1, gradient at eps = 0.15.  dL/deps
    and the derivative of L along a seeded random direction of phi0 equal
    central differences (step 1e-6) of the forward solve converged to 1e-12
    (measured on GB300: 2e-10 and 2e-9)."""
    from paper_1611_06288_gb300 import gradcheck as G
    r = G.run(64, steps=40, every=20)
    assert r["checkpoint_every"] == 20 and r["steps"] == 40
    assert r["rel_err_eps"] <= 1e-7, r
    assert r["rel_err_phi0"] <= 1e-7, r

