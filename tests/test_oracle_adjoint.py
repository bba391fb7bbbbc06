"""Pins of the oracle's discrete adjoint (oracle/pfc_adjoint.py): the
gradients of L = 1/2 ||phi^K - target||_h^2 with respect to eps and phi^0
equal central finite differences of the oracle's own forward solve (converged
to 1e-13), on an 8^3 grid over 4 steps."""

import numpy as np
import pytest

from oracle import pfc_adjoint as A
from oracle import pfc_oracle as O

N, L, DT, STEPS = 8, 8.0, 0.05, 4
H = L / N
TOL = 1e-13


def setup():
    rng = np.random.default_rng(3)
    phi0 = 0.1 + 0.05 * rng.uniform(-1, 1, (N,) * 3)
    tgt0 = 0.1 + 0.05 * rng.uniform(-1, 1, (N,) * 3)
    target = A.forward(tgt0, STEPS, H, O.Params(eps=0.1, tau=DT), TOL)[-1]
    return phi0, target


def loss_at(phi0, eps, target):
    return A.loss(A.forward(phi0, STEPS, H, O.Params(eps=eps, tau=DT), TOL)[-1], target, H)


def gradients(phi0, eps, target):
    prm = O.Params(eps=eps, tau=DT)
    phis = A.forward(phi0, STEPS, H, prm, TOL)
    return A.adjoint(phis, H, prm, H ** 3 * (phis[-1] - target))


def test_adjoint_eps_against_finite_differences():
    phi0, target = setup()
    eps, d = 0.15, 1e-6
    _, geps = gradients(phi0, eps, target)
    fd = (loss_at(phi0, eps + d, target) - loss_at(phi0, eps - d, target)) / (2 * d)
    assert geps == pytest.approx(fd, rel=1e-5)
    assert abs(geps) > 1e-8


def test_adjoint_phi0_against_finite_differences():
    phi0, target = setup()
    eps, d = 0.15, 1e-6
    g0, _ = gradients(phi0, eps, target)
    rng = np.random.default_rng(9)
    for _ in range(2):
        v = rng.standard_normal(phi0.shape)
        fd = (loss_at(phi0 + d * v, eps, target) - loss_at(phi0 - d * v, eps, target)) / (2 * d)
        assert float(np.sum(g0 * v)) == pytest.approx(fd, rel=1e-5)


def test_adjoint_linear_case_closed_form():
    """Without the cubic term the step is linear and diagonal in the DFT
    (pfc_oracle.linear_step_fft): the adjoint of one step applied to a single
    Fourier mode is that mode times the step's amplification factor, so
    dL/dphi^0 for L = <g, phi^1> equals (transfer of g) computed with the
    transposed (= same, symmetric) Fourier multipliers."""
    prm = O.Params(eps=0.2, tau=DT, cubic=False)
    rng = np.random.default_rng(4)
    phi0 = rng.standard_normal((N,) * 3)
    g = rng.standard_normal((N,) * 3)
    phis = A.forward(phi0, 1, H, prm, TOL)
    g0, _ = A.adjoint(phis, H, prm, g)
    # L(phi0) = <g, phi^1(phi0)> is linear in phi0: its gradient applied to
    # any v is <g, phi^1(v)>, the step being linear with c = b = phi0
    v = rng.standard_normal((N,) * 3)
    a_v = O.linear_step_fft(v, v, H, 0.2, DT)
    assert float(np.sum(g0 * v)) == pytest.approx(float(np.sum(g * a_v)), rel=1e-9)
