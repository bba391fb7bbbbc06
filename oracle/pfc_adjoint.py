"""CPU FP64 oracle of the discrete adjoint of the PFC time stepper.

TEST INFRASTRUCTURE ONLY (like ``pfc_oracle``): only ``tests/`` may import it.
It imports ``pfc_oracle`` for the forward scheme and nothing from the CUDA
package.

Each step k of the scheme (Eq. 1.10 in the split form of Section 5) solves
F(u; b, c, eps) = N(u; b) - S(b, c) = 0 for u = (phi^{k+1}, mu, omega), with
b = phi^k, c = phi^{k-1} (c = b at the first step).  For a loss L(phi^K) the
gradient follows from the implicit function theorem, one step at a time from
the last:

    J^T psi = (dL/dphi^{k+1}, 0, 0),          J = dF/du at the solution
    dL/dphi^k     += -(dF/db)^T psi
    dL/dphi^{k-1} += -(dF/dc)^T psi
    dL/deps       += -(dF/deps)^T psi

with, from Eqs. 5.4-5.10 (q = f'(phi) + (1-eps)/2, f(a) = (a+b)(a^2+b^2)/4,
Lap the 7-point Laplacian, symmetric):

    J     = [[I, -tau Lap, 0], [-diag(q), I, -Lap], [-Lap/2, 0, I]]
    dF/db = [-I; -diag(df/db) - (1-eps)/2 I - 3 Lap; -Lap/2],  df/db = (a^2 + 2ab + 3b^2)/4
    dF/dc = [0; Lap; 0]
    dF/deps = [0; (phi + b)/2; 0]

The transposed systems are solved with the dense Jacobian (small grids).
"""

import numpy as np

from . import pfc_oracle as O


def dfdb(a, b):
    """d f / d b for f(a, b) = (a+b)(a^2+b^2)/4 of Eq. 5.2."""
    return 0.25 * (a * a + 2.0 * a * b + 3.0 * b * b)


def forward(phi0, steps, h, prm: O.Params, tol):
    """phi^0 .. phi^K of ``steps`` steps from phi^0 (start rule phi^{-1} := phi^0)."""
    phis = [phi0.copy()]

    def cb(k, a, b, c, mu, om, res):
        phis.append(a.copy())

    O.run(phi0, steps, h, prm, tol=tol, callback=cb)
    return phis


def loss(phiK, target, h):
    """L = 1/2 ||phi^K - target||_h^2 = h^3/2 sum (phi^K - target)^2."""
    return 0.5 * h ** 3 * float(np.sum((phiK - target) ** 2))


def adjoint(phis, h, prm: O.Params, gK):
    """Reverse pass over the trajectory phis = [phi^0 .. phi^K] for the loss
    gradient gK = dL/dphi^K: returns (dL/dphi^0, dL/deps)."""
    m = phis[0].shape[0]
    L = O.laplacian_matrix(m, h)
    K = len(phis) - 1
    g = [np.zeros_like(phis[0]) for _ in range(K + 1)]
    g[K] = gK.copy()
    geps = 0.0
    c1 = 0.5 * (1.0 - prm.eps)
    n = m ** 3
    for k in range(K - 1, -1, -1):
        a = phis[k + 1]
        b = phis[k]
        J = O.jacobian_dense([a, None, None], b, h, prm, L=L)
        ubar = np.concatenate([g[k + 1].ravel(), np.zeros(2 * n)])
        psi = np.linalg.solve(J.T, ubar)
        p1, p2, p3 = psi[:n], psi[n:2 * n], psi[2 * n:]
        dfb = dfdb(a, b).ravel() if prm.cubic else 0.0
        gb = p1 + (dfb + c1) * p2 + 3.0 * (L @ p2) + 0.5 * (L @ p3)
        gc = -(L @ p2)
        g[k] += gb.reshape(b.shape)
        if k >= 1:
            g[k - 1] += gc.reshape(b.shape)
        else:
            g[0] += gc.reshape(b.shape)       # start rule: phi^{-1} = phi^0
        geps += -float(np.dot(p2, 0.5 * (a + b).ravel()))
    return g[0], geps
