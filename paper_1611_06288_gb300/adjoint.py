"""Gradients through the PFC time stepper: a torch.autograd.Function whose
backward is the discrete adjoint of the scheme (pfc_adjoint_step), with the
forward trajectory recomputed segment by segment from checkpoints.

    phiK = rollout(phi0, eps, n=64, L=32.0, dt=0.05, steps=200, every=20)
    loss = 0.5 * h**3 * ((phiK - target)**2).sum()
    loss.backward()          # phi0.grad, eps.grad

Step k solves F(u; phi^k, phi^{k-1}, eps) = N(u; phi^k) - S(phi^k, phi^{k-1})
= 0 (Eqs. 5.4-5.10) for u = (phi^{k+1}, mu, omega); its adjoint solves
J^T psi = (dL/dphi^{k+1}, 0, 0) at the step's solution and passes
-(dF/dphi^k)^T psi, -(dF/dphi^{k-1})^T psi and -(dF/deps)^T psi back (the
formulas are in include/pfc.h).  Every kernel runs in libpfc; this module
only orders the steps and holds the checkpoints.
"""

from __future__ import annotations

import torch

from . import binding as B
from .solver import PFCSolver


class _Rollout(torch.autograd.Function):

    @staticmethod
    def forward(ctx, phi0, eps, cfg):
        n, steps, every = cfg["n"], cfg["steps"], cfg["every"]
        s = PFCSolver(n, cfg["L"], float(eps), cfg["dt"], phi0.detach(), precision="mixed",
                      tol=cfg["tol"], max_cycles=cfg["max_cycles"], **cfg["settings"])
        cur = phi0.detach().to(torch.float64).clone()
        prev = cur
        checkpoints = {0: (cur, prev)}
        for k in range(steps):
            s.step(1)
            prev, cur = cur, s.phi()
            if (k + 1) % every == 0 and k + 1 < steps:
                checkpoints[k + 1] = (cur, prev)
        ctx.solver = s
        ctx.cfg = cfg
        ctx.checkpoints = checkpoints
        ctx.eps = float(eps)
        return cur.clone()

    @staticmethod
    def backward(ctx, gK):
        cfg, s = ctx.cfg, ctx.solver
        n, steps, every = cfg["n"], cfg["steps"], cfg["every"]
        dev = gK.device
        z = torch.empty(3 * n ** 3, dtype=torch.float64, device=dev)
        gn = gK.detach().to(torch.float64).contiguous().clone()       # dL/dphi^{k+1}
        gc = torch.zeros_like(gn)                                        # dL/dphi^k (partial)
        eps_bar = 0.0
        cycles = 0
        starts = sorted(ctx.checkpoints)
        for j0 in reversed(starts):
            j1 = min(j0 + every, steps)
            # recompute phi^{j0} .. phi^{j1} from the checkpoint pair
            cur, prev = ctx.checkpoints[j0]
            if j0 == 0:
                s.set_state(cur)
            else:
                s.set_state(cur, prev)
            phis = [cur]
            for _ in range(j1 - j0):
                s.step(1)
                phis.append(s.phi())
            for k in range(j1 - 1, j0 - 1, -1):
                gp = gc if k == 0 else torch.zeros_like(gn)             # dL/dphi^{k-1}
                e, cyc = B.pfc_adjoint_step(s.ctx, phis[k + 1 - j0], phis[k - j0], gn, gc, gp, z,
                                            cfg["adj_rtol"], cfg["max_cycles"])
                eps_bar += e
                cycles += cyc
                gn, gc = gc, gp
        s.close()
        ctx.adjoint_cycles = cycles
        # after step 0 the complete dL/dphi^0 sits in gn
        g0 = gn.to(gK.dtype)
        geps = torch.tensor(eps_bar, dtype=torch.float64, device=dev)
        return g0, geps, None


def rollout(phi0, eps, n, L, dt, steps, every=20, tol=1e-11, adj_rtol=1e-10, max_cycles=60,
            settings=None):
    """phi^K after `steps` steps of the scheme from phi^0 (start rule phi^{-1}
    := phi^0), differentiable in phi0 (an (n, n, n) float64 CUDA tensor) and
    eps (a 0-d float64 tensor)."""
    cfg = {"n": int(n), "L": float(L), "dt": float(dt), "steps": int(steps),
           "every": int(every), "tol": float(tol), "adj_rtol": float(adj_rtol),
           "max_cycles": int(max_cycles),
           "settings": dict(settings or {"nu1": 1, "nu2": 2, "inner_cycles": 3,
                                         "jacobi_factor": 3, "coarse_sweeps": 2})}
    return _Rollout.apply(phi0, eps, cfg)
