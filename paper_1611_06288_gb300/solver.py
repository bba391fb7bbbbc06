"""User-facing wrapper of the libpfc solver context.

PyTorch provides the device memory (the caller-owned workspace and the
fields) and the stream; every computation runs in libpfc's CUDA kernels.
"""

from __future__ import annotations

import numpy as np
import torch

from . import binding as B

_PREC = {"fp64": B.PFC_FP64, "mixed": B.PFC_MIXED, "mixed_df": B.PFC_MIXED_DF}
_LIN = {"newton": B.PFC_NEWTON, "picard": B.PFC_PICARD}


def make_params(n, L, eps, dt, tol=1e-9, nu1=2, nu2=2, max_cycles=50,
                precision="fp64", smoother="newton", coarsest=2,
                inner_cycles=1, policy="hybrid", jacobi_weight=0.7, jacobi_factor=4,
                jacobi_factor0=2, stiff_hi=1000.0, stiff_lo=0.25,
                coarse_stiffness=0.05, coarse_sweeps=4,
                guess="previous", mobility=(1.0, 0.0), cluster_tail=False,
                step_diagnostics=False, defect_planes=0) -> B.pfc_params:
    p = B.pfc_default_params()
    p.n, p.L, p.eps, p.dt = int(n), float(L), float(eps), float(dt)
    p.tol, p.nu1, p.nu2, p.max_cycles = float(tol), int(nu1), int(nu2), int(max_cycles)
    p.precision = _PREC[precision]
    p.smoother = _LIN[smoother]
    p.coarsest = int(coarsest)
    p.inner_cycles = int(inner_cycles)
    p.policy = {"hybrid": B.PFC_POLICY_HYBRID, "rb": B.PFC_POLICY_RB}[policy]
    p.jacobi_weight = float(jacobi_weight)
    p.jacobi_factor = int(jacobi_factor)
    p.jacobi_factor0 = int(jacobi_factor0)
    p.stiff_hi, p.stiff_lo = float(stiff_hi), float(stiff_lo)
    p.coarse_stiffness = float(coarse_stiffness)
    p.coarse_sweeps = int(coarse_sweeps)
    p.guess = {"previous": B.PFC_GUESS_PREVIOUS, "extrapolate": B.PFC_GUESS_EXTRAPOLATE,
               "extrapolate_all": B.PFC_GUESS_EXTRAPOLATE_ALL}[guess]
    p.mobility_m0, p.mobility_m2 = float(mobility[0]), float(mobility[1])
    p.cluster_tail = int(cluster_tail)
    p.step_diagnostics = 1 if step_diagnostics else 0
    p.defect_planes = int(defect_planes)
    return p


def as_field(x, n, device) -> torch.Tensor:
    """float64 contiguous (n, n, n) tensor on `device` (host copy if needed)."""
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    x = x.to(device=device, dtype=torch.float64).contiguous()
    if tuple(x.shape) != (n, n, n):
        raise ValueError(f"field must have shape {(n, n, n)}, got {tuple(x.shape)}")
    return x


class PFCSolver:
    """Time stepper for Eq. 1.10 on an n^3 periodic grid.

    phi0 (and optionally phi1) may be numpy arrays or tensors; they are copied
    into the caller-owned workspace held by this object.
    """

    def __init__(self, n, L, eps, dt, phi0, phi1=None, device="cuda", stream=None,
                 **solver_kw):
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise RuntimeError("PFCSolver runs on a CUDA device only")
        self.n, self.L, self.eps, self.dt = int(n), float(L), float(eps), float(dt)
        self.h = self.L / self.n
        self.params = make_params(n, L, eps, dt, **solver_kw)
        nbytes = B.pfc_workspace_bytes(self.params)
        if nbytes == 0:
            raise B.PFCError(B.PFC_ESIZE, "pfc_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p0 = as_field(phi0, self.n, self.device)
        p1 = as_field(phi1, self.n, self.device) if phi1 is not None else None
        with torch.cuda.stream(self.stream):
            self.ctx = B.pfc_init(self.params, self.workspace, p0, p1, self.stream.cuda_stream)
        self.stream.synchronize()
        self.last_stats = None

    def step(self, nsteps: int = 1) -> B.pfc_step_stats:
        self.last_stats = B.pfc_step(self.ctx, nsteps)
        return self.last_stats

    def _field(self, getter) -> torch.Tensor:
        out = torch.empty((self.n,) * 3, dtype=torch.float64, device=self.device)
        getter(self.ctx, out)
        self.stream.synchronize()
        return out

    def phi(self) -> torch.Tensor:
        return self._field(B.pfc_get_phi)

    def mu(self) -> torch.Tensor:
        return self._field(B.pfc_get_mu)

    def omega(self) -> torch.Tensor:
        return self._field(B.pfc_get_omega)

    def set_state(self, phi, phi_prev=None) -> None:
        a = as_field(phi, self.n, self.device)
        b = as_field(phi_prev, self.n, self.device) if phi_prev is not None else None
        B.pfc_set_state(self.ctx, a, b)
        self.stream.synchronize()

    def energy(self) -> tuple[float, float]:
        return B.pfc_energy(self.ctx)

    def mass(self) -> float:
        return B.pfc_mass(self.ctx)

    def diagnostics(self) -> dict:
        F, Fm, m, g = B.pfc_diagnostics(self.ctx)
        return {"energy": F, "modified_energy": Fm, "mass": m, "grad_sq": g}

    def profile(self, classes=None) -> None:
        """Time the given kernel classes (names of binding.KERNEL_CLASSES; None
        = all, [] = off) with CUDA events inside pfc_step."""
        if classes is None:
            mask = (1 << len(B.KERNEL_CLASSES)) - 1
        else:
            mask = 0
            for c in classes:
                mask |= 1 << B.KERNEL_CLASSES.index(c)
        B.pfc_profile_enable(self.ctx, mask)

    def profile_read(self) -> dict:
        """{(class, level): (launches, ms)} for every nonzero entry."""
        out = {}
        for ci, name in enumerate(B.KERNEL_CLASSES):
            for lvl in range(B.PROFILE_LEVELS):
                n, ms = B.pfc_profile_read(self.ctx, ci, lvl)
                if n:
                    out[(name, lvl)] = (n, ms)
        return out

    def use_graphs(self, on: bool = True) -> None:
        """Run each step as one CUDA graph launch (default) or host-driven."""
        B.pfc_use_graphs(self.ctx, on)

    @property
    def launches(self) -> int:
        return B.pfc_launch_count(self.ctx)

    @property
    def step_index(self) -> int:
        return B.pfc_step_index(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None) is not None:
            B.pfc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PFCBatch:
    """An ensemble of independent runs of one grid size, box and time step,
    each with its own eps and initial field, advanced together (PFC_MIXED:
    every kernel launch covers all members).

    phi0: array or tensor of shape (members, n, n, n).
    """

    def __init__(self, n, L, eps, dt, phi0, device="cuda", stream=None, **solver_kw):
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise RuntimeError("PFCBatch runs on a CUDA device only")
        self.eps = [float(e) for e in eps]
        self.members = len(self.eps)
        self.n, self.L, self.dt = int(n), float(L), float(dt)
        solver_kw.setdefault("precision", "mixed")
        self.params = make_params(n, L, self.eps[0], dt, **solver_kw)
        nbytes = B.pfc_batch_workspace_bytes(self.params, self.members)
        if nbytes == 0:
            raise B.PFCError(B.PFC_EINVAL, "pfc_batch_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if isinstance(phi0, np.ndarray):
            phi0 = torch.from_numpy(np.ascontiguousarray(phi0, dtype=np.float64))
        p0 = phi0.to(device=self.device, dtype=torch.float64).contiguous()
        if tuple(p0.shape) != (self.members, self.n, self.n, self.n):
            raise ValueError(f"phi0 must have shape {(self.members,) + (self.n,) * 3}")
        with torch.cuda.stream(self.stream):
            self.ctx = B.pfc_batch_init(self.params, self.eps, self.workspace, p0,
                                        self.stream.cuda_stream)
        self.stream.synchronize()

    def step(self, nsteps: int = 1) -> B.pfc_step_stats:
        return B.pfc_step(self.ctx, nsteps)

    def _field(self, getter) -> torch.Tensor:
        out = torch.empty((self.members,) + (self.n,) * 3, dtype=torch.float64,
                          device=self.device)
        getter(self.ctx, out)
        self.stream.synchronize()
        return out

    def phi(self) -> torch.Tensor:
        return self._field(B.pfc_get_phi)

    def mu(self) -> torch.Tensor:
        return self._field(B.pfc_get_mu)

    def omega(self) -> torch.Tensor:
        return self._field(B.pfc_get_omega)

    def diagnostics(self) -> list[dict]:
        return [{"energy": F, "modified_energy": Fm, "mass": m, "grad_sq": g}
                for F, Fm, m, g in B.pfc_batch_diagnostics(self.ctx, self.members)]

    def status(self):
        """(corrections, final RMS residual, initial RMS residual) per member
        of the last step."""
        return B.pfc_batch_status(self.ctx, self.members)

    def use_graphs(self, on: bool = True) -> None:
        B.pfc_use_graphs(self.ctx, on)

    def close(self) -> None:
        if getattr(self, "ctx", None) is not None:
            B.pfc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PFCGroup:
    """Ensembles of different grid sizes (PFCBatch or PFCSolver objects)
    advanced together: one CUDA graph launch per time step runs every
    context's step side by side under one device-side convergence loop.
    The group does not own the contexts; close it before them."""

    def __init__(self, contexts, stream=None):
        self.contexts = list(contexts)
        if not self.contexts:
            raise ValueError("a group needs at least one context")
        dev = self.contexts[0].device
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.g = B.pfc_group_init([c.ctx for c in self.contexts], self.stream.cuda_stream)

    def step(self, nsteps: int = 1) -> list:
        """One pfc_step_stats per context."""
        return B.pfc_group_step(self.g, len(self.contexts), nsteps)

    @property
    def graph_launches(self) -> int:
        return B.pfc_group_graph_launches(self.g)

    def close(self) -> None:
        if getattr(self, "g", None) is not None:
            B.pfc_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
