"""Long-run check of the discrete invariants on the Section 6.2 polycrystal
growth (the soak test): every step, the mass h^3 sum(phi) must stay at its
initial value and the modified energy
    F~(phi^{k+1}, phi^k) = F_h(phi^{k+1}) + 1/2 ||grad_h(phi^{k+1} - phi^k)||^2
must not increase (Prop. 3.1; by the identity of Eq. 1.10 with Lemma 2.1 it
falls by tau ||grad_h mu||^2 + 1/2 ||grad_h(phi^{k+1} - 2 phi^k + phi^{k-1})||^2).

    python -m paper_1611_06288_gb300.soak [--n 128] [--steps 10000] [--precision mixed]
                                          [--workload growth|polycrystal]

(--workload polycrystal: the seeded 256^3 polycrystal of six BCC grains,
h = pi/4, eps = 0.25, dt = 0.1.)

Prints one JSON line: steps, steps/s, corrections per step, the largest
relative mass drift, the largest energy increase relative to |F~|, and F~ at
the start and the end.
"""

from __future__ import annotations

import argparse
import json
import time

import torch

from . import workloads as W
from .solver import PFCSolver


def soak(n=128, steps=10000, precision="mixed", every=1, device="cuda", workload="growth"):
    wl = W.growth(n, steps) if workload == "growth" else W.polycrystal(n, steps)
    kw = wl.settings(precision)
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), device=device, tol=wl.tol,
                  step_diagnostics=every == 1,
                  precision=precision, max_cycles=100, **kw)
    try:
        d = s.diagnostics()
        Fm0, m0 = d["modified_energy"], d["mass"]
        prev = Fm0
        worst_mass = 0.0
        worst_rise = 0.0
        cycles = 0
        t0 = time.perf_counter()
        for k in range(steps):
            st = s.step(1)
            cycles += st.cycles_last
            if (k + 1) % every == 0 or k + 1 == steps:
                d = s.diagnostics()
                Fm, m = d["modified_energy"], d["mass"]
                worst_mass = max(worst_mass, abs(m - m0) / abs(m0))
                worst_rise = max(worst_rise, (Fm - prev) / max(abs(prev), 1e-300))
                prev = Fm
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"workload": wl.name, "n": n, "steps": steps, "precision": precision,
                "settings": kw, "steps_per_s": steps / dt,
                "corrections_per_step": cycles / steps, "max_rel_mass_drift": worst_mass,
                "max_rel_energy_rise": worst_rise, "F_modified_start": Fm0,
                "F_modified_end": prev, "check_every": every}
    finally:
        s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "mixed_df"])
    ap.add_argument("--every", type=int, default=1)
    ap.add_argument("--workload", default="growth", choices=["growth", "polycrystal"])
    a = ap.parse_args()
    print(json.dumps(soak(a.n, a.steps, a.precision, a.every, workload=a.workload)), flush=True)


if __name__ == "__main__":
    main()
