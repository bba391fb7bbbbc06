"""Batched ensemble run (the ensemble workload: independent runs with grids
drawn from {32^3, 48^3, 64^3}, their own eps and initial fields, dt = 0.05,
100 steps each): one PFCBatch per grid size, all of them advanced together by
one PFCGroup (one CUDA graph launch per time step for every run), against the
same runs made one after another through single contexts.

    python -m paper_1611_06288_gb300.ensemble [--count 96] [--steps 100] [--sequential]
                                              [--autotune] [--cluster-tail]

Prints one JSON line: member-steps per second batched (and sequential when
asked), the corrections per step and the largest final residual per group.
"""

from __future__ import annotations

import argparse
import json

import torch

from . import workloads as W
from . import binding as B
from .solver import PFCBatch, PFCGroup, PFCSolver


def _timed(fn):
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    out = fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / 1e3, out


def run(count=96, steps=100, sequential=False, L=32.0, dt=0.05, tol=1e-9, warmup=2,
        autotune=False, cluster_tail=False):
    groups = W.ensemble(count, L=L, dt=dt, steps=steps)
    kw = dict(W.ENSEMBLE_SETTINGS, tol=tol, max_cycles=100, cluster_tail=cluster_tail,
              guess=W.ENSEMBLE_GUESS)
    tuned = {}
    if autotune:
        from .autotune import tune
        for n, (eps, phi0) in groups.items():
            tuned[n], _ = tune(n, L, eps, dt, phi0, tol=tol)
    out = {"count": count, "steps": steps, "L": L, "dt": dt, "tol": tol,
           "cluster_tail": bool(cluster_tail),
           "groups": {n: len(e) for n, (e, _) in groups.items()},
           "settings": dict(W.ENSEMBLE_SETTINGS, guess=W.ENSEMBLE_GUESS)}
    batches = {}
    for n, (eps, phi0) in groups.items():
        gkw = dict(kw, **tuned.get(n, {}))
        batches[n] = (PFCBatch(n, L, eps, dt, phi0, **gkw),
                      torch.as_tensor(phi0, dtype=torch.float64, device="cuda").contiguous())
    grp = PFCGroup([b for b, _ in batches.values()])

    def restart():
        for b, p0 in batches.values():
            B.pfc_set_state(b.ctx, p0)
        torch.cuda.synchronize()

    # warm-up: every step graph the timed run meets (a first step at each of
    # the three ring positions, then warm steps at each) is built here
    for _ in range(3):
        grp.step(1)
        restart()
    grp.step(max(3, warmup))
    restart()
    # the extrapolated start alternates two mu, omega slots over the three
    # ring positions: twelve steps meet every variant, and an even count
    # leaves the slots as the timed run finds them
    grp.step(12)
    restart()
    launches0 = grp.graph_launches

    def go():
        cyc = [0] * len(batches)
        for _ in range(steps):
            for i, st in enumerate(grp.step(1)):
                cyc[i] += st.cycles_last
        return cyc

    total, cyc = _timed(go)
    per_group = {}
    for (n, (b, _)), c in zip(batches.items(), cyc):
        _, res, _ = b.status()
        per_group[n] = {"members": b.members, "corrections_per_step": c / steps,
                        "max_final_residual": max(res),
                        "settings": tuned.get(n, W.ENSEMBLE_SETTINGS)}
    out["batched"] = {"member_steps_per_s": count * steps / total, "seconds": total,
                      "graph_launches_per_step": (grp.graph_launches - launches0) / steps,
                      "per_group": per_group}
    grp.close()
    for b, _ in batches.values():
        b.close()
    if sequential:
        tot = 0.0
        for n, (eps, phi0) in groups.items():
            for m in range(len(eps)):
                s = PFCSolver(n, L, eps[m], dt, phi0[m], precision="mixed", **kw)
                s.step(warmup)
                s.set_state(phi0[m])
                t, _ = _timed(lambda: s.step(steps))
                tot += t
                s.close()
        out["sequential"] = {"member_steps_per_s": count * steps / tot, "seconds": tot}
        out["batched_over_sequential"] = out["batched"]["member_steps_per_s"] / (
            out["sequential"]["member_steps_per_s"])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=96)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--sequential", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="choose each group's cycle settings with autotune.tune first")
    ap.add_argument("--cluster-tail", action="store_true",
                    help="coarse levels in one thread-block-cluster launch (cluster_tail 1)")
    a = ap.parse_args()
    print(json.dumps(run(a.count, a.steps, a.sequential, autotune=a.autotune,
                         cluster_tail=a.cluster_tail)), flush=True)


if __name__ == "__main__":
    main()
