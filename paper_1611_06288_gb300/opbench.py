"""Per-kernel timing of the FP32 multigrid kernels through the op entry points.

    python -m paper_1611_06288_gb300.opbench [--n 256] [--reps 20] [--ops a,b,...]

Each op runs on seeded random colour-split FP32 fields of n^3 cells held on
the device (inputs larger than L2 from n = 192 on), `reps` times after two
warm-up calls, timed with CUDA events on the stream the kernels run on.  One
JSON line per op: microseconds per call and the achieved bandwidth for the
op's algorithmic bytes (each field read or written once per call):

  lin_restrict       r - J d restricted: reads d, r (3 fields each) and q,
                     writes 3 coarse fields: 29.5 B per fine cell
  lin_restrict_zero  d = 0: reads r only: 13.5 B per fine cell
  lin_smooth         one red-black sweep (two colour passes), each reading
                     the other colour's d and its own r, q and writing its own
                     d: 40 B per cell
  lin_prolong        d += P e: d read and written: 24 B per fine cell (+ the
                     coarse e); the _skip0 forms touch the colour-1 half only
                     (12 B), the _assign forms write d only (12 B, 6 B)
  lin_jacobi         one damped Jacobi sweep d -> t: reads d, r (3 fields
                     each) and q, writes t: 40 B per cell
  lin_prolong_jacobi the prolongation fused into the first Jacobi sweep
                     (pfc_op_lin_prolong_smooth): reads d_old, r and q and the
                     coarse e, writes t (d + P e stays in shared memory):
                     40 B per fine cell (+ e); _assign: d_old not read, 28 B

A tool for measuring kernels in isolation (and for capturing one of them
under a profiler); the solver itself never calls it.
"""

from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import binding as B

EPS, TAU, L = 0.025, 0.0125, 32.0

OPS = ("lin_restrict", "lin_restrict_zero", "lin_smooth", "lin_prolong", "lin_prolong_skip0",
       "lin_prolong_assign", "lin_prolong_assign_skip0")


def algorithmic_bytes(op: str, n: int) -> float:
    cells = float(n) ** 3
    coarse = 3 * 4.0 / 8                       # three coarse fields per fine cell
    per_cell = {"lin_restrict": 28.0 + coarse, "lin_restrict_zero": 12.0 + coarse,
                "lin_smooth": 40.0, "lin_prolong": 24.0 + coarse,
                "lin_prolong_skip0": 12.0 + coarse, "lin_prolong_assign": 12.0 + coarse,
                "lin_prolong_assign_skip0": 6.0 + coarse, "lin_jacobi": 40.0,
                "lin_prolong_jacobi": 40.0 + coarse,
                "lin_prolong_jacobi_assign": 28.0 + coarse}[op]
    return per_cell * cells


def make_fields(n: int, dev, seed: int = 0):
    g = torch.Generator(device=dev).manual_seed(seed)

    def field(cells, scale=1.0, shift=0.0):
        return torch.rand(cells, generator=g, device=dev, dtype=torch.float32) * scale + shift

    cells, ccells = n ** 3, (n // 2) ** 3
    f = {"d": [field(cells, 0.2, -0.1) for _ in range(3)],
         "r": [field(cells, 2e-3, -1e-3) for _ in range(3)],
         "q": field(cells, 0.5, -0.3),
         "c": [torch.empty(ccells, device=dev, dtype=torch.float32) for _ in range(3)],
         "e": [field(ccells, 0.2, -0.1) for _ in range(3)]}
    return f


def run_op(op: str, n: int, f) -> None:
    h = L / n
    if op.startswith("lin_restrict"):
        B.pfc_op_lin_residual_restrict(n, h, EPS, TAU, op.endswith("zero"), *f["d"], *f["r"],
                                       f["q"], *f["c"])
    elif op == "lin_smooth":
        B.pfc_op_lin_smooth(n, h, EPS, TAU, 1, False, *f["d"], *f["r"], f["q"])
    else:
        flags = (B.PFC_PROLONG_ASSIGN if "assign" in op else 0) | \
                (B.PFC_PROLONG_SKIP_COLOUR0 if op.endswith("skip0") else 0)
        B.pfc_op_lin_prolong(n, flags, *f["e"], *f["d"])


def time_op(op: str, n: int, reps: int, f) -> float:
    for _ in range(2):
        run_op(op, n, f)
    st = torch.cuda.current_stream()           # the ops run on the default stream
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(reps):
        run_op(op, n, f)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) * 1e3 / reps


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--ops", default=",".join(OPS))
    a = ap.parse_args(argv)
    if a.n % 4 or a.n < 8:
        raise SystemExit("n must be a multiple of 4 and >= 8")
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    dev = torch.device("cuda:0")
    f = make_fields(a.n, dev)
    peak = None
    try:
        import os
        with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                               "MEASURED_PEAKS.json")) as fh:
            peak = float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        pass
    for op in a.ops.split(","):
        if op not in OPS:
            raise SystemExit(f"unknown op {op}; one of {', '.join(OPS)}")
        us = time_op(op, a.n, a.reps, f)
        gbs = algorithmic_bytes(op, a.n) / (us * 1e-6) / 1e9
        print(json.dumps({"op": op, "n": a.n, "us": round(us, 2),
                          "algorithmic_bytes": algorithmic_bytes(op, a.n),
                          "GB/s": round(gbs, 1),
                          "frac_of_measured_hbm": None if peak is None else round(gbs / peak, 3)}),
              flush=True)
    assert np.isfinite(f["d"][0][:16].cpu().numpy()).all()


if __name__ == "__main__":
    main()
