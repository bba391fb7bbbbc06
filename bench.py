#!/usr/bin/env python
"""Benchmark of the PFC time step (second-order convex splitting, FAS /
defect-correction multigrid) on GB300.

Workload: 128^3 cells, L = 32, eps = 0.025, phi0 = 0.1 sin(2 pi x/L)
cos(2 pi y/L) sin(2 pi z/L), dt = 0.0125, residual tolerance 1e-9 (RMS of the
three components).  A "step" is one full time step: source, multigrid
cycles until the residual is below the tolerance, and the energy/mass
diagnostics.  The headline value is the mixed-precision path (FP64 defect
correction around FP32 multigrid); the plain FP64 FAS path and the same
correction with a double-float outer loop are timed beside it.

Prints one JSON line (rank 0).  Under torchrun every rank advances its own
replica (no collective on the data path; weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "steps/s at 128^3 (mixed vs FP64 GPU, residual 1e-9); % HBM roof per V-cycle"
# arithmetic of each path: FP64 outer loop around FP32 multigrid, or the outer
# loop in double-float (FP32 pairs) around FP32 multigrid
DTYPES = {"mixed": "f64+f32", "mixed_df": "df32+f32", "fp64": "f64"}
UNIT = "steps/s"
WORKLOAD = {"workload": "smooth-mode 128^3", "n": 128, "L": 32.0, "eps": 0.025,
            "dt": 0.0125, "tol": 1e-9, "phi0": "0.1 sin(2pi x/L) cos(2pi y/L) sin(2pi z/L)"}

# Algorithmic bytes per cell of one counted launch, and launches per timed
# group, for each kernel class (minimum traffic: every field touched once).
KERNEL_BYTES = {
    "defect": (64.0, 2),          # read df phi,mu,om,b,S2,S3 (48) write r32 x3, q32 (16)
    "lin_smooth": (20.0, 1),      # per colour pass: half of read d (12) + r,q (16) + write d (12)
    "lin_restrict": (29.5, 1),    # read d,r,q (28) + write coarse r (12/8)
    "lin_prolong": (25.5, 1),     # read+write d (24) + coarse d (12/8)
    "correct": (60.0, 1),         # read df u (24) d (12) write df u (24); the mixed form below
    "smooth": (40.0, 1),          # per colour pass: half of (u 24 + S2,S3 16 + b 8 + phi 8 + write u 24)
    "residual_norm": (56.0, 2),   # read u, b, S2, S3 (48), write the Laplacian of phi (8)
    "residual_restrict": (57.0, 1),
    "prolong": (57.0, 2),
    "source": (32.0, 1),
    "restrict": (9.0, 1),
    "coarse_source": (80.0, 1),
    "coarse_solve": (0.0, 1),
    "lin_coarse": (0.0, 1),
    # pointwise start of a step from stored Laplacians, by initial iterate:
    "start": (104.0, 2),          # phi^k: read b, mu, om, 4 Laplacians (56) write S2, S3,
                                  # phi, a Laplacian (32), r32 x3, q32 (16)
}



# Classes whose kernel differs by precision: on the mixed path the correction
# u += d is folded into the last colour-1 pass of the correction's last
# V-cycle (reads colour-0 d 6, colour-1 r and q 8, u 24; writes u 24).
KERNEL_BYTES_BY_PRECISION = {("mixed", "correct"): (62.0, 1)}

# The start from u^{k+1} := 2 u^k - u^{k-1} (k_start64_extrap): reads b, c,
# mu^k, om^k, mu^{k-1}, om^{k-1} and six Laplacians (96); writes S2, S3, phi,
# mu, om and three Laplacians (64) and r32 x3, q32 (16).
START_BYTES = {"previous": 104.0, "extrapolate_all": 176.0}


# DRAM bytes (read + write) of one launch of a kernel class of a precision,
# from the ncu capture summarised in profiles/ (cold L2); absent where no
# capture of the current kernel exists.
# The defect class of the mixed path is the full defect (150.8 MB a launch);
# the start of a step has a class of its own.  Keyed by the finest level's
# size the capture ran at (other sizes: null).
NCU_TRAFFIC = {("mixed", "defect", 128): 150.8e6,   # profiles/k_defect64_fx_128.md
               # the start from the three-field extrapolation:
               ("mixed", "start", 128, "extrapolate_all"): 319.0e6}  # k_start64_extrap_128.md

# FP64-ALU-bound kernel classes of a precision: FP64 flops per cell of one
# counted launch (FMA = 2) and launches per group.  The full FP64 defect forms
# the three Laplacians' neighbour sums in exact int64 fixed point (no FP64
# flops) and its rows in 6 DFMA + 4 DADD + 2 DMUL per cell (ncu: DFMA, DADD
# and DMUL thread-instruction rates 3:2:1): 18 flops.
KERNEL_FLOPS = {("mixed", "defect"): (18.0, 2)}

# Algorithmic bytes per cell of the FP64 defect class (the ALU-bound class
# above), reported beside its FP64 roofline: a full defect reads phi, mu, om,
# b, S2, S3 and writes r(3), q FP32 and three Laplacians FP64 (88 B).
DEFECT_BYTES = 88.0

# FP64 peak of GB300: 2 FP64 FMA lanes per SM per clock (the peak of
# sm__sass_thread_inst_executed_op_dfma_pred_on is 304 per cycle for 152 SMs)
# x 2 flops x 152 SMs x 2.07 GHz.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    # mixed-path solver settings; default: the workload's measured-fastest ones
    ap.add_argument("--inner-cycles", type=int, default=None)
    ap.add_argument("--jacobi-factor", type=int, default=None)
    ap.add_argument("--nu1", type=int, default=None)
    ap.add_argument("--nu2", type=int, default=None)
    ap.add_argument("--coarse-sweeps", type=int, default=None)
    ap.add_argument("--cluster-tail", type=int, default=None)
    ap.add_argument("--guess", default=None,
                    choices=["previous", "extrapolate", "extrapolate_all"],
                    help="initial iterate of a step (default: the workload's, 2 u^k - u^{k-1} "
                         "in all three fields)")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-soak", action="store_true",
                    help="skip the 10^4-step growth soak of the extras (about 25 s)")
    ap.add_argument("--no-cpu-all-cores", action="store_true",
                    help="skip the all-cores oracle timing (one replica per host core)")
    ap.add_argument("--no-n256", dest="n256", action="store_false",
                    help="skip the 256^3 legs (the n256 object)")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the ensemble and gradient workloads")
    # the headline path: FP64 defect correction around FP32 multigrid; the
    # double-float form is timed beside it
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_df"])
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_replicas(local_seconds: float, steps: int, world_size: int, device=None):
    """Whole-job throughput of independent replicas: every rank advanced its
    own grid `steps` steps in `local_seconds`; the job time is the maximum
    over ranks (all_reduce MAX) and the value is all steps / that time."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    if world_size > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    t_max = float(t.item())
    return t_max, world_size * steps / t_max


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self, busy=None):
        """busy: called repeatedly (untimed GPU work) while nvidia-smi starts,
        so the GPU stays under load until its first sample."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return
        # nvidia-smi's start-up (driver and NVML initialisation) can hold the
        # driver for tens of milliseconds: let it finish before the timed
        # region begins (the first sample marks it), at most a few seconds
        t0 = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
            if busy is not None:
                busy()
            else:
                time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Algorithmic HBM bytes of one FP32 V-cycle of the mixed path that does not
# start from d = 0 (the second and later V-cycles of a defect correction):
# every field a kernel reads or writes counted once per pass (FP32, 4 B).
# Level 0: full residual restriction (d, r, q read, coarse r written:
# 28 + 12/8 B/cell), additive prolongation (d read and written, coarse d
# read: 24 + 12/8), post-smoothing; lower levels start from d = 0: the
# restriction reads only r (12 + 12/8) and the prolongation assigns d
# (12 + 12/8).  A red-black sweep is two colour passes of 20 B/cell (half
# of: d 12, r and q 16, d written 12); a damped Jacobi sweep reads d, r, q
# and writes t (40 B/cell), an odd count adds one copy back (24 B/cell).
# The coarse tail (from the first level of at most 16^3 cells) reads r and q
# and writes d of its top level (28 B/cell); its lower levels stay in
# shared memory.
# ---------------------------------------------------------------------------

def chained_levels(params, levels):
    """Levels whose zero-start restriction the one-launch descent takes over
    (k_lin_restrict_chain32: from the first level restricting to at most 64^3
    cells, n/2 a multiple of 16, up to two more levels above the tail): their
    r is averaged in shared memory and not read back."""
    if params.nu1 > 0:
        return set()
    for l, (m, _) in enumerate(levels):
        nc = m // 2
        if m > 16 and l + 1 < len(levels) and nc <= 64 and nc % 16 == 0:
            out = set()
            for j in range(l + 1, min(l + 3, len(levels) - 1)):
                if levels[j][0] <= 16:
                    break
                out.add(j)
            return out
    return set()


def vcycle_bytes(params, levels):
    """levels: [(n, kind)] of the mixed hierarchy, finest first."""
    from paper_1611_06288_gb300 import binding as B
    total = 0.0
    chained = chained_levels(params, levels)
    for l, (m, kind) in enumerate(levels):
        cells = float(m) ** 3
        if m <= 16:
            total += 28.0 * cells
            break
        first = l == 0
        rbytes = 28.0 if first else (0.0 if l in chained else 12.0)
        total += cells * (rbytes + 1.5)                                      # restriction
        # prolongation: d read and written (first level: the measured V-cycle
        # starts from d != 0) or written; before a red-black pass of colour 0
        # only the colour-1 half of d is touched
        dbytes = 24.0 if first else 12.0
        if kind != B.PFC_SWEEP_JACOBI and params.nu2 > 0:
            dbytes /= 2
        total += cells * (dbytes + 1.5)
        if kind == B.PFC_SWEEP_JACOBI:
            sweeps = params.nu2 * (params.jacobi_factor0 if first else params.jacobi_factor)
            total += cells * (40.0 * sweeps + (24.0 if sweeps % 2 else 0.0))
            if sweeps > 0 and m % 32 == 0:
                # the prolongation fused into the first sweep: d + P e stays
                # in shared memory (not written, not read back)
                total -= cells * 24.0
        else:
            total += cells * 40.0 * params.nu2
    return total


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def host_cpu() -> dict:
    """Logical cores and CPU model of the host the oracle runs on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    import platform
    # Arm cores report a part number only
    parts = {"0xd4f": "Arm Neoverse V2 (part 0xd4f)", "0xd40": "Arm Neoverse V1 (part 0xd40)",
             "0xd0c": "Arm Neoverse N1 (part 0xd0c)", "0xd49": "Arm Neoverse N2 (part 0xd49)"}
    model = parts.get(model, model)
    return {"nproc": os.cpu_count(), "model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


class OracleSteps:
    """The oracle (numpy FP64) on the bench workload: a first step by the
    start rule (phi^{-1} := phi^0), then warm steps from the previous step's
    solution, as the GPU's timed steps are.  numpy's elementwise kernels run
    on one thread, so the oracle uses one core."""

    def __init__(self, n: int):
        from oracle import pfc_oracle as O
        from paper_1611_06288_gb300 import workloads as W
        self.O = O
        self.wl = W.smooth_sweep(n, dt=WORKLOAD["dt"], tol=WORKLOAD["tol"])
        self.prm = O.Params(eps=self.wl.eps, tau=self.wl.dt)
        phi0 = self.wl.phi0()
        self.b, self.c = phi0, phi0
        self.mu, self.om = 0 * phi0, 0 * phi0
        self.k = 0

    def step(self):
        """One time step with the energy/mass diagnostics; returns (s, cycles)."""
        O, wl = self.O, self.wl
        t0 = time.perf_counter()
        res = O.solve_step(self.b, self.c, [self.b, self.mu, self.om], wl.h, self.prm, wl.tol)
        a, self.mu, self.om = res.u
        O.energy(a, wl.h, wl.eps)
        O.modified_energy(a, self.b, wl.h, wl.eps)
        O.mass(a, wl.h)
        dt = time.perf_counter() - t0
        self.c, self.b = self.b, a
        self.k += 1
        return dt, res.cycles


def _oracle_replica(n: int, barrier, results) -> None:
    """One oracle replica of the all-cores timing: its start step, then (all
    replicas together) one timed warm step."""
    orc = OracleSteps(n)
    orc.step()
    barrier.wait()
    t, cycles = orc.step()
    results.put((t, cycles))


def oracle_all_cores(n: int, procs: int):
    """The oracle on every host core: `procs` independent replicas of the
    bench workload in spawned processes (one numpy thread each), their warm
    steps started together; returns (aggregate steps/s, slowest step s,
    cycles).  numpy has no parallel elementwise kernels, so independent
    replicas are how the plain oracle uses all cores."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=(n, barrier, results)) for _ in range(procs)]
    for p in ps:
        p.start()
    out = [results.get(timeout=900) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    slowest = max(t for t, _ in out)
    return procs / slowest, slowest, [c for _, c in out]


def run_reference(args):
    """The oracle (numpy FP64, host cores) on the same workload and metric:
    one untimed start step, then warm steps timed one by one."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n = args.n
    # One oracle step is ~10 s at 128^3 on the GPU hosts: the bounded sample
    # of each bench step is one warm oracle time step.  As on the GPU, the
    # first `warmup` steps (the first by the start rule) are untimed and the
    # next ones timed; both counts are capped so the run ends within a few
    # minutes.
    warm = max(1, min(args.warmup, 5))
    steps = max(1, min(args.steps, 5))
    orc = OracleSteps(n)
    for _ in range(warm):
        orc.step()
    times, cycles = [], []
    for _ in range(steps):
        t, c = orc.step()
        times.append(t)
        cycles.append(c)
    tot = sum(times)
    value = steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * tot / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(WORKLOAD, workload=f"smooth-mode {n}^3", n=n,
                                            l2="inputs > L2 not applicable (CPU)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "host": host_cpu(),
                         "sample": f"oracle time steps {warm + 1}..{warm + steps} at {n}^3 "
                                   f"after {warm} untimed (warm: each from "
                                   f"the previous step's solution, as the GPU's timed steps), "
                                   f"FAS V(2,2) cycles {cycles}, energy/mass each step; numpy "
                                   f"elementwise on one thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

# FP64 FAS smoother: FP64 flops per updated cell of one launch (a red-black
# colour pass updates n^3/2 cells, a Jacobi sweep n^3): three neighbour sums
# (15 DADD), the source terms, the Newton coefficient and its cubic, and the
# 3x3 solve by elimination with one division (k_smooth_colour, Section 5).
FP64_SMOOTH_FLOPS = 66.0


def fp64_class_roofline(cls, m, red_black, launches, ms, hbm_gbs, hbm_source):
    """Roofline of an FP64 FAS kernel class from its event-timed launches at a
    level of m^3 cells (ms in total over `launches`): the red-black or Jacobi
    smoother in FP64 flops against the FP64 pipe, a class with a byte model
    in algorithmic bytes against the measured HBM peak, else no fraction."""
    if cls == "smooth":
        units = m ** 3 / (2 if red_black else 1)
        achieved = FP64_SMOOTH_FLOPS * units * launches / (ms / 1e3) / 1e12 if ms > 0 else 0.0
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "flops_per_updated_cell": FP64_SMOOTH_FLOPS,
                "peak_source": "FP64: 2 FMA lanes/SM/clock x 2 flops x 152 SMs x 2.07 GHz "
                               "(derived)"}
    per_cell, per_group = KERNEL_BYTES.get(cls, (0.0, 1))
    if per_cell > 0:
        groups = launches / per_group
        gbs = per_cell * m ** 3 * groups / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        return {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s",
                "frac": gbs / hbm_gbs, "algorithmic_bytes_per_cell": per_cell,
                "launches_per_pass": per_group, "ms_per_pass": ms / max(groups, 1e-30),
                "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({hbm_source})"}
    return {"bound": None, "note": "dominant class without a flop or byte model"}


def fp64_roofline(s, n, B, prof_steps=1):
    """Roofline of the dominant kernel class of the plain FP64 FAS path: one
    host-driven step with every class timed by CUDA events picks the class,
    then `prof_steps` steps time that class alone."""
    s.profile(None)
    s.step(1)
    prof = s.profile_read()
    (cls, lvl), _ = max(prof.items(), key=lambda kv: kv[1][1])
    s.profile([cls])
    for _ in range(prof_steps):
        s.step(1)
    launches, ms = B.pfc_profile_read(s.ctx, B.KERNEL_CLASSES.index(cls), lvl)
    s.profile([])
    m, _, kind = B.pfc_level_info(s.params, lvl)
    out = {"kernel": f"{cls} (level {lvl}, {m}^3)", "ms_per_launch": ms / max(launches, 1),
           "timing": f"CUDA events around each launch, {prof_steps} host-driven step(s)"}
    peaks, src = measured_peaks()
    out.update(fp64_class_roofline(cls, m, kind == B.PFC_SWEEP_RB, launches, ms,
                                   peaks["hbm_gbs"], src))
    out["kernel_profile_ms"] = {f"{k[0]}@{n >> k[1]}": round(v[1], 4)
                                for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])[:8]}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as tdist

    from paper_1611_06288_gb300 import binding as B
    from paper_1611_06288_gb300 import workloads as W
    from paper_1611_06288_gb300.solver import PFCSolver

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        tdist.init_process_group("nccl", device_id=dev)
    B.lib()  # fails loudly if libpfc.so is missing
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        if ws > 1:
            tdist.barrier()
        torch.cuda.synchronize(dev)

    def time_steps(s, k, diag=True):
        """k timed steps, L2 flushed (untimed) before each; returns total ms."""
        st = s.stream
        total = 0.0
        cycles = []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            stats = s.step(1)
            if diag:
                s.diagnostics()
            e1.record(st)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            cycles.append(stats.cycles_last)
        return total, cycles

    def measure(n, steps, warmup, fp64_steps, mixed_over=None, precision="mixed",
                other_leg=True):
        """Every GPU leg of one grid size; returns a dict of results."""
        # untimed steps before the secondary legs' timed ones: a context caches
        # one step graph per ring position (3) and, with the three-field
        # extrapolated start, per mu/omega slot (2); eight steps build them all
        # outside the timed region (the headline leg's clock sampler runs many
        # more untimed steps before its timed region)
        prime = max(warmup, 8)
        wl = W.smooth_sweep(n, dt=WORKLOAD["dt"], tol=WORKLOAD["tol"])
        phi0 = wl.phi0()
        mixed_kw = wl.settings(precision)
        mixed_kw.update(mixed_over or {})
        cells = n ** 3
        # ---- mixed path (headline) ----------------------------------------
        # every leg forms the energy/mass diagnostics of each new state inside
        # the step (step_diagnostics): the timed step includes them, with no
        # extra host round trip
        s = PFCSolver(n, wl.L, wl.eps, wl.dt, phi0, device=dev, tol=wl.tol,
                      step_diagnostics=True, precision=precision, **mixed_kw)
        # the W warm-up steps, and more until every step graph the timed
        # steps meet is built (see prime above)
        for _ in range(prime):
            s.step(1)
            s.diagnostics()
        # the clock sampler starts under load (more untimed steps until its
        # first sample), then every rank enters the timed region together
        clocks = ClockSampler(local)
        clocks.start(busy=lambda: (s.step(1), s.diagnostics()))
        barrier()
        # timed region: each step is one CUDA graph launch (device-side loop)
        launches0 = s.launches
        ms_total, cycles = time_steps(s, steps)
        launches = s.launches - launches0
        barrier()
        clk = clocks.stop()
        # kernel timing: the same steps driven from the host with every launch
        # of the dominant kernel class bracketed by CUDA events on the solver
        # stream
        s.profile(None)
        time_steps(s, 2)
        prof = s.profile_read()
        (dom_cls, dom_lvl), _ = max(prof.items(), key=lambda kv: kv[1][1])
        s.profile([dom_cls])
        prof_steps = max(2, min(steps, 10))
        ms_instr, _ = time_steps(s, prof_steps)
        dom_launches, dom_time = B.pfc_profile_read(s.ctx, B.KERNEL_CLASSES.index(dom_cls),
                                                    dom_lvl)
        s.profile([])
        s.close()
        t_max, value = aggregate_replicas(ms_total / 1e3, steps, ws, dev)

        # one FP32 V-cycle, graph-launched: the step time with one more
        # V-cycle per correction, at the same corrections per step, minus the
        # step time as configured, per correction (no events inside the graph)
        vcyc = None
        if precision == "mixed" and mixed_kw.get("nu1", 0) == 0:
            vk = max(10, min(steps, 40))
            res = {}
            for extra in (0, 1):
                kw = dict(mixed_kw, inner_cycles=mixed_kw.get("inner_cycles", 1) + extra)
                sv = PFCSolver(n, wl.L, wl.eps, wl.dt, phi0, device=dev, tol=wl.tol,
                               step_diagnostics=True, precision="mixed", **kw)
                for _ in range(prime):
                    sv.step(1)
                res[extra] = time_steps(sv, vk, diag=False)
                if extra == 0:
                    levels = []
                    for lv in range(24):
                        try:
                            m, _, kind = B.pfc_level_info(sv.params, lv)
                        except B.PFCError:
                            break
                        levels.append((m, kind))
                    vbytes = vcycle_bytes(sv.params, levels)
                sv.close()
            (t0_ms, c0), (t1_ms, c1) = res[0], res[1]
            if c0 == c1 and sum(c0) > 0:
                v_ms = (t1_ms - t0_ms) / sum(c0)
                peaks_v, src_v = measured_peaks()
                gbs = vbytes / (v_ms / 1e3) / 1e9
                vcyc = {"ms": v_ms, "algorithmic_bytes": vbytes, "achieved": gbs,
                        "unit": "GB/s", "peak": peaks_v["hbm_gbs"],
                        "frac": gbs / peaks_v["hbm_gbs"],
                        "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({src_v})",
                        "levels": [m for m, _ in levels],
                        "method": f"({vk} steps at inner_cycles+1 - {vk} steps as configured) / "
                                  f"{sum(c0)} corrections, graph-launched, L2 flushed per "
                                  f"step; a V-cycle that does not start from d = 0"}
            else:
                vcyc = {"ms": None, "reason": f"corrections differ: {c0} vs {c1}"}

        # roofline of the dominant kernel
        peaks, peak_src = measured_peaks()
        m = n >> dom_lvl
        if (precision, dom_cls) in KERNEL_FLOPS:
            per_cell, per_group = KERNEL_FLOPS[(precision, dom_cls)]
            groups = dom_launches / per_group
            achieved = per_cell * m ** 3 * groups / (dom_time / 1e3) / 1e12 \
                if dom_time > 0 else 0.0
            bound, peak, unit = "alu", FP64_PEAK_TFLOPS, "TFLOP/s"
            peak_src = "FP64: 2 FMA lanes/SM/clock x 2 flops x 152 SMs x 2.07 GHz (derived)"
        else:
            per_cell, per_group = KERNEL_BYTES_BY_PRECISION.get(
                (precision, dom_cls), KERNEL_BYTES.get(dom_cls, (0.0, 1)))
            if dom_cls == "start":
                per_cell = START_BYTES[mixed_kw.get("guess", "previous")]
            groups = dom_launches / per_group
            achieved = per_cell * m ** 3 * groups / (dom_time / 1e3) / 1e9 \
                if dom_time > 0 else 0.0
            bound, peak, unit = "hbm", peaks["hbm_gbs"], "GB/s"
            peak_src = f"hbm_gbs of MEASURED_PEAKS.json ({peak_src})"
        traffic = NCU_TRAFFIC.get((precision, dom_cls, m, mixed_kw.get("guess", "previous")),
                                  NCU_TRAFFIC.get((precision, dom_cls, m)))
        bytes_cell = KERNEL_BYTES.get(dom_cls, (None, 1))[0]
        roofline = {"bound": bound, "achieved": achieved, "peak": peak,
                    "unit": unit, "frac": achieved / peak,
                    "traffic": traffic / 1e9 if traffic is not None else None,
                    "traffic_unit": "GB per launch (ncu dram__bytes_read + write)",
                    "kernel": f"{dom_cls} (level {dom_lvl}, {m}^3)",
                    "ms_per_launch": dom_time / max(groups, 1),
                    "timing": f"CUDA events around each launch, {prof_steps} host-driven steps "
                              f"after the timed region ({1e3 * prof_steps / ms_instr:.1f} "
                              f"steps/s with the events)",
                    "peak_source": peak_src}
        if bound == "alu" and bytes_cell and dom_time > 0:
            gbs = DEFECT_BYTES * m ** 3 * groups / (dom_time / 1e3) / 1e9
            roofline["hbm"] = {"algorithmic_bytes_per_cell": DEFECT_BYTES, "achieved": gbs,
                               "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"]}

        # ---- plain FP64 FAS path, same workload, tolerance and initial
        # iterate (and from phi^k alone, for comparison) ---------------------
        guess = mixed_kw.get("guess", "previous")
        guess64 = guess
        fp64 = None
        for g in dict.fromkeys((guess64, "previous")):
            kw64 = dict(wl.settings("fp64"), guess=g)
            s64 = PFCSolver(n, wl.L, wl.eps, wl.dt, phi0, device=dev, tol=wl.tol,
                            precision="fp64", step_diagnostics=True, **kw64)
            for _ in range(prime):
                s64.step(1)
                s64.diagnostics()
            ms64, cyc64 = time_steps(s64, fp64_steps)
            if fp64 is None:
                fp64 = {"value": fp64_steps / (ms64 / 1e3), "unit": UNIT, "steps": fp64_steps,
                        "cycles_per_step": cyc64, "guess": g, "settings": kw64,
                        "solver": "FAS V-cycles with the workload's measured FP64 settings "
                                  "(the fastest of a sweep of cycle shapes and Jacobi "
                                  "factors), Newton pointwise smoother, full coarsening to 2^3"}
                fp64["roofline"] = fp64_roofline(s64, n, B)
            else:
                fp64["guess_previous"] = {"value": fp64_steps / (ms64 / 1e3), "unit": UNIT,
                                          "cycles_per_step": cyc64}
            s64.close()

        # ---- the headline path started from phi^k (mu, omega of step k) ----
        prev = None
        if guess != "previous":
            sp = PFCSolver(n, wl.L, wl.eps, wl.dt, phi0, device=dev, tol=wl.tol,
                           step_diagnostics=True, precision=precision,
                           **dict(mixed_kw, guess="previous"))
            for _ in range(prime):
                sp.step(1)
                sp.diagnostics()
            ms_p, cyc_p = time_steps(sp, steps)
            prev = {"value": steps / (ms_p / 1e3), "unit": UNIT, "steps": steps,
                    "ms_per_step": ms_p / steps, "cycles_per_step": cyc_p}
            sp.close()

        out = {"n": n, "wl": wl, "phi0": phi0, "mixed_kw": mixed_kw, "value": value,
               "t_max": t_max, "cycles": cycles, "launches": launches, "clocks": clk,
               "roofline": roofline, "vcycle": vcyc, "fp64": fp64, "guess_previous": prev,
               "kernel_profile_ms": {f"{k[0]}@{n >> k[1]}": round(v[1], 4)
                                     for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}}

        # ---- the other mixed form, same workload, tolerance and settings ---
        if other_leg:
            other = "mixed_df" if precision == "mixed" else "mixed"
            kw_o = dict(mixed_kw)
            if other == "mixed_df" and kw_o.get("guess") == "extrapolate_all":
                kw_o["guess"] = "previous"       # no three-field extrapolation there
            so = PFCSolver(n, wl.L, wl.eps, wl.dt, phi0, device=dev, tol=wl.tol,
                           precision=other, step_diagnostics=True, **kw_o)
            for _ in range(prime):
                so.step(1)
                so.diagnostics()
            ms_o, cyc_o = time_steps(so, steps)
            out["alt"] = {"precision": other, "dtype": DTYPES[other], "guess": kw_o["guess"],
                          "value": steps / (ms_o / 1e3), "unit": UNIT, "steps": steps,
                          "ms_per_step": ms_o / steps, "cycles_per_step": cyc_o}
            so.close()
        return out

    overrides = {k: getattr(args, k) for k in ("inner_cycles", "jacobi_factor", "nu1", "nu2",
                                                "coarse_sweeps", "guess", "cluster_tail")
                 if getattr(args, k) is not None}
    n = args.n
    r = measure(n, args.steps, args.warmup, args.fp64_steps, overrides, args.precision)
    wl, phi0, mixed_kw, value = r["wl"], r["phi0"], r["mixed_kw"], r["value"]
    cells = n ** 3

    # ---- end to end through the C ABI with host buffers -------------------
    pin_a = torch.from_numpy(phi0.copy()).pin_memory()
    pin_b = torch.from_numpy(phi0.copy()).pin_memory()
    pin_out = torch.empty_like(pin_a).pin_memory()
    se = PFCSolver(n, wl.L, wl.eps, wl.dt, phi0, device=dev, tol=wl.tol, step_diagnostics=True,
                   precision=args.precision, **mixed_kw)
    e2e_steps = max(1, min(args.steps, 10))

    bufs = [pin_a, pin_b, pin_out]               # phi^k, phi^{k-1}, phi^{k+1}: rotated

    def host_step():
        a, b, out = bufs
        B.pfc_set_state(se.ctx, a, b)             # H2D of phi^k, phi^{k-1}
        B.pfc_step(se.ctx, 1)
        B.pfc_get_phi(se.ctx, out)                # D2H of phi^{k+1}
        B.pfc_diagnostics(se.ctx)                 # D2H of the diagnostics (blocking)
        bufs[:] = [out, a, b]

    # two untimed steps: pfc_set_state restarts the ring, and the two mu/omega
    # slots of the extrapolated start alternate, so two step graphs are used
    host_step()
    host_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_step()
    e2e_t = time.perf_counter() - t0
    e2e = {"value": e2e_steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 2 * cells * 8,
           "d2h_bytes_per_step": cells * 8 + 6 * 8}
    se.close()

    # ---- 256^3: the second size of the target, its own legs and clocks ----
    n256 = None
    if args.n256 and n != 256:
        r2 = measure(256, max(3, min(args.steps, 10)), args.warmup, 2, None, args.precision,
                     other_leg=False)
        n256 = {"workload": "smooth-mode 256^3", "value": r2["value"], "unit": UNIT,
                "steps": max(3, min(args.steps, 10)), "ms_per_step": r2["t_max"] * 1e3 /
                max(3, min(args.steps, 10)), "solver": r2["mixed_kw"],
                "cycles_per_step": r2["cycles"], "dof_updates_per_s": r2["value"] * 256 ** 3,
                "fp64": r2["fp64"], "guess_previous": r2["guess_previous"],
                "mixed_over_fp64": r2["value"] / ws / r2["fp64"]["value"],
                "roofline": r2["roofline"], "vcycle": r2["vcycle"],
                "gpu_launches": r2["launches"], "clocks": r2["clocks"],
                "kernel_profile_ms": r2["kernel_profile_ms"]}

    # ---- the ensemble and gradient workloads (secondary lines) -------------
    extras = {}
    if args.extras:
        from paper_1611_06288_gb300 import ensemble as EN
        from paper_1611_06288_gb300 import gradcheck as GC
        ens = EN.run()
        extras["ensemble"] = {
            "workload": "96 independent runs, grids drawn from {32,48,64}^3, eps ~ U[0.02,0.3], "
                        "mean phi ~ U[-0.3,0.1] + 0.05 U(-1,1), dt = 0.05, 100 steps each, "
                        "tol 1e-9, one PFCGroup of three ensembles",
            "member_steps_per_s": ens["batched"]["member_steps_per_s"],
            "seconds": ens["batched"]["seconds"],
            "graph_launches_per_step": ens["batched"]["graph_launches_per_step"],
            "groups": ens["groups"],
            "corrections_per_step": {k: v["corrections_per_step"]
                                     for k, v in ens["batched"]["per_group"].items()},
            "max_final_residual": max(v["max_final_residual"]
                                      for v in ens["batched"]["per_group"].values())}
        extras["gradient"] = dict(GC.run(), workload="64^3, L = 32, dt = 0.05, 200 steps, "
                                  "checkpoints every 20, target from eps = 0.1, gradient at "
                                  "eps = 0.15, central differences with step 1e-6")
        if not args.no_soak:
            from paper_1611_06288_gb300 import soak as SK
            extras["soak"] = dict(
                SK.soak(n=128, steps=10000, workload="growth"),
                description="Section 6.2 polycrystal growth, Omega = [0,64]^3, eps = 0.25, "
                            "dt = 0.01, 10^4 steps (t = 100), diagnostics after every step: "
                            "largest relative mass drift and largest rise of the modified energy")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        orc = OracleSteps(n)
        _, cyc_start = orc.step()                  # start step: untimed
        t_cpu, cyc_cpu = orc.step()
        cpu = {"value": 1.0 / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "host": host_cpu(),
               "sample": f"oracle time step 2 at {n}^3 (warm: from step 1's solution, as the "
                         f"GPU's timed steps are), {cyc_cpu} FAS V(2,2) cycles to the same "
                         f"tolerance, energy/mass included (the untimed step 1, start rule, "
                         f"took {cyc_start}); numpy elementwise on one thread"}
        if not args.no_cpu_all_cores:
            procs = os.cpu_count() or 1
            agg, slowest, cyc_all = oracle_all_cores(n, procs)
            cpu["all_cores"] = {
                "value": agg, "unit": UNIT, "cores": procs, "kind": "oracle",
                "sample": f"{procs} independent replicas of the same workload, one per host "
                          f"core (spawned processes, one numpy thread each): each an untimed "
                          f"start step, then one warm step started together; value = replicas "
                          f"/ slowest warm step ({slowest:.2f} s, cycles {sorted(set(cyc_all))})"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["t_max"] * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": {"workload": f"smooth-mode {n}^3", "n": n, "L": wl.L, "eps": wl.eps,
                       "dt": wl.dt, "tol": wl.tol, "precision": args.precision,
                       "solver": mixed_kw, "step_execution": "CUDA graph",
                       "parallelism": f"replicas x{ws}",
                       "l2": "flushed (256 MiB write) before every timed step"},
            "cycles_per_step": r["cycles"],
            "dof_updates_per_s": value * cells,
            "fp64": r["fp64"],
            "guess_previous": r["guess_previous"],
            "mixed_over_fp64": value / ws / r["fp64"]["value"],
            ("mixed_df" if args.precision == "mixed" else "mixed_fp64_outer"): r.get("alt"),
            "roofline": r["roofline"],
            "vcycle": r["vcycle"],
            "e2e": e2e,
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
            "kernel_profile_ms": r["kernel_profile_ms"],
        }
        if n256 is not None:
            line["n256"] = n256
        line.update(extras)
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if ws > 1:
        tdist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
