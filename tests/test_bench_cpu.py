"""bench.py's host-side legs run without a GPU: the reference arm (the
oracle on the host cores) prints its JSON line, and the cpu_baseline leg's
oracle step timer works on a small grid."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "8",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "steps/s"
    assert line["config"]["workload"] == "smooth-mode 8^3"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == 1 and "warm" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_step_timer():
    """The cpu_baseline leg: a start step, then a warm step from its solution
    (the work of the GPU's timed steps), each converged to the tolerance."""
    sys.path.insert(0, ROOT)
    import bench
    orc = bench.OracleSteps(8)
    t0, c0 = orc.step()
    t1, c1 = orc.step()
    assert t0 > 0 and t1 > 0 and c0 >= 1 and c1 >= 1 and orc.k == 2
    host = bench.host_cpu()
    assert host["nproc"] >= 1 and host["model"]


def test_vcycle_byte_model_matches_the_kernel_counts():
    """The V-cycle byte model of bench.py against the per-kernel algorithmic
    bytes of opbench at 128^3 with the smooth-mode settings (V(0,1), red-black
    finest level, Jacobi factor 4 below): finest level = restriction (d != 0)
    + prolongation with the colour-0 half skipped + one red-black sweep."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1611_06288_gb300 import binding as B
    from paper_1611_06288_gb300 import opbench as OB
    p = B.pfc_default_params()
    p.nu1, p.nu2, p.jacobi_factor, p.jacobi_factor0 = 0, 1, 4, 4
    n = 128
    finest = bench.vcycle_bytes(p, [(n, B.PFC_SWEEP_RB)])
    assert finest == OB.algorithmic_bytes("lin_restrict", n) + \
        OB.algorithmic_bytes("lin_prolong_skip0", n) + OB.algorithmic_bytes("lin_smooth", n)
    # a Jacobi level: zero-start restriction, the assigning prolongation
    # fused into the first of four sweeps, three plain sweeps
    jac = [(n, B.PFC_SWEEP_RB), (64, B.PFC_SWEEP_JACOBI), (32, B.PFC_SWEEP_JACOBI),
           (16, B.PFC_SWEEP_JACOBI)]
    assert bench.vcycle_bytes(p, jac[:2]) - finest == \
        OB.algorithmic_bytes("lin_restrict_zero", 64) + \
        OB.algorithmic_bytes("lin_prolong_jacobi_assign", 64) + \
        3 * OB.algorithmic_bytes("lin_jacobi", 64)
    # a level the fused kernel's tiles do not cover (48^3): separate launches
    odd = [(96, B.PFC_SWEEP_RB), (48, B.PFC_SWEEP_JACOBI), (24, B.PFC_SWEEP_JACOBI)]
    assert bench.vcycle_bytes(p, odd[:2]) - bench.vcycle_bytes(p, odd[:1]) == \
        OB.algorithmic_bytes("lin_restrict_zero", 48) + \
        OB.algorithmic_bytes("lin_prolong_assign", 48) + 4 * OB.algorithmic_bytes("lin_jacobi", 48)
    # without pre-smoothing the 64^3 and 32^3 levels' averages come from the
    # first restriction's launch: only their 1.5 B per cell of output count
    assert bench.chained_levels(p, jac) == {1, 2}
    full = bench.vcycle_bytes(p, jac)
    p.nu1 = 1
    assert bench.chained_levels(p, jac) == set()
    assert bench.vcycle_bytes(p, jac) - full == 12.0 * (64 ** 3 + 32 ** 3)
    # 256^3: the descent starts one level lower (128^3 -> 64^3, 32^3, 16^3)
    p.nu1 = 0
    big = [(256, B.PFC_SWEEP_RB)] + jac
    assert bench.chained_levels(p, big) == {2, 3}


def test_oracle_all_cores_timing_runs_spawned_replicas():
    """The all-cores CPU baseline: independent oracle replicas in spawned
    processes, warm steps started together (two replicas at 8^3 here)."""
    sys.path.insert(0, ROOT)
    import bench
    agg, slowest, cycles = bench.oracle_all_cores(8, 2)
    assert slowest > 0 and agg == pytest.approx(2 / slowest)
    assert len(cycles) == 2 and all(c >= 1 for c in cycles)


def test_workload_settings_by_precision():
    """The timed runs of the smooth sweep start from the three-field
    extrapolation on the FP64 and mixed paths; the double-float state, which
    has none, starts from phi^k; the FP64 path takes its own cycle settings,
    not the mixed ones."""
    from paper_1611_06288_gb300 import workloads as W
    wl = W.smooth_sweep(128)
    assert wl.settings("mixed") == dict(wl.mixed(), guess="extrapolate_all")
    assert wl.settings("fp64") == {"nu1": 0, "nu2": 1, "jacobi_factor": 2,
                                   "guess": "extrapolate_all"}
    assert wl.settings("mixed_df")["guess"] == "previous"
    assert "guess" not in wl.mixed()
    assert W.growth(32).settings("mixed")["guess"] == "extrapolate_all"
    assert W.cosine_table(16).settings("mixed")["guess"] == "previous"


def test_fp64_class_roofline():
    """The FP64 arm's kernel-class fractions: the smoother in flops against the
    FP64 pipe (half the cells per red-black pass), the residual norm (kernel
    and reduction: two launches a pass) in bytes against HBM."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.fp64_class_roofline("smooth", 128, True, 4, 1.0, 6781.8, "measured")
    flops = bench.FP64_SMOOTH_FLOPS * 128 ** 3 / 2 * 4 / 1e-3 / 1e12
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(flops)
    assert r["frac"] == pytest.approx(flops / bench.FP64_PEAK_TFLOPS)
    r = bench.fp64_class_roofline("residual_norm", 128, True, 2, 0.072, 6781.8, "measured")
    gbs = 56.0 * 128 ** 3 / 0.072e-3 / 1e9
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(gbs)
    assert r["frac"] == pytest.approx(gbs / 6781.8) and r["ms_per_pass"] == pytest.approx(0.072)
    assert bench.fp64_class_roofline("coarse_solve", 2, False, 1, 0.01, 1.0, "")["bound"] is None
