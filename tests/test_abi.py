"""The C ABI library builds, loads and exports every entry point declared in
include/pfc.h; host-only entry points behave as documented (no GPU needed, no
compute call is made)."""

import ctypes
import os
import re

import pytest

from paper_1611_06288_gb300 import binding as B
from paper_1611_06288_gb300 import build as BLD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpfc():
    BLD.build()
    return B.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pfc_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(libpfc):
    names = declared_symbols()
    assert "pfc_init" in names and "pfc_step" in names
    missing = [n for n in names if not hasattr(libpfc, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    assert set(declared_symbols()) == set(B._SIGS), (
        set(declared_symbols()) ^ set(B._SIGS))


def test_default_params_and_workspace(libpfc):
    p = B.pfc_default_params()
    assert (p.nu1, p.nu2, p.smoother, p.precision, p.coarsest) == (2, 2, 0, 0, 2)
    assert B.pfc_workspace_bytes(p) == 0          # n, L, dt unset -> invalid
    p.n, p.L, p.eps, p.dt = 16, 32.0, 0.025, 0.01
    n16 = B.pfc_workspace_bytes(p)
    # 13 fine FP64 fields (3 levels of phi and their 3 Laplacians, mu, omega,
    # S2, S3, 3 Jacobi scratch) + 13 per coarse level (8, 4, 2) + reduction
    # buffers
    fields = 13 * 16 ** 3 + 13 * (8 ** 3 + 4 ** 3 + 2 ** 3)
    assert fields * 8 <= n16 <= fields * 8 + 100_000
    p.precision = B.PFC_MIXED
    assert B.pfc_workspace_bytes(p) > n16
    p.n = 6                                   # 6 -> 3: odd coarsest level
    assert B.pfc_workspace_bytes(p) == 0
    p.n, p.coarsest = 12, 6                   # 12 -> 6: accepted
    assert B.pfc_workspace_bytes(p) > 0


def test_level_policy(libpfc):
    """Level sizes and the hybrid smoother choice (host-side): red-black where
    108 tau/h^6 >= 1000 or <= 0.25, damped Jacobi in between."""
    p = B.pfc_default_params()
    p.n, p.L, p.eps, p.dt = 128, 32.0, 0.025, 0.0125
    p.precision = B.PFC_MIXED
    info = []
    lvl = 0
    while True:
        try:
            info.append(B.pfc_level_info(p, lvl))
        except B.PFCError:
            break
        lvl += 1
    # coarsening stops at 16^3: h = 2, 108 tau/h^6 = 0.021 <= 0.05
    assert [x[0] for x in info] == [128, 64, 32, 16]
    for n, h, kind in info:
        s = 108 * p.dt / h ** 6
        want = B.PFC_SWEEP_JACOBI if 0.25 < s < 1000 else B.PFC_SWEEP_RB
        assert kind == want and h == 32.0 / n
    assert [x[2] for x in info][:3] == [B.PFC_SWEEP_RB, B.PFC_SWEEP_JACOBI, B.PFC_SWEEP_JACOBI]
    p.policy = B.PFC_POLICY_RB
    assert all(B.pfc_level_info(p, l)[2] == B.PFC_SWEEP_RB for l in range(4))
    p.coarse_stiffness = 0.0                  # full hierarchy down to 2^3
    assert B.pfc_level_info(p, 6)[0] == 2
    p.coarse_stiffness, p.precision = 0.05, B.PFC_FP64   # FP64 path: full hierarchy
    assert B.pfc_level_info(p, 6)[0] == 2


def test_validation_errors_without_gpu(libpfc):
    p = B.pfc_default_params()
    p.n, p.L, p.eps, p.dt = 16, 32.0, 0.025, 0.01
    ctx = ctypes.c_void_p()
    # null workspace / phi0 are rejected before any CUDA call
    assert libpfc.pfc_init(ctypes.byref(ctx), ctypes.byref(p), None, 0, None, None, None) \
        == B.PFC_EINVAL
    p.eps = 1.0
    assert B.pfc_workspace_bytes(p) == 0
    assert libpfc.pfc_step(None, 1, None) == B.PFC_EINVAL
    assert libpfc.pfc_op_smooth(5, 1.0, 0.1, 0.1, 0, 1, *([None] * 7), None) == B.PFC_EINVAL
    for code in (0, -1, -2, -3, -4, -5):
        assert B.strerror(code)


def test_batch_workspace(libpfc):
    """Ensemble workspaces: per-member fields and FP32 hierarchy scale with the
    member count; more than one member needs PFC_MIXED."""
    p = B.pfc_default_params()
    p.n, p.L, p.eps, p.dt = 32, 32.0, 0.1, 0.05
    p.precision = B.PFC_MIXED
    one = B.pfc_batch_workspace_bytes(p, 1)
    assert one == B.pfc_workspace_bytes(p)
    four = B.pfc_batch_workspace_bytes(p, 4)
    # 10 fine FP64 fields and at least the 10 FP32 fields of the finest level per member
    assert four - one >= 3 * (10 * 8 + 10 * 4) * 32 ** 3
    assert B.pfc_batch_workspace_bytes(p, 0) == 0
    assert B.pfc_batch_workspace_bytes(p, 1025) == 0
    # the launch grids' z extent (65535) bounds 3 n members / 2
    assert B.pfc_batch_workspace_bytes(p, 1024) > 0          # 3 * 32 * 1024 / 2 = 49152
    p.n = 64
    assert B.pfc_batch_workspace_bytes(p, 682) > 0           # 65472
    assert B.pfc_batch_workspace_bytes(p, 683) == 0          # 65568
    p.n = 32
    p.precision = B.PFC_FP64
    assert B.pfc_batch_workspace_bytes(p, 2) == 0
    p.precision = B.PFC_MIXED_DF
    assert B.pfc_batch_workspace_bytes(p, 2) == 0


def test_mobility_params(libpfc):
    """M(phi) = m0 + m2 phi^2 needs m0 > 0, m2 >= 0, and anything but M == 1
    needs PFC_MIXED; the three face mobility fields are part of the workspace
    and the two Laplacian fields of the pointwise first defect (M == 1) are
    not."""
    p = B.pfc_default_params()
    assert (p.mobility_m0, p.mobility_m2) == (1.0, 0.0)
    assert p.cluster_tail == 0
    p.n, p.L, p.eps, p.dt = 32, 32.0, 0.1, 0.05
    p.precision = B.PFC_MIXED
    base = B.pfc_workspace_bytes(p)
    p.mobility_m2 = 5.0
    assert B.pfc_workspace_bytes(p) >= base + (3 - 2) * 8 * 32 ** 3
    p.mobility_m0 = 0.0
    assert B.pfc_workspace_bytes(p) == 0
    p.mobility_m0, p.precision = 1.0, B.PFC_FP64
    assert B.pfc_workspace_bytes(p) == 0
    p.precision = B.PFC_MIXED
    assert B.pfc_batch_workspace_bytes(p, 2) > 0     # size only; pfc_batch_init refuses


def test_guess_param(libpfc):
    """guess 0..2; extrapolating all three fields holds a second mu and omega
    (and, on the mixed path, a second pair of their Laplacians) and is
    refused with the double-float state."""
    p = B.pfc_default_params()
    p.n, p.L, p.eps, p.dt = 32, 32.0, 0.1, 0.05
    for prec, fields in ((B.PFC_FP64, 2), (B.PFC_MIXED, 4)):
        p.precision, p.guess = prec, B.PFC_GUESS_PREVIOUS
        base = B.pfc_workspace_bytes(p)
        p.guess = B.PFC_GUESS_EXTRAPOLATE_ALL
        extra = fields * 8 * 32 ** 3
        assert base + extra <= B.pfc_workspace_bytes(p) <= base + extra + 4096
        p.guess = 3
        assert B.pfc_workspace_bytes(p) == 0
    p.precision, p.guess = B.PFC_MIXED_DF, B.PFC_GUESS_EXTRAPOLATE_ALL
    assert B.pfc_workspace_bytes(p) == 0


def test_guess_param_batch_workspace(libpfc):
    """An ensemble with the three-field extrapolated start holds the second
    mu, omega slot and its Laplacians for every member."""
    p = B.pfc_default_params()
    p.n, p.L, p.eps, p.dt = 16, 32.0, 0.1, 0.05
    p.precision, p.guess = B.PFC_MIXED, B.PFC_GUESS_PREVIOUS
    for members in (1, 3, 7):
        base = B.pfc_batch_workspace_bytes(p, members)
        p.guess = B.PFC_GUESS_EXTRAPOLATE_ALL
        extra = 4 * 8 * 16 ** 3 * members
        assert base + extra <= B.pfc_batch_workspace_bytes(p, members) <= base + extra + 4096
        p.guess = B.PFC_GUESS_PREVIOUS


def test_cluster_tail_param(libpfc):
    """cluster_tail is 0, 1 or 2 (default 0) and does not change the
    workspace: the cluster kernel keeps its levels in shared memory."""
    p = B.pfc_default_params()
    p.n, p.L, p.eps, p.dt = 64, 32.0, 0.1, 0.05
    p.precision = B.PFC_MIXED
    off = B.pfc_workspace_bytes(p)
    for mode in (1, 2):
        p.cluster_tail = mode
        assert B.pfc_workspace_bytes(p) == off > 0
    p.cluster_tail = 3
    assert B.pfc_workspace_bytes(p) == 0


def test_step_diagnostics_param(libpfc):
    """step_diagnostics is 0 (default) or 1 and needs no workspace."""
    p = B.pfc_default_params()
    assert p.step_diagnostics == 0
    p.n, p.L, p.eps, p.dt = 32, 32.0, 0.1, 0.05
    base = B.pfc_workspace_bytes(p)
    p.step_diagnostics = 1
    assert B.pfc_workspace_bytes(p) == base > 0
    p.step_diagnostics = 2
    assert B.pfc_workspace_bytes(p) == 0


def test_defect_planes_param(libpfc):
    """defect_planes is >= 0 (default 0, the SM-count heuristic) and needs no
    workspace: a fixed depth whose blocks would not fit the per-block partial
    sums falls back to the heuristic at launch."""
    p = B.pfc_default_params()
    assert p.defect_planes == 0
    p.n, p.L, p.eps, p.dt = 64, 32.0, 0.1, 0.05
    p.precision = B.PFC_MIXED
    base = B.pfc_workspace_bytes(p)
    for z in (1, 8, 64, 1000):
        p.defect_planes = z
        assert B.pfc_workspace_bytes(p) == base > 0
    p.defect_planes = -1
    assert B.pfc_workspace_bytes(p) == 0


def test_group_init_checks_its_arguments(libpfc):
    """pfc_group_init refuses a count outside 1..PFC_MAX_GROUP, a NULL
    context and a repeated context before it touches the device."""
    out = ctypes.c_void_p()
    fake = [ctypes.c_void_p(4096), ctypes.c_void_p(8192)]

    def init(ptrs, count):
        arr = (ctypes.c_void_p * max(1, len(ptrs)))(*ptrs)
        return libpfc.pfc_group_init(ctypes.byref(out), arr, count, None)

    assert init([], 0) == B.PFC_EINVAL
    assert init(fake, B.PFC_MAX_GROUP + 1) == B.PFC_EINVAL
    assert init([fake[0], None], 2) == B.PFC_EINVAL
    assert init([fake[0], fake[0]], 2) == B.PFC_EINVAL
    assert libpfc.pfc_group_step(None, 1, None) == B.PFC_EINVAL
    assert libpfc.pfc_group_graph_launches(None) == -1
    libpfc.pfc_group_destroy(None)


def test_fused_prolong_smooth_checks_arguments(libpfc):
    """pfc_op_lin_prolong_smooth refuses sizes its tiles do not cover (n not
    a multiple of 32), an unknown sweep kind or flag and NULL fields before
    any CUDA call."""
    f = libpfc.pfc_op_lin_prolong_smooth
    fake = [ctypes.c_void_p(4096)] * 13
    assert f(48, 1.0, 0.1, 0.05, B.PFC_SWEEP_RB, 0, 0.7, *fake, None) == B.PFC_EINVAL
    assert f(16, 1.0, 0.1, 0.05, B.PFC_SWEEP_RB, 0, 0.7, *fake, None) == B.PFC_EINVAL
    assert f(64, 1.0, 0.1, 0.05, 7, 0, 0.7, *fake, None) == B.PFC_EINVAL
    assert f(64, 1.0, 0.1, 0.05, B.PFC_SWEEP_RB, 2, 0.7, *fake, None) == B.PFC_EINVAL
    assert f(64, 1.0, 0.1, 0.05, B.PFC_SWEEP_JACOBI, 0, 0.0, *fake, None) == B.PFC_EINVAL
    assert f(64, 1.0, 0.1, 0.05, B.PFC_SWEEP_RB, 0, 0.7, *([None] * 13), None) == B.PFC_EINVAL


def test_start_extrap_checks_arguments(libpfc):
    """pfc_op_start_extrap: an even n >= 2, h > 0 and every pointer (checked
    before any launch)."""
    f = libpfc.pfc_op_start_extrap
    fake = [ctypes.c_void_p(4096 * (i + 1)) for i in range(21)]
    out = ctypes.c_double()
    assert f(7, 1.0, 0.1, 0.05, *fake, ctypes.byref(out), None) == B.PFC_EINVAL
    assert f(8, 0.0, 0.1, 0.05, *fake, ctypes.byref(out), None) == B.PFC_EINVAL
    assert f(8, 1.0, 0.1, 0.05, *([None] * 21), ctypes.byref(out), None) == B.PFC_EINVAL
    assert f(8, 1.0, 0.1, 0.05, *fake, None, None) == B.PFC_EINVAL


def test_folded_correction_checks_arguments(libpfc):
    """pfc_op_lin_smooth_correct refuses n not a multiple of 4, no sweep,
    NULL fields and an FP64 state not 16-byte aligned before any CUDA call."""
    f = libpfc.pfc_op_lin_smooth_correct
    fake = [ctypes.c_void_p(4096)] * 10
    assert f(6, 1.0, 0.1, 0.05, 1, *fake, None) == B.PFC_EINVAL
    assert f(8, 1.0, 0.1, 0.05, 0, *fake, None) == B.PFC_EINVAL
    assert f(8, 1.0, 0.1, 0.05, 1, *([None] * 10), None) == B.PFC_EINVAL
    assert f(8, 1.0, 0.1, 0.05, 1, *fake[:7], ctypes.c_void_p(4104), *fake[8:], None) == \
        B.PFC_EINVAL
