"""ctypes binding of libpfc (include/pfc.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes
torch tensors (device pointers) or plain numbers; every step of the solver runs
in the CUDA library.  Loading fails loudly if libpfc.so is missing: there is no
CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpfc.so")

PFC_OK, PFC_EINVAL, PFC_ESIZE, PFC_ENOCONV, PFC_ENAN, PFC_ECUDA = 0, -1, -2, -3, -4, -5
PFC_FP64, PFC_MIXED, PFC_MIXED_DF = 0, 1, 2
PFC_GUESS_PREVIOUS, PFC_GUESS_EXTRAPOLATE, PFC_GUESS_EXTRAPOLATE_ALL = 0, 1, 2
PFC_NEWTON, PFC_PICARD = 0, 1
PFC_POLICY_HYBRID, PFC_POLICY_RB = 0, 1
PFC_SWEEP_RB, PFC_SWEEP_JACOBI = 0, 1
PFC_PROLONG_ASSIGN, PFC_PROLONG_SKIP_COLOUR0 = 1, 2


class PFCError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        msg = f"{what}: {strerror(code)} ({code})"
        if detail:
            msg += f" [{detail}]"
        super().__init__(msg)


class pfc_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("L", ctypes.c_double), ("eps", ctypes.c_double),
                ("dt", ctypes.c_double), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_cycles", ctypes.c_int),
                ("precision", ctypes.c_int), ("smoother", ctypes.c_int),
                ("coarsest", ctypes.c_int), ("inner_cycles", ctypes.c_int),
                ("policy", ctypes.c_int), ("jacobi_weight", ctypes.c_double),
                ("jacobi_factor", ctypes.c_int), ("jacobi_factor0", ctypes.c_int),
                ("stiff_hi", ctypes.c_double),
                ("stiff_lo", ctypes.c_double), ("coarse_stiffness", ctypes.c_double),
                ("coarse_sweeps", ctypes.c_int), ("guess", ctypes.c_int),
                ("mobility_m0", ctypes.c_double), ("mobility_m2", ctypes.c_double),
                ("cluster_tail", ctypes.c_int), ("step_diagnostics", ctypes.c_int),
                ("defect_planes", ctypes.c_int)]


class pfc_step_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("cycles_last", ctypes.c_int),
                ("cycles_total", ctypes.c_int), ("residual", ctypes.c_double),
                ("residual0", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t

# name -> (restype, argtypes)
_SIGS = {
    "pfc_default_params": (None, [ctypes.POINTER(pfc_params)]),
    "pfc_workspace_bytes": (_SZ, [ctypes.POINTER(pfc_params)]),
    "pfc_init": (_I, [ctypes.POINTER(_P), ctypes.POINTER(pfc_params), _P, _SZ, _P, _P, _P]),
    "pfc_step": (_I, [_P, _I, ctypes.POINTER(pfc_step_stats)]),
    "pfc_set_state": (_I, [_P, _P, _P]),
    "pfc_get_phi": (_I, [_P, _P]),
    "pfc_get_mu": (_I, [_P, _P]),
    "pfc_get_omega": (_I, [_P, _P]),
    "pfc_energy": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "pfc_mass": (_I, [_P, ctypes.POINTER(_D)]),
    "pfc_step_index": (_I, [_P]),
    "pfc_diagnostics": (_I, [_P, ctypes.POINTER(_D)]),
    "pfc_launch_count": (ctypes.c_longlong, [_P]),
    "pfc_use_graphs": (_I, [_P, _I]),
    "pfc_destroy": (None, [_P]),
    "pfc_strerror": (ctypes.c_char_p, [_I]),
    "pfc_last_error": (ctypes.c_char_p, []),
    "pfc_op_source": (_I, [_I, _D, _D, _P, _P, _P, _P, _P]),
    "pfc_op_smooth": (_I, [_I, _D, _D, _D, _I, _I] + [_P] * 7 + [_P]),
    "pfc_op_residual": (_I, [_I, _D, _D, _D] + [_P] * 10 + [_P]),
    "pfc_op_residual_restrict": (_I, [_I, _D, _D, _D] + [_P] * 13 + [_P]),
    "pfc_op_restrict": (_I, [_I, _P, _P, _P]),
    "pfc_op_coarse_source": (_I, [_I, _D, _D, _D] + [_P] * 7 + [_P]),
    "pfc_op_prolong_correct": (_I, [_I] + [_P] * 9 + [_P]),
    "pfc_op_coarse_solve": (_I, [_I, _D, _D, _D, _I, _I, _D, _I] + [_P] * 10 + [_P]),
    "pfc_op_jacobi": (_I, [_I, _D, _D, _D, _I, _I, _D] + [_P] * 10 + [_P]),
    "pfc_op_lin_jacobi": (_I, [_I, _D, _D, _D, _I, _D, _I] + [_P] * 10 + [_P]),
    "pfc_level_info": (_I, [ctypes.POINTER(pfc_params), _I, ctypes.POINTER(_I),
                            ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "pfc_reduce_scratch_bytes": (_SZ, [_I]),
    "pfc_op_diagnostics": (_I, [_I, _D, _D, _P, _P, _P, ctypes.POINTER(_D), _P]),
    "pfc_op_diagnostics_df": (_I, [_I, _D, _D, _P, _P, _P, ctypes.POINTER(_D), _P]),
    "pfc_op_residual_norm": (_I, [_I, _D, _D, _D] + [_P] * 8 + [ctypes.POINTER(_D), _P]),
    "pfc_op_residual_norm_static": (_I, [_I, _D, _D, _D] + [_P] * 7 +
                                    [ctypes.POINTER(_D), _P]),
    "pfc_op_defect": (_I, [_I, _D, _D, _D] + [_P] * 12 + [ctypes.POINTER(_D), _P, _P]),
    "pfc_op_start_extrap": (_I, [_I, _D, _D, _D] + [_P] * 21 + [ctypes.POINTER(_D), _P]),
    "pfc_op_lin_smooth": (_I, [_I, _D, _D, _D, _I, _I] + [_P] * 7 + [_P]),
    "pfc_op_correct": (_I, [_I] + [_P] * 6 + [_P]),
    "pfc_op_defect_df": (_I, [_I, _D, _D, _D] + [_P] * 12 + [ctypes.POINTER(_D), _P, _P]),
    "pfc_op_correct_df": (_I, [_I] + [_P] * 6 + [_P]),
    "pfc_batch_workspace_bytes": (_SZ, [ctypes.POINTER(pfc_params), _I]),
    "pfc_batch_init": (_I, [ctypes.POINTER(_P), ctypes.POINTER(pfc_params), _I,
                            ctypes.POINTER(_D), _P, _SZ, _P, _P]),
    "pfc_batch_members": (_I, [_P]),
    "pfc_adjoint_step": (_I, [_P, _P, _P, _P, _P, _P, _P, _D, _I, ctypes.POINTER(_D),
                              ctypes.POINTER(_I)]),
    "pfc_batch_diagnostics": (_I, [_P, ctypes.POINTER(_D)]),
    "pfc_group_init": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _P]),
    "pfc_group_step": (_I, [_P, _I, ctypes.POINTER(pfc_step_stats)]),
    "pfc_group_graph_launches": (ctypes.c_longlong, [_P]),
    "pfc_group_destroy": (None, [_P]),
    "pfc_batch_status": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "pfc_op_lin_residual_restrict": (_I, [_I, _D, _D, _D, _I] + [_P] * 10 + [_P]),
    "pfc_op_lin_restrict_chain": (_I, [_I, _D, _D, _D, _I, _I] + [_P] * 16 + [_P]),
    "pfc_op_lin_prolong": (_I, [_I, _I] + [_P] * 6 + [_P]),
    "pfc_op_lin_prolong_smooth": (_I, [_I, _D, _D, _D, _I, _I, _D] + [_P] * 13 + [_P]),
    "pfc_op_lin_smooth_correct": (_I, [_I, _D, _D, _D, _I] + [_P] * 10 + [_P]),
    "pfc_op_restrict_q": (_I, [_I, _I] + [_P] * 4 + [_P]),
    "pfc_op_guess": (_I, [_I, _D, _D] + [_P] * 7 + [_P]),
    "pfc_op_guess_df": (_I, [_I, _D, _D] + [_P] * 7 + [_P]),
    "pfc_op_round_f32": (_I, [ctypes.c_longlong, _P, _P, _P]),
    "pfc_op_widen_f64": (_I, [ctypes.c_longlong, _P, _P, _P]),
    "pfc_op_df_from_f64": (_I, [ctypes.c_longlong, _P, _P, _P]),
    "pfc_op_df_to_f64": (_I, [ctypes.c_longlong, _P, _P, _P]),
    "pfc_op_source_df": (_I, [_I, _D, _D, _P, _P, _P, _P, _P]),
    "pfc_profile_enable": (_I, [_P, ctypes.c_uint]),
    "pfc_profile_read": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(_D)]),
}

# kernel classes of pfc_profile_enable / pfc_profile_read
KERNEL_CLASSES = ["source", "restrict", "smooth", "residual_restrict", "coarse_source",
                  "prolong", "coarse_solve", "residual_norm", "defect", "lin_smooth",
                  "lin_restrict", "lin_prolong", "lin_coarse", "correct", "start"]
PROFILE_LEVELS = 24

_lib = None


def lib():
    """Load libpfc.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise PFCError(PFC_EINVAL, "load libpfc.so",
                           f"{LIB_PATH} missing: run `python -m paper_1611_06288_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().pfc_strerror(code).decode()
    except Exception:  # library not loadable: still format the error
        return "error"


def check(rc: int, what: str) -> None:
    if rc != PFC_OK:
        detail = lib().pfc_last_error().decode() if rc in (PFC_ECUDA, PFC_ESIZE) else ""
        raise PFCError(rc, what, detail)


def ptr(t) -> int | None:
    """Device (or host) address of a tensor, None for None."""
    if t is None:
        return None
    return t.data_ptr()


def stream_of(t=None):
    """cudaStream_t of torch's current stream on the tensor's device."""
    import torch
    dev = t.device if t is not None else torch.device("cuda")
    return torch.cuda.current_stream(dev).cuda_stream


# ---------------------------------------------------------------------------
# Solver context
# ---------------------------------------------------------------------------

def pfc_default_params() -> pfc_params:
    p = pfc_params()
    lib().pfc_default_params(ctypes.byref(p))
    return p


def pfc_workspace_bytes(p: pfc_params) -> int:
    return int(lib().pfc_workspace_bytes(ctypes.byref(p)))


def pfc_init(p: pfc_params, workspace, phi0, phi1=None, stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    rc = lib().pfc_init(ctypes.byref(ctx), ctypes.byref(p), ptr(workspace),
                        workspace.numel() * workspace.element_size(), ptr(phi0),
                        ptr(phi1), stream)
    check(rc, "pfc_init")
    return ctx


def pfc_batch_workspace_bytes(p: pfc_params, members: int) -> int:
    return lib().pfc_batch_workspace_bytes(ctypes.byref(p), members)


def pfc_batch_init(p: pfc_params, eps, workspace, phi0, stream=None) -> ctypes.c_void_p:
    members = len(eps)
    e = (ctypes.c_double * members)(*[float(x) for x in eps])
    ctx = ctypes.c_void_p()
    rc = lib().pfc_batch_init(ctypes.byref(ctx), ctypes.byref(p), members, e, ptr(workspace),
                              workspace.numel() * workspace.element_size(), ptr(phi0), stream)
    check(rc, "pfc_batch_init")
    return ctx


PFC_MAX_GROUP = 16


def pfc_group_init(ctxs, stream=None) -> ctypes.c_void_p:
    """A group of contexts advanced together (one graph launch per step)."""
    arr = (_P * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    g = ctypes.c_void_p()
    check(lib().pfc_group_init(ctypes.byref(g), arr, len(ctxs), stream), "pfc_group_init")
    return g


def pfc_group_step(g, count: int, nsteps: int = 1) -> list:
    """Advance the group; returns one pfc_step_stats per context."""
    st = (pfc_step_stats * count)()
    check(lib().pfc_group_step(g, nsteps, st), "pfc_group_step")
    return list(st)


def pfc_group_graph_launches(g) -> int:
    return int(lib().pfc_group_graph_launches(g))


def pfc_group_destroy(g) -> None:
    lib().pfc_group_destroy(g)


def pfc_adjoint_step(ctx, phi_next, phi_k, gnext, gk, gkm1, z, rtol=1e-10, max_cycles=50):
    """One adjoint step (see pfc.h); returns (dL/deps contribution, corrections)."""
    eb = ctypes.c_double(0.0)
    cyc = ctypes.c_int(0)
    check(lib().pfc_adjoint_step(ctx, ptr(phi_next), ptr(phi_k), ptr(gnext), ptr(gk), ptr(gkm1),
                                 ptr(z), rtol, max_cycles, ctypes.byref(eb), ctypes.byref(cyc)),
          "pfc_adjoint_step")
    return eb.value, cyc.value


def pfc_batch_members(ctx) -> int:
    return lib().pfc_batch_members(ctx)


def pfc_batch_diagnostics(ctx, members: int):
    out = (ctypes.c_double * (4 * members))()
    check(lib().pfc_batch_diagnostics(ctx, out), "pfc_batch_diagnostics")
    return [tuple(out[4 * m:4 * m + 4]) for m in range(members)]


def pfc_batch_status(ctx, members: int):
    it = (ctypes.c_int * members)()
    r = (ctypes.c_double * members)()
    r0 = (ctypes.c_double * members)()
    check(lib().pfc_batch_status(ctx, it, r, r0), "pfc_batch_status")
    return list(it), list(r), list(r0)


def pfc_step(ctx, nsteps: int = 1) -> pfc_step_stats:
    st = pfc_step_stats()
    check(lib().pfc_step(ctx, nsteps, ctypes.byref(st)), "pfc_step")
    return st


def pfc_set_state(ctx, phi, phi_prev=None) -> None:
    check(lib().pfc_set_state(ctx, ptr(phi), ptr(phi_prev)), "pfc_set_state")


def pfc_get_phi(ctx, dst) -> None:
    check(lib().pfc_get_phi(ctx, ptr(dst)), "pfc_get_phi")


def pfc_get_mu(ctx, dst) -> None:
    check(lib().pfc_get_mu(ctx, ptr(dst)), "pfc_get_mu")


def pfc_get_omega(ctx, dst) -> None:
    check(lib().pfc_get_omega(ctx, ptr(dst)), "pfc_get_omega")


def pfc_energy(ctx) -> tuple[float, float]:
    F, Fm = ctypes.c_double(), ctypes.c_double()
    check(lib().pfc_energy(ctx, ctypes.byref(F), ctypes.byref(Fm)), "pfc_energy")
    return F.value, Fm.value


def pfc_mass(ctx) -> float:
    m = ctypes.c_double()
    check(lib().pfc_mass(ctx, ctypes.byref(m)), "pfc_mass")
    return m.value


def pfc_step_index(ctx) -> int:
    return int(lib().pfc_step_index(ctx))


def pfc_diagnostics(ctx) -> list[float]:
    out = (ctypes.c_double * 4)()
    check(lib().pfc_diagnostics(ctx, out), "pfc_diagnostics")
    return list(out)


def pfc_use_graphs(ctx, on: bool) -> None:
    check(lib().pfc_use_graphs(ctx, int(bool(on))), "pfc_use_graphs")


def pfc_launch_count(ctx) -> int:
    return int(lib().pfc_launch_count(ctx))


def pfc_destroy(ctx) -> None:
    lib().pfc_destroy(ctx)


def pfc_profile_enable(ctx, mask: int) -> None:
    check(lib().pfc_profile_enable(ctx, mask), "pfc_profile_enable")


def pfc_profile_read(ctx, kclass: int, level: int) -> tuple[int, float]:
    n, ms = ctypes.c_longlong(), ctypes.c_double()
    check(lib().pfc_profile_read(ctx, kclass, level, ctypes.byref(n), ctypes.byref(ms)),
          "pfc_profile_read")
    return n.value, ms.value


# ---------------------------------------------------------------------------
# Primitive operations (tensors in, results written into tensors)
# ---------------------------------------------------------------------------

def pfc_op_source(n, h, eps, b, c, S2, S3, stream=None):
    check(lib().pfc_op_source(n, h, eps, ptr(b), ptr(c), ptr(S2), ptr(S3), stream),
          "pfc_op_source")


def pfc_op_smooth(n, h, eps, tau, smoother, sweeps, phi, mu, om, S1, S2, S3, b, stream=None):
    check(lib().pfc_op_smooth(n, h, eps, tau, smoother, sweeps, ptr(phi), ptr(mu), ptr(om),
                              ptr(S1), ptr(S2), ptr(S3), ptr(b), stream), "pfc_op_smooth")


def pfc_op_residual(n, h, eps, tau, phi, mu, om, S1, S2, S3, b, r1, r2, r3, stream=None):
    check(lib().pfc_op_residual(n, h, eps, tau, ptr(phi), ptr(mu), ptr(om), ptr(S1), ptr(S2),
                                ptr(S3), ptr(b), ptr(r1), ptr(r2), ptr(r3), stream),
          "pfc_op_residual")


def pfc_op_residual_restrict(n, h, eps, tau, phi, mu, om, S1, S2, S3, b,
                             rc1, rc2, rc3, uc1, uc2, uc3, stream=None):
    check(lib().pfc_op_residual_restrict(
        n, h, eps, tau, ptr(phi), ptr(mu), ptr(om), ptr(S1), ptr(S2), ptr(S3), ptr(b),
        ptr(rc1), ptr(rc2), ptr(rc3), ptr(uc1), ptr(uc2), ptr(uc3), stream),
        "pfc_op_residual_restrict")


def pfc_op_restrict(n, fine, coarse, stream=None):
    check(lib().pfc_op_restrict(n, ptr(fine), ptr(coarse), stream), "pfc_op_restrict")


def pfc_op_coarse_source(n, h, eps, tau, uc1, uc2, uc3, bc, r1, r2, r3, stream=None):
    check(lib().pfc_op_coarse_source(n, h, eps, tau, ptr(uc1), ptr(uc2), ptr(uc3), ptr(bc),
                                     ptr(r1), ptr(r2), ptr(r3), stream),
          "pfc_op_coarse_source")


def pfc_op_prolong_correct(n, vc1, vc2, vc3, wc1, wc2, wc3, u1, u2, u3, stream=None):
    check(lib().pfc_op_prolong_correct(n, ptr(vc1), ptr(vc2), ptr(vc3), ptr(wc1), ptr(wc2),
                                       ptr(wc3), ptr(u1), ptr(u2), ptr(u3), stream),
          "pfc_op_prolong_correct")


def pfc_op_coarse_solve(n, h, eps, tau, smoother, kind, weight, max_sweeps, phi, mu, om,
                        t1, t2, t3, S1, S2, S3, b, stream=None):
    check(lib().pfc_op_coarse_solve(n, h, eps, tau, smoother, kind, weight, max_sweeps,
                                    ptr(phi), ptr(mu), ptr(om), ptr(t1), ptr(t2), ptr(t3),
                                    ptr(S1), ptr(S2), ptr(S3), ptr(b), stream),
          "pfc_op_coarse_solve")


def pfc_op_jacobi(n, h, eps, tau, smoother, sweeps, weight, phi, mu, om, t1, t2, t3,
                  S1, S2, S3, b, stream=None):
    check(lib().pfc_op_jacobi(n, h, eps, tau, smoother, sweeps, weight, ptr(phi), ptr(mu),
                              ptr(om), ptr(t1), ptr(t2), ptr(t3), ptr(S1), ptr(S2), ptr(S3),
                              ptr(b), stream), "pfc_op_jacobi")


def pfc_op_lin_jacobi(n, h, eps, tau, sweeps, weight, zero_init, d1, d2, d3, t1, t2, t3,
                      r1, r2, r3, q, stream=None):
    check(lib().pfc_op_lin_jacobi(n, h, eps, tau, sweeps, weight, int(bool(zero_init)),
                                  ptr(d1), ptr(d2), ptr(d3), ptr(t1), ptr(t2), ptr(t3),
                                  ptr(r1), ptr(r2), ptr(r3), ptr(q), stream),
          "pfc_op_lin_jacobi")


def pfc_level_info(p: pfc_params, level: int):
    n, h, kind = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    check(lib().pfc_level_info(ctypes.byref(p), level, ctypes.byref(n), ctypes.byref(h),
                               ctypes.byref(kind)), "pfc_level_info")
    return n.value, h.value, kind.value


def pfc_reduce_scratch_bytes(n) -> int:
    return int(lib().pfc_reduce_scratch_bytes(n))


def pfc_op_diagnostics(n, h, eps, a, b, scratch, stream=None):
    out = (ctypes.c_double * 4)()
    check(lib().pfc_op_diagnostics(n, h, eps, ptr(a), ptr(b), ptr(scratch), out, stream),
          "pfc_op_diagnostics")
    return list(out)


def pfc_op_diagnostics_df(n, h, eps, a, b, scratch, stream=None):
    out = (ctypes.c_double * 4)()
    check(lib().pfc_op_diagnostics_df(n, h, eps, ptr(a), ptr(b), ptr(scratch), out, stream),
          "pfc_op_diagnostics_df")
    return list(out)


def pfc_op_residual_norm(n, h, eps, tau, phi, mu, om, S1, S2, S3, b, scratch, stream=None):
    out = ctypes.c_double()
    check(lib().pfc_op_residual_norm(n, h, eps, tau, ptr(phi), ptr(mu), ptr(om), ptr(S1),
                                     ptr(S2), ptr(S3), ptr(b), ptr(scratch),
                                     ctypes.byref(out), stream), "pfc_op_residual_norm")
    return out.value


def pfc_op_residual_norm_static(n, h, eps, tau, phi, mu, om, S1, S2, S3, b, stream=None):
    """RMS residual with the library's own static scratch (no allocation)."""
    out = ctypes.c_double()
    check(lib().pfc_op_residual_norm_static(n, h, eps, tau, ptr(phi), ptr(mu), ptr(om),
                                            ptr(S1), ptr(S2), ptr(S3), ptr(b),
                                            ctypes.byref(out), stream),
          "pfc_op_residual_norm_static")
    return out.value


def pfc_op_start_extrap(n, h, eps, tau, b, c, lapb, lapc, mu0, om0, lapmu0, lapom0, mu1, om1,
                        lapmu1, lapom1, S2, S3, phi, lap, r1, r2, r3, q, scratch,
                        stream=None):
    out = ctypes.c_double()
    args = [b, c, lapb, lapc, mu0, om0, lapmu0, lapom0, mu1, om1, lapmu1, lapom1, S2, S3, phi,
            lap, r1, r2, r3, q, scratch]
    check(lib().pfc_op_start_extrap(n, h, eps, tau, *[ptr(a) for a in args], ctypes.byref(out),
                                    stream), "pfc_op_start_extrap")
    return out.value


def pfc_op_defect(n, h, eps, tau, phi, mu, om, S1, S2, S3, b, r1, r2, r3, q, scratch,
                  stream=None, lap=None):
    out = ctypes.c_double()
    check(lib().pfc_op_defect(n, h, eps, tau, ptr(phi), ptr(mu), ptr(om), ptr(S1), ptr(S2),
                              ptr(S3), ptr(b), ptr(r1), ptr(r2), ptr(r3), ptr(q),
                              ptr(scratch), ctypes.byref(out), ptr(lap), stream), "pfc_op_defect")
    return out.value


def pfc_op_defect_df(n, h, eps, tau, phi, mu, om, S1, S2, S3, b, r1, r2, r3, q, scratch,
                  stream=None, lap=None):
    out = ctypes.c_double()
    check(lib().pfc_op_defect_df(n, h, eps, tau, ptr(phi), ptr(mu), ptr(om), ptr(S1), ptr(S2),
                              ptr(S3), ptr(b), ptr(r1), ptr(r2), ptr(r3), ptr(q),
                              ptr(scratch), ctypes.byref(out), ptr(lap), stream), "pfc_op_defect_df")
    return out.value


def pfc_op_lin_smooth(n, h, eps, tau, sweeps, zero_init, d1, d2, d3, r1, r2, r3, q,
                      stream=None):
    check(lib().pfc_op_lin_smooth(n, h, eps, tau, sweeps, int(bool(zero_init)), ptr(d1),
                                  ptr(d2), ptr(d3), ptr(r1), ptr(r2), ptr(r3), ptr(q),
                                  stream), "pfc_op_lin_smooth")


def pfc_op_lin_residual_restrict(n, h, eps, tau, zero_init, d1, d2, d3, r1, r2, r3, q, c1, c2,
                                 c3, stream=None):
    check(lib().pfc_op_lin_residual_restrict(n, h, eps, tau, int(bool(zero_init)), ptr(d1),
                                             ptr(d2), ptr(d3), ptr(r1), ptr(r2), ptr(r3),
                                             ptr(q), ptr(c1), ptr(c2), ptr(c3), stream),
          "pfc_op_lin_residual_restrict")


def pfc_op_restrict_q(n, levels, q, c, e=None, g=None, stream=None):
    check(lib().pfc_op_restrict_q(n, levels, ptr(q), ptr(c), ptr(e), ptr(g), stream),
          "pfc_op_restrict_q")


def pfc_op_lin_restrict_chain(n, h, eps, tau, zero_init, levels, d1, d2, d3, r1, r2, r3, q,
                              c1, c2, c3, e1, e2, e3, g1=None, g2=None, g3=None, stream=None):
    check(lib().pfc_op_lin_restrict_chain(n, h, eps, tau, int(bool(zero_init)), levels,
                                          *[ptr(x) for x in (d1, d2, d3, r1, r2, r3, q, c1, c2,
                                                             c3, e1, e2, e3, g1, g2, g3)],
                                          stream), "pfc_op_lin_restrict_chain")


def pfc_op_lin_prolong(n, assign, e1, e2, e3, d1, d2, d3, stream=None):
    """assign: a bool, or the flags PFC_PROLONG_ASSIGN | PFC_PROLONG_SKIP_COLOUR0."""
    check(lib().pfc_op_lin_prolong(n, int(assign), ptr(e1), ptr(e2), ptr(e3), ptr(d1),
                                   ptr(d2), ptr(d3), stream), "pfc_op_lin_prolong")


def pfc_op_lin_smooth_correct(n, h, eps, tau, sweeps, d1, d2, d3, r1, r2, r3, q, u1, u2, u3,
                              stream=None):
    """Red-black sweeps whose last colour-1 pass adds d to the FP64 state u."""
    check(lib().pfc_op_lin_smooth_correct(n, h, eps, tau, sweeps,
                                          *[ptr(x) for x in (d1, d2, d3, r1, r2, r3, q, u1, u2,
                                                             u3)], stream),
          "pfc_op_lin_smooth_correct")


def pfc_op_lin_prolong_smooth(n, h, eps, tau, kind, assign, weight, e1, e2, e3, d1, d2, d3,
                              t1, t2, t3, r1, r2, r3, q, stream=None):
    """d (+)= P e and one post-smoothing sweep of `kind` (PFC_SWEEP_RB or
    PFC_SWEEP_JACOBI), the prolongation fused into the first pass."""
    check(lib().pfc_op_lin_prolong_smooth(n, h, eps, tau, kind,
                                          PFC_PROLONG_ASSIGN if assign else 0, weight,
                                          *[ptr(x) for x in (e1, e2, e3, d1, d2, d3, t1, t2, t3,
                                                             r1, r2, r3, q)], stream),
          "pfc_op_lin_prolong_smooth")


def pfc_op_guess(n, h, eps, b, c, S2, S3, phi, mu, om, stream=None):
    check(lib().pfc_op_guess(n, h, eps, ptr(b), ptr(c), ptr(S2), ptr(S3), ptr(phi), ptr(mu),
                             ptr(om), stream), "pfc_op_guess")


def pfc_op_guess_df(n, h, eps, b, c, S2, S3, phi, mu, om, stream=None):
    check(lib().pfc_op_guess_df(n, h, eps, ptr(b), ptr(c), ptr(S2), ptr(S3), ptr(phi), ptr(mu),
                                ptr(om), stream), "pfc_op_guess_df")


def pfc_op_round_f32(count, x, y, stream=None):
    check(lib().pfc_op_round_f32(count, ptr(x), ptr(y), stream), "pfc_op_round_f32")


def pfc_op_widen_f64(count, x, y, stream=None):
    check(lib().pfc_op_widen_f64(count, ptr(x), ptr(y), stream), "pfc_op_widen_f64")


def pfc_op_df_from_f64(count, x, y, stream=None):
    check(lib().pfc_op_df_from_f64(count, ptr(x), ptr(y), stream), "pfc_op_df_from_f64")


def pfc_op_df_to_f64(count, y, x, stream=None):
    check(lib().pfc_op_df_to_f64(count, ptr(y), ptr(x), stream), "pfc_op_df_to_f64")


def pfc_op_source_df(n, h, eps, b, c, S2, S3, stream=None):
    check(lib().pfc_op_source_df(n, h, eps, ptr(b), ptr(c), ptr(S2), ptr(S3), stream),
          "pfc_op_source_df")


def pfc_op_correct(n, u1, u2, u3, d1, d2, d3, stream=None):
    check(lib().pfc_op_correct(n, ptr(u1), ptr(u2), ptr(u3), ptr(d1), ptr(d2), ptr(d3),
                               stream), "pfc_op_correct")



def pfc_op_correct_df(n, u1, u2, u3, d1, d2, d3, stream=None):
    check(lib().pfc_op_correct_df(n, ptr(u1), ptr(u2), ptr(u3), ptr(d1), ptr(d2), ptr(d3),
                               stream), "pfc_op_correct_df")
