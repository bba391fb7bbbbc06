"""Plant plausible mistakes in the CPU oracle (monkeypatched, CPU only) and
check that the pins of test_oracle_pins.py catch each one."""

import numpy as np
import pytest

import test_oracle_pins as P
from oracle import pfc_oracle as O


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_wrong_cubic_average_is_caught(monkeypatch):
    # phi^3 at the new level instead of the Crank-Nicolson-type average
    monkeypatch.setattr(O, "cubic_f", lambda a, b: a ** 3)
    monkeypatch.setattr(O, "cubic_fprime", lambda a, b: 3 * a * a)
    _fails(P.test_energy_law_and_mass_random16)


def test_wrong_explicit_sign_is_caught(monkeypatch):
    def bad_source(b, c, h, prm):
        s1, s2, s3 = b.copy(), None, 0.5 * O.lap(b, h)
        s2 = 0.5 * (1 - prm.eps) * b - 3.0 * O.lap(b, h) + O.lap(c, h)
        return [s1, s2, s3]
    monkeypatch.setattr(O, "source_S", bad_source)
    _fails(P.test_linear_scheme_fourier_closed_form, 8, 12.0)


def test_dropped_previous_level_is_caught(monkeypatch):
    def bad_source(b, c, h, prm):
        return [b.copy(), 0.5 * (1 - prm.eps) * b + 3.0 * O.lap(b, h),
                0.5 * O.lap(b, h)]
    monkeypatch.setattr(O, "source_S", bad_source)
    _fails(P.test_linear_scheme_fourier_closed_form, 8, 12.0)


def test_omega_misprint_is_caught(monkeypatch):
    # omega := Delta_h phi^{k+1} (the misprint of Eq. 1.10) instead of Eq. 5.3
    orig = O.operator_N

    def bad_N(u, b, h, prm):
        n1, n2, _ = orig(u, b, h, prm)
        return [n1, n2, u[2] - O.lap(u[0], h)]

    def bad_source(b, c, h, prm):
        s = [b.copy(), 0.5 * (1 - prm.eps) * b + 3 * O.lap(b, h) - O.lap(c, h),
             0.0 * b]
        return s
    monkeypatch.setattr(O, "operator_N", bad_N)
    monkeypatch.setattr(O, "source_S", bad_source)
    _fails(P.test_linear_scheme_fourier_closed_form, 8, 12.0)


def test_wrong_smoother_entry_is_caught(monkeypatch):
    orig = O.cramer3

    def bad(A, rhs):
        A = [list(row) for row in A]
        A[1][2] = 0.5 * A[1][2]          # 3/h^2 in place of 6/h^2
        return orig(A, rhs)
    monkeypatch.setattr(O, "cramer3", bad)
    _fails(P.test_exact_solution_is_smoother_fixed_point)


def test_transposed_cramer_is_caught(monkeypatch):
    orig = O.cramer3

    def bad(A, rhs):
        At = [[A[j][i] for j in range(3)] for i in range(3)]
        return orig(At, rhs)
    monkeypatch.setattr(O, "cramer3", bad)
    _fails(P.test_cramer_matches_lapack)


def test_swapped_prolongation_weights_are_caught(monkeypatch):
    def bad_axis(v, ax):
        lo = 0.75 * v + 0.25 * np.roll(v, -1, ax)
        hi = 0.75 * v + 0.25 * np.roll(v, 1, ax)
        out = np.stack([lo, hi], axis=ax + 1)
        shape = list(v.shape)
        shape[ax] *= 2
        return out.reshape(shape)
    monkeypatch.setattr(O, "_prolong_axis", bad_axis)
    _fails(P.test_transfers)


def test_wrong_energy_sign_is_caught(monkeypatch):
    orig = O.grad_norm2_sq
    monkeypatch.setattr(O, "energy", lambda phi, h, eps: (
        0.25 * O.norm_p(phi, h, 4) ** 4 + 0.5 * (1 - eps) * O.norm2(phi, h) ** 2
        + orig(phi, h) + 0.5 * O.norm2(O.lap(phi, h), h) ** 2))
    _fails(P.test_energy_single_mode_closed_form)


def test_wrong_laplacian_neighbour_is_caught(monkeypatch):
    # forward difference taken twice in z: a wrong index in one direction
    monkeypatch.setattr(O, "op_d", lambda w, axis, h: (
        (np.roll(w, -1, axis) - w) / h if axis == O.AX_Z else (w - np.roll(w, 1, axis)) / h))
    _fails(P.test_laplacian_fourier_symbol, 8, 32.0)


def test_cell_corner_sampling_is_caught(monkeypatch):
    # fields sampled at i h (cell corners) instead of the cell centres (i + 1/2) h
    from paper_1611_06288_gb300 import workloads as W

    def corners(n, L):
        c = np.arange(n) * (L / n)
        return c[:, None, None], c[None, :, None], c[None, None, :]
    monkeypatch.setattr(W, "cell_centres", corners)
    _fails(P.test_second_order_in_space, P_golden())


def test_wrong_spacing_on_one_level_is_caught(monkeypatch):
    # the 16^3 grid of the refinement run with twice its spacing
    orig = O.run

    def bad_run(phi0, nsteps, h, prm, *a, **kw):
        if phi0.shape[0] == 16:
            h = 2.0 * h
        return orig(phi0, nsteps, h, prm, *a, **kw)
    monkeypatch.setattr(O, "run", bad_run)
    _fails(P.test_second_order_in_space, P_golden())


def P_golden():
    import os
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
