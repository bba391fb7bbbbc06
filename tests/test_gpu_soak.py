"""Short form of the polycrystal-growth soak (Section 6.2 parameters) on the
GPU: every step the mass stays at its initial value and the modified energy
does not rise (Prop. 3.1), for the FP64 and both mixed paths."""

import pytest

from paper_1611_06288_gb300.soak import soak

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
def test_growth_soak_short(precision):
    steps, tol, mean_phi = 300, 1e-9, 0.2025
    r = soak(n=32, steps=steps, precision=precision)
    # mass: a converged step changes h^3 sum(phi) by h^3 sum(r1), and
    # |sum r1| <= sqrt(n^3) ||r1||_2 <= sqrt(3) n^3 tol for an RMS residual
    # tol over the three components, i.e. sqrt(3) tol L^3 against a mass of
    # mean(phi) L^3 per step
    assert r["max_rel_mass_drift"] <= steps * 3 ** 0.5 * tol / mean_phi, r
    # the energy falls by tau |grad mu|^2 + ... >= 0; the residual tolerance can
    # only move it by O(tol)
    assert r["max_rel_energy_rise"] <= 1e-10, r
    assert r["F_modified_end"] < r["F_modified_start"], r
