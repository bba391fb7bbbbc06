"""Parity of the full CUDA time step (pfc_init / pfc_step / pfc_energy /
pfc_mass through the C ABI) with the CPU oracle, and properties that hold at
any size checked on the full-size workloads in the launch configuration the
benchmark uses."""

import math

import numpy as np
import pytest
import torch

from gpu_helpers import host, rel_l2
from oracle import pfc_oracle as O
from paper_1611_06288_gb300 import binding as B
from paper_1611_06288_gb300 import workloads as W
from paper_1611_06288_gb300.solver import PFCSolver

pytestmark = pytest.mark.gpu

# Both sides converged to an RMS residual of 1e-12: the solution of N(u) = S
# is unique (Prop. 3.1) and the residual-to-error gain is O(1), so the fields
# agree to ~1e-11 relative; the bound of the method is 1e-10.
PARITY_RTOL = 1e-10


def oracle_run(phi0, steps, h, eps, dt, lin, tol=1e-12):
    p = O.Params(eps=eps, tau=dt, linearization=lin)
    traj = []

    def cb(k, a, b, c, mu, om, res):
        traj.append((a.copy(), mu.copy(), om.copy()))

    O.run(phi0, steps, h, p, tol=tol, callback=cb)
    return traj


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
@pytest.mark.parametrize("smoother", ["newton", "picard"])
@pytest.mark.parametrize("graphs", [True, False])
def test_random16_ten_steps(precision, smoother, graphs):
    """16^3, L = 32, eps = 0.025, phi0 = 0.07 + 0.07 U(-1,1), dt = 0.01, 10
    steps with the phi^{-1} := phi^0 start: every step matches the oracle, with
    the device-side (graph) loop and with the host-driven loop."""
    wl = W.random16()
    phi0 = wl.phi0()
    ref = oracle_run(phi0, wl.steps, wl.h, wl.eps, wl.dt, smoother)
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=1e-12, precision=precision,
                  smoother=smoother, max_cycles=60)
    s.use_graphs(graphs)
    for k in range(wl.steps):
        st = s.step(1)
        assert st.residual <= 1e-12
        a, mu, om = host(s.phi()), host(s.mu()), host(s.omega())
        assert rel_l2(a, ref[k][0]) <= PARITY_RTOL, (k, rel_l2(a, ref[k][0]))
        assert rel_l2(mu, ref[k][1]) <= PARITY_RTOL
        assert rel_l2(om, ref[k][2]) <= PARITY_RTOL
    F, Fm = s.energy()
    assert F == pytest.approx(O.energy(ref[-1][0], wl.h, wl.eps), rel=1e-10)
    assert Fm == pytest.approx(O.modified_energy(ref[-1][0], ref[-2][0], wl.h, wl.eps),
                               rel=1e-10)
    assert s.mass() == pytest.approx(O.mass(phi0, wl.h), rel=1e-12)
    assert s.step_index == wl.steps


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
@pytest.mark.parametrize("nu", [(0, 1), (1, 0), (0, 2), (1, 2)])
@pytest.mark.parametrize("graphs", [True, False])
def test_mixed_cycle_shapes(nu, graphs, precision):
    """Mixed path with V(nu1, nu2) inner cycles, including no pre-smoothing
    (the zero-start restriction and assigning prolongation) and no
    post-smoothing: the converged steps match the oracle."""
    n, L = 32, 48.0           # levels 32 (global memory) and 16 (shared-memory tail)
    rng = np.random.default_rng(32)
    phi0 = 0.1 + 0.1 * rng.uniform(-1, 1, (n,) * 3)
    ref = oracle_run(phi0, 2, L / n, 0.2, 0.05, "newton")
    s = PFCSolver(n, L, 0.2, 0.05, phi0, tol=1e-12, precision=precision, nu1=nu[0], nu2=nu[1],
                  inner_cycles=2, coarse_sweeps=2, max_cycles=80)
    s.use_graphs(graphs)
    for k in range(2):
        st = s.step(1)
        assert st.residual <= 1e-12
        assert rel_l2(host(s.phi()), ref[k][0]) <= PARITY_RTOL


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
@pytest.mark.parametrize("graphs", [True, False])
def test_extrapolated_guess(precision, graphs):
    """guess = extrapolate starts each step from 2 phi^k - phi^{k-1} with
    omega and mu from rows 3 and 2: the same converged trajectory as the
    oracle (which starts from phi^k), and on a smooth trajectory fewer
    corrections than the plain start."""
    wl = W.random16()
    phi0 = wl.phi0()
    ref = oracle_run(phi0, 5, wl.h, wl.eps, wl.dt, "newton")
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=1e-12, precision=precision,
                  guess="extrapolate", max_cycles=60)
    s.use_graphs(graphs)
    for k in range(5):
        st = s.step(1)
        assert st.residual <= 1e-12
        assert rel_l2(host(s.phi()), ref[k][0]) <= PARITY_RTOL
        assert rel_l2(host(s.mu()), ref[k][1]) <= PARITY_RTOL
    wl = W.smooth_sweep(32)
    kw = wl.mixed() if precision != "fp64" else {}
    cyc = {}
    for guess in ("previous", "extrapolate"):
        s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), tol=wl.tol, precision=precision,
                      guess=guess, **kw)
        s.use_graphs(graphs)
        s.step(2)
        cyc[guess] = s.step(4).cycles_total
    assert cyc["extrapolate"] < cyc["previous"], cyc


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graphs", [True, False])
def test_extrapolate_all_guess(precision, graphs):
    """guess = extrapolate_all starts a step from 2 u^k - u^{k-1} in phi, mu
    and omega once two steps in a row have converged: the same converged
    trajectory as the oracle (which starts from phi^k); pfc_set_state drops
    back to u^k for two steps and keeps the trajectory; on a smooth
    trajectory the mixed path then takes one correction per step."""
    wl = W.random16()
    phi0 = wl.phi0()
    ref = oracle_run(phi0, 7, wl.h, wl.eps, wl.dt, "newton")
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=1e-12, precision=precision,
                  guess="extrapolate_all", max_cycles=60)
    s.use_graphs(graphs)
    for k in range(7):
        if k == 4:
            s.set_state(ref[3][0], ref[2][0])
        st = s.step(1)
        assert st.residual <= 1e-12
        assert rel_l2(host(s.phi()), ref[k][0]) <= PARITY_RTOL, k
        assert rel_l2(host(s.mu()), ref[k][1]) <= PARITY_RTOL, k
    s.close()
    wl = W.smooth_sweep(32)
    kw = wl.mixed() if precision != "fp64" else {}
    cyc = {}
    for guess in ("previous", "extrapolate_all"):
        s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), tol=wl.tol, precision=precision,
                      guess=guess, **kw)
        s.use_graphs(graphs)
        s.step(3)
        cyc[guess] = s.step(4).cycles_total
        s.close()
    assert cyc["extrapolate_all"] < cyc["previous"], cyc
    if precision == "mixed":
        assert cyc["extrapolate_all"] == 4, cyc


def test_extrapolate_all_guess_is_refused_with_df_state():
    """The double-float state path has no extrapolated mu, omega: the
    parameters are refused (no workspace size) before any allocation."""
    wl = W.random16()
    with pytest.raises(B.PFCError):
        PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), precision="mixed_df",
                  guess="extrapolate_all")


@pytest.mark.parametrize("n,coarsest", [(4, 2), (12, 6), (20, 10), (24, 6)])
def test_uneven_sizes_and_level_counts(n, coarsest):
    """Grids that are not powers of two and the smallest grid, against the
    oracle (one step from a random start on a box with h = 1.5)."""
    L = 1.5 * n
    rng = np.random.default_rng(n)
    phi0 = 0.1 + 0.1 * rng.uniform(-1, 1, (n,) * 3)
    ref = oracle_run(phi0, 2, L / n, 0.2, 0.05, "newton")
    for precision in ("fp64", "mixed", "mixed_df"):
        s = PFCSolver(n, L, 0.2, 0.05, phi0, tol=1e-12, coarsest=coarsest,
                      precision=precision, max_cycles=200)
        s.step(2)
        assert rel_l2(host(s.phi()), ref[1][0]) <= PARITY_RTOL


def test_constant_state_is_fixed_point():
    n = 16
    phi0 = np.full((n,) * 3, 0.3)
    s = PFCSolver(n, 10.0, 0.3, 0.1, phi0, tol=1e-13)
    s.step(3)
    np.testing.assert_allclose(host(s.phi()), 0.3, rtol=1e-13)
    # mu carries the residual tolerance (1e-13) times O(1) gains
    np.testing.assert_allclose(host(s.mu()), 0.3 ** 3 + 0.7 * 0.3, rtol=1e-11)


def test_start_from_two_levels_and_set_state():
    """phi^1 given explicitly: the same trajectory as the oracle started from
    (phi^0, phi^1); pfc_set_state restarts from a stored pair."""
    wl = W.random16()
    phi0 = wl.phi0()
    p = O.Params(eps=wl.eps, tau=wl.dt)
    phi1 = O.run(phi0, 1, wl.h, p, tol=1e-13)[0]
    a_ref, *_ = O.run(phi0, 3, wl.h, p, tol=1e-13, phi1=phi1)
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, phi1=phi1, tol=1e-13)
    assert s.step_index == 1
    s.step(3)
    assert rel_l2(host(s.phi()), a_ref) <= PARITY_RTOL
    s.set_state(phi1, phi0)
    s.step(3)
    assert rel_l2(host(s.phi()), a_ref) <= PARITY_RTOL


def test_energy_law_and_mass_on_gpu_trajectory():
    """The discrete energy law of Eq. 1.10 and mass conservation hold along
    the GPU trajectory (checked with the oracle's norms)."""
    wl = W.cosine_table(16)
    # at h = 0.2 the FP64 rounding floor of the residual is near 1e-13
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), tol=1e-12, smoother="picard")
    c = b = wl.phi0()
    m0 = O.mass(b, wl.h)
    for _ in range(4):
        s.step(1)
        a, mu = host(s.phi()), host(s.mu())
        lhs = O.modified_energy(a, b, wl.h, wl.eps) - O.modified_energy(b, c, wl.h, wl.eps)
        rhs = (-wl.dt * O.grad_norm2_sq(mu, wl.h)
               - 0.5 * O.grad_norm2_sq(a - 2 * b + c, wl.h))
        assert lhs == pytest.approx(rhs, rel=1e-7)
        assert O.mass(a, wl.h) == pytest.approx(m0, rel=1e-13)
        c, b = b, a


@pytest.mark.parametrize("n,precision", [(128, "mixed"), (128, "mixed_df"), (128, "fp64"),
                                         (256, "mixed")])
def test_full_size_residual_by_oracle(n, precision):
    """Smooth-mode workload (L = 32, eps = 0.025, dt = 0.0125, tol 1e-9) at
    128^3 and 256^3 in the benchmark's configuration (the workload's timed
    settings for the precision, the step diagnostics inside the step; on the
    mixed and FP64 paths the fourth step starts from the three-field
    extrapolation): the oracle evaluates S - N(u) of the GPU's fourth step on
    the CPU in FP64 and finds it below the tolerance, the energy the step
    formed equals the oracle's F_h of the same field, and mass is
    conserved."""
    wl = W.smooth_sweep(n)
    phi0 = wl.phi0()
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=wl.tol, precision=precision,
                  step_diagnostics=True, **wl.settings(precision))
    hist = [phi0]
    for _ in range(3):
        s.step(1)
        hist.append(host(s.phi()))
    st = s.step(1)
    assert st.residual <= wl.tol
    a, mu, om = host(s.phi()), host(s.mu()), host(s.omega())
    b, c = hist[-1], hist[-2]
    p = O.Params(eps=wl.eps, tau=wl.dt)
    r = O.residual(O.source_S(b, c, wl.h, p), [a, mu, om], b, wl.h, p)
    assert O.rms(r) <= wl.tol * 1.0001
    F, _ = s.energy()
    assert F == pytest.approx(O.energy(a, wl.h, wl.eps), rel=1e-10)
    # a converged step moves the mass by at most sqrt(3) tol L^3
    assert O.mass(a, wl.h) == pytest.approx(O.mass(phi0, wl.h),
                                            abs=4 * 3 ** 0.5 * wl.tol * wl.L ** 3)


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
def test_full_size_256_polycrystal_one_step(precision):
    """256^3 polycrystal workload (h = pi/4, eps = 0.25, dt = 0.1), mixed
    precision: the oracle's FP64 residual of the GPU step is below 1e-9 and
    the energy reported by the GPU equals the oracle's F_h of the same field."""
    wl = W.polycrystal(256)
    phi0 = wl.phi0()
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=wl.tol, precision=precision,
                  **wl.mixed())
    st = s.step(1)
    assert st.residual <= wl.tol
    a, mu, om = host(s.phi()), host(s.mu()), host(s.omega())
    p = O.Params(eps=wl.eps, tau=wl.dt)
    r = O.residual(O.source_S(phi0, phi0, wl.h, p), [a, mu, om], phi0, wl.h, p)
    assert O.rms(r) <= wl.tol * 1.0001
    F, _ = s.energy()
    assert F == pytest.approx(O.energy(a, wl.h, wl.eps), rel=1e-11)


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
def test_graph_and_host_loops_agree_at_64(precision):
    """64^3 smooth mode (h = 0.5, tau = 0.0125, hybrid levels): the graph
    loop and the host loop take the same number of cycles and give the same
    fields to rounding."""
    wl = W.smooth_sweep(64)
    out = []
    for graphs in (True, False):
        s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), tol=1e-10, precision=precision,
                      inner_cycles=2)
        s.use_graphs(graphs)
        cyc = [s.step(1).cycles_last for _ in range(3)]
        out.append((cyc, host(s.phi())))
    assert out[0][0] == out[1][0]
    assert rel_l2(out[0][1], out[1][1]) <= 1e-12


@pytest.mark.parametrize("graphs", [True, False])
def test_error_codes(graphs):
    wl = W.random16()
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), tol=1e-14, max_cycles=1)
    s.use_graphs(graphs)
    with pytest.raises(B.PFCError) as e:
        s.step(1)
    assert e.value.code == B.PFC_ENOCONV
    bad = wl.phi0()
    bad[3, 4, 5] = np.nan
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, bad)
    s.use_graphs(graphs)
    with pytest.raises(B.PFCError) as e:
        s.step(1)
    assert e.value.code == B.PFC_ENAN
    # after a NaN the state can be replaced and stepping resumes
    s.set_state(wl.phi0())
    s.step(1)
    with pytest.raises(B.PFCError) as e:
        PFCSolver(6, 6.0, 0.1, 0.1, np.zeros((6, 6, 6)))
    assert e.value.code == B.PFC_ESIZE
    # a failed step leaves the state where it was
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), tol=1e-14, max_cycles=1)
    s.use_graphs(graphs)
    before = host(s.phi())
    with pytest.raises(B.PFCError):
        s.step(1)
    np.testing.assert_array_equal(host(s.phi()), before)
    assert s.step_index == 0


@pytest.mark.parametrize("n", [32, 64])
def test_pointwise_first_defect_matches_full_defect(n):
    """From the second step on, the first defect of a mixed step is formed
    pointwise from the Laplacians the previous step's last defect stored
    (the state is that step's solution).  A run forced onto the full stencil
    defect every step (pfc_set_state with the same fields before each step)
    reaches the same fields: both converge to the 1e-10 residual tolerance
    of the same uniquely solvable steps (Prop. 3.1); set_state's FP64
    Laplacians differ from the stored ones by rounding only.  The warm run's
    last step also passes the oracle's FP64 residual check."""
    wl = W.smooth_sweep(n)
    phi0 = wl.phi0()
    kw = dict(wl.mixed())
    a = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=1e-10, precision="mixed", **kw)
    bsol = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=1e-10, precision="mixed", **kw)
    hist = [phi0]                                   # phi^0, phi^1, ... of run B
    for k in range(5):
        if k == 4:
            prev_a = host(a.phi())
        a.step(1)
        if k > 0:
            bsol.set_state(hist[-1], hist[-2])     # cold: the full defect again
        bsol.step(1)
        hist.append(host(bsol.phi()))
    pa, pb = host(a.phi()), host(bsol.phi())
    assert rel_l2(pa, pb) <= 1e-8
    mu, om = host(a.mu()), host(a.omega())
    p = O.Params(eps=wl.eps, tau=wl.dt)
    r = O.residual(O.source_S(prev_a, prev_a, wl.h, p), [pa, mu, om], prev_a, wl.h, p)
    # rows 1 and 3 need only phi^k (S1 = phi^k, S3 = Lap phi^k / 2)
    assert np.sqrt(np.mean(r[0] ** 2 + r[2] ** 2) / 3) <= 1e-10 * 1.0001
    a.close()
    bsol.close()


@pytest.mark.parametrize("precision", ["mixed", "mixed_df", "fp64"])
def test_step_diagnostics_match_on_request(precision):
    """step_diagnostics forms the energy/mass sums of each new state inside
    the step's graph; pfc_diagnostics then returns them without a launch.
    They equal the on-request values bit for bit (same kernels, same
    inputs), and after pfc_set_state they are formed on request again."""
    wl = W.smooth_sweep(32)
    phi0 = wl.phi0()
    kw = wl.mixed() if precision != "fp64" else {}
    runs = []
    for sd in (True, False):
        s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=1e-10, precision=precision,
                      step_diagnostics=sd, **kw)
        out = []
        for _ in range(3):
            s.step(1)
            launches = B.pfc_launch_count(s.ctx)
            out.append(s.diagnostics())
            if sd:
                assert B.pfc_launch_count(s.ctx) == launches      # nothing launched
        s.set_state(host(s.phi()))
        out.append(s.diagnostics())
        runs.append(out)
        s.close()
    assert runs[0] == runs[1]


@pytest.mark.parametrize("n", [48, 64])
def test_defect_tile_depth_does_not_change_the_step(n):
    """defect_planes fixes the planes per block of the FP64 defect (the
    autotuner's tile dimension): 1 plane per block, ragged last columns
    (5 planes of 48 or 64), one column per tile (n and beyond) and the
    heuristic's choice.  Each cell's rows are the same arithmetic whatever the
    tile, so r and the iterates are identical; only the residual norm's
    summation order changes.  Equal cycle counts therefore give bit-equal
    fields.  Each thread sums the three rows' squares over its planes and the
    block over its threads in FP32 (positive terms: relative error <=
    (terms - 1) 2^-24), so each norm is within (3n + 256) 2^-24 relative of
    the exact sum and two tilings' norms within twice that."""
    wl = W.smooth_sweep(n)
    phi0 = wl.phi0()
    kw = dict(wl.mixed())
    out = {}
    for z in (0, 1, 5, n, 4 * n):
        s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, tol=1e-10, precision="mixed",
                      defect_planes=z, **kw)
        cyc, res = [], []
        for _ in range(3):
            st = s.step(1)
            cyc.append(st.cycles_last)
            res.append(st.residual)
        out[z] = (cyc, res, host(s.phi()), host(s.mu()), host(s.omega()))
        s.close()
    cyc0, res0, *f0 = out[0]
    for z, (cyc, res, *f) in out.items():
        assert cyc == cyc0, (z, cyc, cyc0)
        np.testing.assert_allclose(res, res0, rtol=2 * (3 * n + 256) * 2.0 ** -24, atol=0)
        for x, y in zip(f, f0):
            assert np.array_equal(x, y), z
