"""Variable mobility M(A phi_*), M(phi) = m0 + m2 phi^2 (Section 5 scheme),
on the PFC_MIXED path: the FP64 defect uses the face mobilities of each step,
the FP32 correction solve a reference mobility; the converged trajectory
equals the oracle's and keeps mass and the weighted energy law."""

import numpy as np
import pytest

from gpu_helpers import host, rel_l2
from oracle import pfc_oracle as O
from paper_1611_06288_gb300 import binding as B
from paper_1611_06288_gb300 import workloads as W
from paper_1611_06288_gb300.solver import PFCSolver

pytestmark = pytest.mark.gpu

MOB = (1.0, 40.0)       # M from 1 to ~1.8 over the random16 field


@pytest.mark.parametrize("graphs", [True, False])
def test_mobility_matches_oracle(graphs):
    wl = W.random16()
    phi0 = wl.phi0()
    prm = O.Params(eps=wl.eps, tau=wl.dt, mobility=MOB)
    ref = []
    O.run(phi0, 4, wl.h, prm, tol=1e-12,
          callback=lambda k, a, b, c, mu, om, res: ref.append((a.copy(), mu.copy())))
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, phi0, precision="mixed", tol=1e-12,
                  max_cycles=100, mobility=MOB)
    s.use_graphs(graphs)
    for k in range(4):
        st = s.step(1)
        assert st.residual <= 1e-12
        assert rel_l2(host(s.phi()), ref[k][0]) <= 1e-10, k
        assert rel_l2(host(s.mu()), ref[k][1]) <= 1e-10, k
    s.close()


def test_mobility_energy_law_and_mass_on_gpu_trajectory():
    """The law with the face-weighted dissipation tau [M D mu, D mu] holds
    along the GPU trajectory of the 32^3 smooth mode with M = 1 + 10 phi^2."""
    wl = W.smooth_sweep(32)
    mob = (1.0, 10.0)
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), precision="mixed", tol=1e-12,
                  max_cycles=100, mobility=mob)
    c = b = wl.phi0()
    m0 = O.mass(b, wl.h)
    for _ in range(3):
        s.step(1)
        a, mu = host(s.phi()), host(s.mu())
        M = O.face_mobilities(b, c, *mob)
        lhs = O.modified_energy(a, b, wl.h, wl.eps) - O.modified_energy(b, c, wl.h, wl.eps)
        diss = sum(O.face_ip(M[ax] * O.op_D(mu, ax, wl.h), O.op_D(mu, ax, wl.h), ax, wl.h)
                   for ax in O.AXES)
        rhs = -wl.dt * diss - 0.5 * O.grad_norm2_sq(a - 2 * b + c, wl.h)
        assert lhs == pytest.approx(rhs, rel=1e-7)
        assert O.mass(a, wl.h) == pytest.approx(m0, rel=1e-12)
        c, b = b, a
    s.close()


def test_mobility_full_size_residual_by_oracle():
    """128^3 smooth mode with M = 1 + 10 phi^2, workload settings: the
    oracle's FP64 residual (with the face mobilities of the step) of the GPU
    step is below the tolerance."""
    wl = W.smooth_sweep(128)
    mob = (1.0, 10.0)
    s = PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), precision="mixed", tol=wl.tol,
                  mobility=mob, **wl.mixed())
    st = s.step(1)
    assert st.residual <= wl.tol
    b = wl.phi0()
    a, mu, om = host(s.phi()), host(s.mu()), host(s.omega())
    p = O.Params(eps=wl.eps, tau=wl.dt, mob=O.face_mobilities(b, b, *mob))
    r = O.residual(O.source_S(b, b, wl.h, p), [a, mu, om], b, wl.h, p)
    assert O.rms(r) <= wl.tol * 1.0001
    s.close()


def test_mobility_validation():
    wl = W.random16()
    for prec in ("fp64", "mixed_df"):
        with pytest.raises(B.PFCError):
            PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), precision=prec, mobility=MOB)
    with pytest.raises(B.PFCError):
        PFCSolver(wl.n, wl.L, wl.eps, wl.dt, wl.phi0(), precision="mixed", mobility=(0.0, 1.0))
