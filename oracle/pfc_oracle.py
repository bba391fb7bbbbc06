"""CPU FP64 oracle for the second-order convex-splitting scheme of the periodic
3D phase field crystal (PFC) equation and its nonlinear FAS multigrid solver
(Dong, Feng, Wang, Wise, Zhang, arXiv:1611.06288).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import it.  It imports
nothing from the CUDA package and shares no code with it.

Everything is numpy float64, written to be read against the paper:

* Section 2: cell-centred periodic grid, the average / difference operators
  A, D, a, d, the 7-point Laplacian, the discrete inner products and norms,
  and the discrete energy F_h (Eq. 2.1).
* Section 3: the scheme (Eq. 1.10) in its split form, Section 5 Eqs. 5.1-5.10:
  unknowns u = (phi^{k+1}, mu^{k+1/2}, omega^{k+1/2}), operator N, source S.
* Section 5: the red-black nonlinear Gauss-Seidel smoother with the pointwise
  3x3 system solved by Cramer's rule, and the FAS V-cycle of Algorithm 1.

Readings of points where the paper is silent or garbled (each is repeated in
the design notes of the repository):

* omega^{k+1/2} = (Delta_h phi^{k+1} + Delta_h phi^k) / 2 (Eq. 5.3); the
  "omega := Delta_h phi^{k+1}" of Eq. 1.10 is a misprint.
* Mobility M == 1 (Theorem 3.4); the face mobilities are kept as an argument of
  the flux term so that a variable M can be passed in later.
* Red-black ordering: red = cells with (i + j + k) even (0-based), red first.
* Restriction: 8-cell average; prolongation: trilinear cell-centred
  (1-D weights 3/4, 1/4); coarse operator: the same scheme rediscretised at 2h
  with the restricted phi^k inside the cubic term.
* FAS coarse right-hand side S_c = N_c(I u) + I r; correction u += P(v_c - I u).
* Coarsest level (size <= ``coarsest`` or odd): N(v) = S solved exactly by
  Newton's method with a dense Jacobian (at one cell this is the pointwise
  Cramer solve the paper names).
* Residual norm: RMS over the three components on the finest grid,
  sqrt(sum r^2 / (3 m^3)), compared to an absolute tolerance.
* Start rule: the first step uses phi^{-1} := phi^0, i.e. c = b in the source.
* Pointwise linearisation: "picard" is the paper's local Picard linearisation
  of the cubic term; "newton" linearises f(a) = (a+b)(a^2+b^2)/4 at the current
  value.  Both have the same fixed point.

Array convention: a grid function in C_per is an (m, m, m) float64 array indexed
[k, j, i] = (z, y, x), so the flat C-order index is i + m*(j + m*k).  Cell
centres are ((i+1/2)h, (j+1/2)h, (k+1/2)h) for 0-based indices, which is the
paper's x_i = (i-1/2)h with 1-based i.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

# Array axis used for each coordinate direction (x is the fastest index).
AX_X, AX_Y, AX_Z = 2, 1, 0
AXES = (AX_X, AX_Y, AX_Z)


# --------------------------------------------------------------------------
# Section 2: average and difference operators on the periodic grid
# --------------------------------------------------------------------------

def op_A(v, axis):
    """A_x v at face i+1/2 = (v_{i+1} + v_i)/2; the face i+1/2 is stored at i."""
    return 0.5 * (np.roll(v, -1, axis) + v)


def op_D(v, axis, h):
    """D_x v at face i+1/2 = (v_{i+1} - v_i)/h; the face i+1/2 is stored at i."""
    return (np.roll(v, -1, axis) - v) / h


def op_a(w, axis):
    """a_x w at cell i = (w_{i+1/2} + w_{i-1/2})/2 for a face function w."""
    return 0.5 * (w + np.roll(w, 1, axis))


def op_d(w, axis, h):
    """d_x w at cell i = (w_{i+1/2} - w_{i-1/2})/h for a face function w."""
    return (w - np.roll(w, 1, axis)) / h


def lap(v, h):
    """Discrete Laplacian Delta_h = d_x D_x + d_y D_y + d_z D_z (Section 2)."""
    return sum(op_d(op_D(v, ax, h), ax, h) for ax in AXES)


def div_M_grad(v, h, mob=None):
    """d_x(M^x D_x v) + d_y(M^y D_y v) + d_z(M^z D_z v) (Eq. 5.1).

    ``mob`` is None for M == 1, else a dict axis -> face mobility array.
    """
    total = 0.0
    for ax in AXES:
        flux = op_D(v, ax, h)
        if mob is not None:
            flux = mob[ax] * flux
        total = total + op_d(flux, ax, h)
    return total


def face_mobilities(b, c, m0, m2):
    """M(A phi_*) on the faces i+1/2 of every axis for M(phi) = m0 + m2 phi^2
    and phi_* = 3/2 b - 1/2 c (b = phi^k, c = phi^{k-1})."""
    ps = 1.5 * b - 0.5 * c
    mob = {}
    for ax in AXES:
        a = op_A(ps, ax)
        mob[ax] = m0 + m2 * a * a
    return mob


def face_mobility_sums(shape, mob):
    """Sum of the six face mobilities around each cell (Section 5 smoother)."""
    if mob is None:
        return np.full(shape, 6.0)
    return sum(mob[ax] + np.roll(mob[ax], 1, ax) for ax in AXES)


# --------------------------------------------------------------------------
# Section 2: inner products, norms, energy
# --------------------------------------------------------------------------

def ip2(f, g, h):
    """(f, g)_2 = h^3 sum f g over one period."""
    return h ** 3 * float(np.sum(f * g))


def face_ip(f, g, axis, h):
    """[f, g]_x = (a_x(f g), 1)_2 for face functions f, g."""
    return ip2(op_a(f * g, axis), 1.0, h)


def norm2(v, h):
    return np.sqrt(ip2(v, v, h))


def norm_p(v, h, p):
    """||v||_p = ((|v|^p, 1)_2)^(1/p)."""
    return ip2(np.abs(v) ** p, 1.0, h) ** (1.0 / p)


def grad_norm2_sq(v, h):
    """||grad_h v||_2^2 = [D_x v, D_x v]_x + [D_y v, D_y v]_y + [D_z v, D_z v]_z."""
    return sum(face_ip(op_D(v, ax, h), op_D(v, ax, h), ax, h) for ax in AXES)


def energy(phi, h, eps):
    """Discrete energy F_h(phi), Eq. 2.1."""
    return (0.25 * norm_p(phi, h, 4) ** 4
            + 0.5 * (1.0 - eps) * norm2(phi, h) ** 2
            - grad_norm2_sq(phi, h)
            + 0.5 * norm2(lap(phi, h), h) ** 2)


def modified_energy(a, b, h, eps):
    """F_h(a) + 1/2 ||grad_h (a - b)||^2, the quantity bounded in Prop. 3.1."""
    return energy(a, h, eps) + 0.5 * grad_norm2_sq(a - b, h)


def mass(phi, h):
    """(phi, 1)_2 = h^3 sum phi."""
    return ip2(phi, 1.0, h)


# --------------------------------------------------------------------------
# Section 5: the split nonlinear system N(u) = S (Eqs. 5.4-5.10)
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Params:
    """Scheme and solver parameters.

    eps, tau: model epsilon and time step.  nu1, nu2: pre/post smoothing
    sweeps of Algorithm 1.  linearization: "newton" or "picard" (pointwise
    3x3 system).  coarsest: levels of this size or smaller (or odd) are solved
    exactly.  prolongation: "trilinear" or "constant".  cubic: False drops the
    cubic term (an oracle-only switch used for the Fourier closed form).

    mob: face mobilities of the current step (dict axis -> array), or None
    for M == 1.  mobility: (m0, m2) for the variable mobility
    M(phi) = m0 + m2 phi^2 evaluated by ``run`` at every step on the faces
    at A phi_*, phi_* = 3/2 phi^k - 1/2 phi^{k-1} (Section 5's scheme with
    the extrapolated argument), or None for M == 1.

    smoother: "rb" is the paper's red-black sweep on every level; "hybrid"
    keeps it on levels whose stiffness s = (6 tau/h^2)(18/h^4) is >= stiff_hi
    or <= stiff_lo and uses ``jacobi_factor`` times as many damped collective
    Jacobi sweeps (weight ``jacobi_weight``) on the levels in between, where
    the red-black sweep is unstable (its red/black mode-pair amplification
    exceeds 1) and its V-cycles stall or diverge.
    """
    eps: float
    tau: float
    nu1: int = 2
    nu2: int = 2
    linearization: str = "newton"
    coarsest: int = 4
    prolongation: str = "trilinear"
    cubic: bool = True
    mob: object = field(default=None, compare=False)
    mobility: object = field(default=None, compare=False)
    smoother: str = "hybrid"
    jacobi_weight: float = 0.7
    jacobi_factor: int = 2
    stiff_hi: float = 1000.0
    stiff_lo: float = 0.25


def cubic_f(a, b):
    """f(a) = (a+b)(a^2+b^2)/4 = phi^{k+1/2} (phi^2)^{k+1/2}, Eq. 5.2."""
    return 0.25 * (a + b) * (a * a + b * b)


def cubic_fprime(a, b):
    """d f / d a for f of ``cubic_f``."""
    return 0.75 * a * a + 0.5 * a * b + 0.25 * b * b


def operator_N(u, b, h, prm: Params):
    """N(u) of Eqs. 5.4-5.6 for u = (phi, mu, omega); b = phi^k."""
    phi, mu, om = u
    n1 = phi - prm.tau * div_M_grad(mu, h, prm.mob)
    cub = cubic_f(phi, b) if prm.cubic else 0.0
    n2 = mu - cub - 0.5 * (1.0 - prm.eps) * phi - lap(om, h)
    n3 = om - 0.5 * lap(phi, h)
    return [n1, n2, n3]


def source_S(b, c, h, prm: Params):
    """S of Eqs. 5.8-5.10; b = phi^k, c = phi^{k-1}."""
    s1 = b.copy()
    s2 = 0.5 * (1.0 - prm.eps) * b + 3.0 * lap(b, h) - lap(c, h)
    s3 = 0.5 * lap(b, h)
    return [s1, s2, s3]


def residual(S, u, b, h, prm: Params):
    """r = S - N(u) (Algorithm 1)."""
    n = operator_N(u, b, h, prm)
    return [s - x for s, x in zip(S, n)]


def rms(r):
    """RMS over the three residual components: sqrt(sum r^2 / (3 m^3))."""
    tot = sum(float(np.sum(x * x)) for x in r)
    return np.sqrt(tot / (len(r) * r[0].size))


# --------------------------------------------------------------------------
# Section 5: red-black nonlinear Gauss-Seidel with a pointwise 3x3 solve
# --------------------------------------------------------------------------

def det3(a11, a12, a13, a21, a22, a23, a31, a32, a33):
    """Determinant of a 3x3 matrix by cofactor expansion along the first row."""
    return (a11 * (a22 * a33 - a23 * a32)
            - a12 * (a21 * a33 - a23 * a31)
            + a13 * (a21 * a32 - a22 * a31))


def cramer3(A, rhs):
    """Solve A x = rhs by Cramer's rule; A is 3x3 nested lists of arrays/scalars."""
    (a11, a12, a13), (a21, a22, a23), (a31, a32, a33) = A
    r1, r2, r3 = rhs
    det = det3(a11, a12, a13, a21, a22, a23, a31, a32, a33)
    x1 = det3(r1, a12, a13, r2, a22, a23, r3, a32, a33) / det
    x2 = det3(a11, r1, a13, a21, r2, a23, a31, r3, a33) / det
    x3 = det3(a11, a12, r1, a21, a22, r2, a31, a32, r3) / det
    return x1, x2, x3


def neighbour_sum(v):
    """Sum of the six face neighbours of each cell (periodic)."""
    return sum(np.roll(v, s, ax) for ax in AXES for s in (1, -1))


def colour_mask(m):
    """Red (0) / black (1) colour of each cell: (i + j + k) mod 2."""
    k, j, i = np.indices((m, m, m))
    return (i + j + k) % 2


def level_stiffness(h, prm: Params):
    """s = kappa * 18/h^4 with kappa = 6 tau/h^2: the product of the
    couplings that close the phi -> omega -> mu -> phi cycle of the
    pointwise system relative to its identity part."""
    return 108.0 * prm.tau / h ** 6


def uses_jacobi(h, prm: Params):
    s = level_stiffness(h, prm)
    return prm.smoother == "hybrid" and prm.stiff_lo < s < prm.stiff_hi


def smooth(u, S, b, h, prm: Params, sweeps):
    """Smoothing of level h: ``sweeps`` red-black sweeps, or
    ``jacobi_factor * sweeps`` damped Jacobi sweeps on hybrid levels."""
    if uses_jacobi(h, prm):
        return jacobi_smooth(u, S, b, h, prm, sweeps * prm.jacobi_factor)
    return rb_smooth(u, S, b, h, prm, sweeps)


def point_system(phi, mu, om, S, b, h, prm: Params):
    """The Section 5 pointwise 3x3 system of every cell, with all six
    neighbours at their current values: returns (A, rhs) for Cramer's rule."""
    s1, s2, s3 = S
    g = 1.0 / (h * h)
    kap = prm.tau * g * face_mobility_sums(phi.shape, prm.mob)
    if prm.mob is None:
        flux_nb = neighbour_sum(mu)
    else:
        flux_nb = sum(prm.mob[ax] * np.roll(mu, -1, ax)
                      + np.roll(prm.mob[ax], 1, ax) * np.roll(mu, 1, ax)
                      for ax in AXES)
    st1 = s1 + prm.tau * g * flux_nb
    phin = phi
    if not prm.cubic:
        q = np.full_like(phi, 0.5 * (1.0 - prm.eps))
        extra = 0.0
    elif prm.linearization == "picard":
        p = 0.25 * (phin * phin + b * b)
        q = p + 0.5 * (1.0 - prm.eps)
        extra = p * b
    elif prm.linearization == "newton":
        fp = cubic_fprime(phin, b)
        q = fp + 0.5 * (1.0 - prm.eps)
        extra = cubic_f(phin, b) - fp * phin
    else:
        raise ValueError(prm.linearization)
    st2 = s2 + extra + g * neighbour_sum(om)
    st3 = s3 + 0.5 * g * neighbour_sum(phi)
    A = [[1.0, kap, 0.0],
         [-q, 1.0, 6.0 * g],
         [3.0 * g, 0.0, 1.0]]
    return A, (st1, st2, st3)


def jacobi_smooth(u, S, b, h, prm: Params, sweeps):
    """Damped collective Jacobi: every cell solves its 3x3 system with the
    neighbours of the previous sweep, and moves by ``jacobi_weight`` of the
    change."""
    phi, mu, om = (x.copy() for x in u)
    w = prm.jacobi_weight
    for _ in range(sweeps):
        A, rhs = point_system(phi, mu, om, S, b, h, prm)
        x1, x2, x3 = cramer3(A, rhs)
        phi = phi + w * (x1 - phi)
        mu = mu + w * (x2 - mu)
        om = om + w * (x3 - om)
    return [phi, mu, om]


def rb_smooth(u, S, b, h, prm: Params, sweeps):
    """``sweeps`` red-black nonlinear Gauss-Seidel sweeps (Section 5).

    For every cell of the active colour the 3x3 system

        [ 1            tau/h^2 sum M    0      ] [phi]   [S~1]
        [ -q           1                6/h^2  ] [mu ] = [S~2]
        [ 3/h^2        0                1      ] [om ]   [S~3]

    is solved by Cramer's rule with the neighbours held at their latest
    values.  With the paper's Picard linearisation q = (phi_n^2 + b^2)/4 +
    (1-eps)/2 and S~2 carries (phi_n^2 + b^2) b / 4; with the Newton variant
    q = f'(phi_n) + (1-eps)/2 and S~2 carries f(phi_n) - f'(phi_n) phi_n.
    All cells of one colour are updated together (for even m no two of them
    are neighbours).
    """
    phi, mu, om = (x.copy() for x in u)
    colour = colour_mask(phi.shape[0])
    for _ in range(sweeps):
        for col in (0, 1):
            sel = colour == col
            A, rhs = point_system(phi, mu, om, S, b, h, prm)
            x1, x2, x3 = cramer3(A, rhs)
            phi = np.where(sel, x1, phi)
            mu = np.where(sel, x2, mu)
            om = np.where(sel, x3, om)
    return [phi, mu, om]


# --------------------------------------------------------------------------
# Linearisation of N at u (used by the mixed-precision defect correction)
# --------------------------------------------------------------------------

def jacobian_coefficient(phi, b, prm: Params):
    """q = f'(phi) + (1-eps)/2: the only u-dependent entry of dN/du."""
    q = np.full_like(phi, 0.5 * (1.0 - prm.eps))
    if prm.cubic:
        q = q + cubic_fprime(phi, b)
    return q


def jacobian_apply(d, q, h, prm: Params):
    """J d for J = dN/du of Eqs. 5.4-5.6 with the coefficient field q."""
    dp, dm, dw = d
    j1 = dp - prm.tau * div_M_grad(dm, h, prm.mob)
    j2 = dm - q * dp - lap(dw, h)
    j3 = dw - 0.5 * lap(dp, h)
    return [j1, j2, j3]


def linear_point_system(d, r, q, h, prm: Params):
    """The pointwise 3x3 system of J d = r (q frozen, no cubic right-hand
    side term) with all neighbours at their current values."""
    dp, dm, dw = d
    r1, r2, r3 = r
    g = 1.0 / (h * h)
    kap = prm.tau * g * face_mobility_sums(dp.shape, prm.mob)
    st1 = r1 + prm.tau * g * neighbour_sum(dm)
    st2 = r2 + g * neighbour_sum(dw)
    st3 = r3 + 0.5 * g * neighbour_sum(dp)
    return [[1.0, kap, 0.0], [-q, 1.0, 6.0 * g], [3.0 * g, 0.0, 1.0]], (st1, st2, st3)


def linear_smooth(d, r, q, h, prm: Params, sweeps, kind="rb"):
    """Relaxation of J d = r with the Section 5 pointwise system: red-black
    Gauss-Seidel (kind "rb") or damped collective Jacobi (kind "jacobi",
    weight ``prm.jacobi_weight``)."""
    d = [x.copy() for x in d]
    colour = colour_mask(d[0].shape[0])
    for _ in range(sweeps):
        if kind == "jacobi":
            A, rhs = linear_point_system(d, r, q, h, prm)
            x = cramer3(A, rhs)
            d = [y + prm.jacobi_weight * (xn - y) for y, xn in zip(d, x)]
            continue
        for col in (0, 1):
            sel = colour == col
            A, rhs = linear_point_system(d, r, q, h, prm)
            x = cramer3(A, rhs)
            d = [np.where(sel, xn, y) for y, xn in zip(d, x)]
    return d


def linear_smooth_level(d, r, q, h, prm: Params, sweeps):
    """Level smoothing of J d = r under the same policy as ``smooth``."""
    if uses_jacobi(h, prm):
        return linear_smooth(d, r, q, h, prm, sweeps * prm.jacobi_factor, "jacobi")
    return linear_smooth(d, r, q, h, prm, sweeps, "rb")


# --------------------------------------------------------------------------
# Transfers between levels
# --------------------------------------------------------------------------

def restrict(v):
    """8-cell average onto the grid of twice the spacing."""
    m = v.shape[0]
    mc = m // 2
    return v.reshape(mc, 2, mc, 2, mc, 2).mean(axis=(1, 3, 5))


def _prolong_axis(v, ax):
    """Linear cell-centred interpolation along one axis: fine cell 2I takes
    3/4 v_I + 1/4 v_{I-1}, fine cell 2I+1 takes 3/4 v_I + 1/4 v_{I+1}."""
    lo = 0.75 * v + 0.25 * np.roll(v, 1, ax)
    hi = 0.75 * v + 0.25 * np.roll(v, -1, ax)
    out = np.stack([lo, hi], axis=ax + 1)
    shape = list(v.shape)
    shape[ax] *= 2
    return out.reshape(shape)


def prolong(vc, kind="trilinear"):
    """Coarse-to-fine interpolation: trilinear (tensor product of the 1-D
    cell-centred rule) or piecewise constant."""
    if kind == "constant":
        return np.repeat(np.repeat(np.repeat(vc, 2, 0), 2, 1), 2, 2)
    out = vc
    for ax in AXES:
        out = _prolong_axis(out, ax)
    return out


# --------------------------------------------------------------------------
# Dense Newton solve of N(u) = S (plain definition; also the coarsest solve)
# --------------------------------------------------------------------------

def laplacian_matrix(m, h):
    """Dense matrix of Delta_h on an m^3 periodic grid, built column by column
    by applying ``lap`` to unit grid functions."""
    n = m ** 3
    L = np.empty((n, n))
    e = np.zeros(n)
    for col in range(n):
        e[col] = 1.0
        L[:, col] = lap(e.reshape(m, m, m), h).ravel()
        e[col] = 0.0
    return L


def div_M_grad_matrix(m, h, mob):
    n = m ** 3
    if mob is None:
        return laplacian_matrix(m, h)
    K = np.empty((n, n))
    e = np.zeros(n)
    for col in range(n):
        e[col] = 1.0
        K[:, col] = div_M_grad(e.reshape(m, m, m), h, mob).ravel()
        e[col] = 0.0
    return K


def jacobian_dense(u, b, h, prm: Params, L=None, K=None):
    """Dense Jacobian dN/du of Eqs. 5.4-5.6 in the unknown order (phi, mu, om)."""
    m = u[0].shape[0]
    n = m ** 3
    if L is None:
        L = laplacian_matrix(m, h)
    if K is None:
        K = L if prm.mob is None else div_M_grad_matrix(m, h, prm.mob)
    I = np.eye(n)
    q = 0.5 * (1.0 - prm.eps) * np.ones(n)
    if prm.cubic:
        q = q + cubic_fprime(u[0], b).ravel()
    Z = np.zeros((n, n))
    return np.block([[I, -prm.tau * K, Z],
                     [-np.diag(q), I, -L],
                     [-0.5 * L, Z, I]])


def newton_dense(S, u0, b, h, prm: Params, tol=1e-14, max_iter=30):
    """Solve N(u) = S by Newton's method with a dense Jacobian and LU solve.

    Stops when the RMS residual is below ``tol`` times (1 + RMS of S), or
    when the Newton update stops shrinking.  Returns (u, iterations).
    """
    m = u0[0].shape[0]
    L = laplacian_matrix(m, h)
    K = L if prm.mob is None else div_M_grad_matrix(m, h, prm.mob)
    u = [x.copy() for x in u0]
    scale = 1.0 + rms(S)
    it = 0
    for it in range(1, max_iter + 1):
        r = residual(S, u, b, h, prm)
        if rms(r) <= tol * scale:
            return u, it - 1
        J = jacobian_dense(u, b, h, prm, L, K)
        du = np.linalg.solve(J, np.concatenate([x.ravel() for x in r]))
        n = m ** 3
        u = [u[i] + du[i * n:(i + 1) * n].reshape(m, m, m) for i in range(3)]
        if np.max(np.abs(du)) <= 1e-16 * (1.0 + max(np.max(np.abs(x)) for x in u)):
            return u, it
    return u, it


# --------------------------------------------------------------------------
# Algorithm 1: FAS V-cycle
# --------------------------------------------------------------------------

def is_coarsest(m, prm: Params):
    return m <= prm.coarsest or m % 2 == 1


def fas_vcycle(u, S, b, h, prm: Params):
    """One FAS V-cycle (Algorithm 1) on the level of spacing h.

    Pre-smooth, residual, restrict u, r and phi^k, form the coarse source
    S_c = N_c(I u) + I r, recurse (or solve exactly on the coarsest level),
    correct u += P(v_c - I u), post-smooth.
    """
    m = u[0].shape[0]
    if is_coarsest(m, prm):
        v, _ = newton_dense(S, u, b, h, prm)
        return v
    u = smooth(u, S, b, h, prm, prm.nu1)
    r = residual(S, u, b, h, prm)
    uc = [restrict(x) for x in u]
    rc = [restrict(x) for x in r]
    bc = restrict(b)
    hc = 2.0 * h
    prm_c = prm if prm.mob is None else replace(
        prm, mob={ax: restrict_face(prm.mob[ax], ax) for ax in AXES})
    Sc = [n + x for n, x in zip(operator_N(uc, bc, hc, prm_c), rc)]
    vc = fas_vcycle([x.copy() for x in uc], Sc, bc, hc, prm_c)
    u = [x + prolong(v - w, prm.prolongation) for x, v, w in zip(u, vc, uc)]
    u = smooth(u, S, b, h, prm, prm.nu2)
    return u


def restrict_face(w, ax):
    """Average of the four fine faces that make up one coarse face (for a
    variable mobility; unused when M == 1)."""
    m = w.shape[0]
    mc = m // 2
    # the coarse face I+1/2 along ax is the fine face 2I+1+1/2, i.e. index 2I+1
    sl = [slice(None)] * 3
    sl[ax] = slice(1, None, 2)
    wf = w[tuple(sl)]
    shp = [mc, 2, mc, 2, mc, 2]
    shp_ax = {AX_Z: 1, AX_Y: 3, AX_X: 5}[ax]
    shp[shp_ax] = 1
    return wf.reshape(shp).mean(axis=(1, 3, 5))


@dataclass
class StepResult:
    u: list
    cycles: int
    history: list


def solve_step(b, c, u0, h, prm: Params, tol, max_cycles=100):
    """Solve one time step of Eq. 1.10: V-cycles until RMS(S - N(u)) <= tol."""
    S = source_S(b, c, h, prm)
    u = [x.copy() for x in u0]
    res = rms(residual(S, u, b, h, prm))
    hist = [res]
    cycles = 0
    while res > tol and cycles < max_cycles:
        u = fas_vcycle(u, S, b, h, prm)
        cycles += 1
        res = rms(residual(S, u, b, h, prm))
        hist.append(res)
    return StepResult(u, cycles, hist)


def run(phi0, nsteps, h, prm: Params, tol, max_cycles=100, phi1=None,
        callback=None):
    """Advance Eq. 1.10 ``nsteps`` steps from phi^0.

    The first step uses phi^{-1} := phi^0 unless ``phi1`` (phi^1) is given, in
    which case stepping starts from the pair (phi^0, phi^1).  Each step starts
    from u = (phi^k, mu, omega) of the previous step (mu = omega = 0 at first).
    Returns (phi_k, phi_{k-1}, mu, omega, cycles_per_step).
    """
    c = phi0.copy()
    b = phi0.copy() if phi1 is None else phi1.copy()
    mu = np.zeros_like(b)
    om = np.zeros_like(b)
    cycles = []
    for k in range(nsteps):
        prm_k = prm
        if prm.mobility is not None:
            prm_k = replace(prm, mob=face_mobilities(b, c, *prm.mobility))
        res = solve_step(b, c, [b, mu, om], h, prm_k, tol, max_cycles)
        phi_new, mu, om = res.u
        cycles.append(res.cycles)
        if callback is not None:
            callback(k, phi_new, b, c, mu, om, res)
        c, b = b, phi_new
    return b, c, mu, om, cycles


# --------------------------------------------------------------------------
# Closed form of the scheme with the cubic term removed (Fourier diagonal)
# --------------------------------------------------------------------------

def laplacian_symbol(m, h):
    """Eigenvalue of Delta_h on the Fourier mode r: -(4/h^2) sum sin^2(pi r_d/m).

    This is |u_r|^2 summed over directions, with u_r = 2 i sin(pi r h/L)/h the
    symbol of D_x (Section 4.1)."""
    r = np.arange(m)
    s = np.sin(np.pi * r / m) ** 2
    return -(4.0 / (h * h)) * (s[:, None, None] + s[None, :, None]
                               + s[None, None, :])


def linear_step_fft(b, c, h, eps, tau):
    """phi^{k+1} of Eq. 1.10 without the cubic term, solved mode by mode:

        a^ = [b^(1 + tau lam((1-eps)/2 + 3 lam + lam^2/2)) - tau lam^2 c^]
             / (1 - tau lam ((1-eps)/2 + lam^2/2)).
    """
    m = b.shape[0]
    lam = laplacian_symbol(m, h)
    bh = np.fft.fftn(b)
    ch = np.fft.fftn(c)
    g = 0.5 * (1.0 - eps) + 0.5 * lam * lam
    ah = (bh * (1.0 + tau * lam * (g + 3.0 * lam)) - tau * lam * lam * ch) \
        / (1.0 - tau * lam * g)
    return np.real(np.fft.ifftn(ah))
