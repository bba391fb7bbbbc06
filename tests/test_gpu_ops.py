"""Parity of every CUDA stage of the V-cycle with the CPU oracle, through the
C ABI, element by element, on seeded inputs.  Sizes span several thread
blocks with a ragged tail (12^3 = 1728 cells = 6.75 blocks of 256) and the
smallest levels (2^3, 4^3)."""

import numpy as np
import pytest
import torch

from gpu_helpers import (assert_close_field, dev, dev_df, empty, from_df, from_split, host,
                         host_df, split_perm, to_df, to_split)
from oracle import pfc_oracle as O
from paper_1611_06288_gb300 import binding as B

pytestmark = pytest.mark.gpu

SIZES = [2, 4, 12, 32]
EPS, TAU = 0.1, 0.05
# FP64 stages differ from the oracle only by rounding order and FMA
# contraction: a few ulps of the largest term.  The Laplacian amplifies by
# up to 12/h^2 relative to the field, hence the h-dependent scale.
FP64_RTOL = 1e-12
# Double-float stages (unit roundoff u = 2^-48): each of the <= 16 df
# operations on the path to a value adds at most ~3u of its operands, and the
# largest operand is a neighbour sum times 1/h^2 (about 6 max|field| / h^2 <=
# 10 at these sizes), so the absolute error is below 16 * 3 * 3.6e-15 * 10
# ~ 1.7e-12 against a scale max(|ref|, 1) >= 1.
DF_RTOL = 2e-12


def case(n, seed=0):
    rng = np.random.default_rng(1000 + n + seed)
    L = 0.8 * n
    h = L / n
    b = 0.2 + 0.1 * rng.standard_normal((n, n, n))
    c = b + 0.01 * rng.standard_normal((n, n, n))
    u = [b + 0.02 * rng.standard_normal((n, n, n)), rng.standard_normal((n, n, n)),
         rng.standard_normal((n, n, n))]
    return h, b, c, u


def prm(lin="newton"):
    return O.Params(eps=EPS, tau=TAU, linearization=lin)


@pytest.mark.parametrize("n", SIZES)
def test_source(n):
    h, b, c, _ = case(n)
    S2, S3 = empty(n), empty(n)
    B.pfc_op_source(n, h, EPS, dev(b), dev(c), S2, S3)
    ref = O.source_S(b, c, h, prm())
    assert_close_field(host(S2), ref[1], FP64_RTOL, "S2")
    assert_close_field(host(S3), ref[2], FP64_RTOL, "S3")


@pytest.mark.parametrize("n", [2, 4, 12, 32])
@pytest.mark.parametrize("lin", ["newton", "picard"])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_smooth(n, lin, sweeps):
    h, b, c, u = case(n)
    S = O.source_S(b, c, h, prm(lin))
    d = [dev(x) for x in u]
    B.pfc_op_smooth(n, h, EPS, TAU, B.PFC_NEWTON if lin == "newton" else B.PFC_PICARD,
                    sweeps, *d, *[dev(s) for s in S], dev(b))
    ref = O.rb_smooth(u, S, b, h, prm(lin), sweeps)
    for g, r, name in zip(d, ref, ("phi", "mu", "om")):
        assert_close_field(host(g), r, FP64_RTOL, name)


@pytest.mark.parametrize("n", SIZES)
def test_residual(n):
    h, b, c, u = case(n)
    S = O.source_S(b, c, h, prm())
    r = [empty(n) for _ in range(3)]
    B.pfc_op_residual(n, h, EPS, TAU, *[dev(x) for x in u], *[dev(s) for s in S], dev(b), *r)
    ref = O.residual(S, u, b, h, prm())
    for g, x in zip(r, ref):
        assert_close_field(host(g), x, FP64_RTOL, "r")


@pytest.mark.parametrize("n", [2, 4, 12, 32])
def test_residual_restrict_and_restrict(n):
    h, b, c, u = case(n)
    S = O.source_S(b, c, h, prm())
    nc = n // 2
    rc = [empty(nc) for _ in range(3)]
    uc = [empty(nc) for _ in range(3)]
    B.pfc_op_residual_restrict(n, h, EPS, TAU, *[dev(x) for x in u], *[dev(s) for s in S],
                               dev(b), *rc, *uc)
    ref_r = [O.restrict(x) for x in O.residual(S, u, b, h, prm())]
    for g, x in zip(rc, ref_r):
        assert_close_field(host(g), x, FP64_RTOL, "rc")
    for g, x in zip(uc, u):
        assert_close_field(host(g), O.restrict(x), 1e-15, "uc")
    bc = empty(nc)
    B.pfc_op_restrict(n, dev(b), bc)
    assert_close_field(host(bc), O.restrict(b), 1e-15, "bc")


@pytest.mark.parametrize("nc", [1, 2, 6, 16])
def test_coarse_source(nc):
    h, b, c, u = case(nc)
    rng = np.random.default_rng(7)
    r = [rng.standard_normal((nc,) * 3) for _ in range(3)]
    d = [dev(x) for x in r]
    B.pfc_op_coarse_source(nc, h, EPS, TAU, *[dev(x) for x in u], dev(b), *d)
    ref = [n_ + x for n_, x in zip(O.operator_N(u, b, h, prm()), r)]
    for g, x in zip(d, ref):
        assert_close_field(host(g), x, FP64_RTOL, "Sc")


@pytest.mark.parametrize("n", [2, 4, 12, 32])
def test_prolong_correct(n):
    rng = np.random.default_rng(3 + n)
    nc = n // 2
    v = [rng.standard_normal((nc,) * 3) for _ in range(3)]
    w = [rng.standard_normal((nc,) * 3) for _ in range(3)]
    u = [rng.standard_normal((n,) * 3) for _ in range(3)]
    du = [dev(x) for x in u]
    B.pfc_op_prolong_correct(n, *[dev(x) for x in v], *[dev(x) for x in w], *du)
    for g, x, vv, ww in zip(du, u, v, w):
        assert_close_field(host(g), x + O.prolong(vv - ww), 1e-14, "u+Pe")


@pytest.mark.parametrize("n", [4, 12, 32])
@pytest.mark.parametrize("lin", ["newton", "picard"])
@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_jacobi(n, lin, sweeps):
    h, b, c, u = case(n)
    p = prm(lin)
    S = O.source_S(b, c, h, p)
    d = [dev(x) for x in u]
    t = [empty(n) for _ in range(3)]
    B.pfc_op_jacobi(n, h, EPS, TAU, B.PFC_NEWTON if lin == "newton" else B.PFC_PICARD,
                    sweeps, 0.7, *d, *t, *[dev(s_) for s_ in S], dev(b))
    ref = O.jacobi_smooth(u, S, b, h, p, sweeps)
    for g, r, name in zip(d, ref, ("phi", "mu", "om")):
        assert_close_field(host(g), r, FP64_RTOL, name)


@pytest.mark.parametrize("n", [2, 4, 8])
@pytest.mark.parametrize("lin", ["newton", "picard"])
@pytest.mark.parametrize("kind", ["rb", "jacobi"])
def test_coarse_solve(n, lin, kind):
    """The coarsest-level solve reaches the unique solution of N(u) = S that the
    oracle's dense Newton solve finds."""
    L = 2.0 * n           # coarse spacing 2
    h = L / n
    rng = np.random.default_rng(11)
    b = 0.2 + 0.1 * rng.standard_normal((n,) * 3)
    c = b + 0.01 * rng.standard_normal((n,) * 3)
    p = prm(lin)
    S = O.source_S(b, c, h, p)
    ref, _ = O.newton_dense(S, [b, 0 * b, 0 * b], b, h, p)
    d = [dev(b), dev(0 * b), dev(0 * b)]
    t = [empty(n) for _ in range(3)]
    B.pfc_op_coarse_solve(n, h, EPS, TAU, B.PFC_NEWTON if lin == "newton" else B.PFC_PICARD,
                          B.PFC_SWEEP_RB if kind == "rb" else B.PFC_SWEEP_JACOBI, 0.7, 2000,
                          *d, *t, *[dev(s) for s in S], dev(b))
    got = [host(x) for x in d]
    assert O.rms(O.residual(S, got, b, h, p)) < 1e-12
    for g, r in zip(got, ref):
        assert_close_field(g, r, 1e-11, "coarse")


@pytest.mark.parametrize("n", [4, 12, 32])
def test_diagnostics_and_residual_norm(n):
    h, b, c, u = case(n)
    a = u[0]
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    out = B.pfc_op_diagnostics(n, h, EPS, dev(a), dev(b), scratch)
    assert out[0] == pytest.approx(O.energy(a, h, EPS), rel=1e-12)
    assert out[1] == pytest.approx(O.modified_energy(a, b, h, EPS), rel=1e-12)
    assert out[2] == pytest.approx(O.mass(a, h), rel=1e-12)
    assert out[3] == pytest.approx(O.grad_norm2_sq(a, h), rel=1e-12)
    S = O.source_S(b, c, h, prm())
    rms = B.pfc_op_residual_norm(n, h, EPS, TAU, *[dev(x) for x in u], *[dev(s) for s in S],
                                 dev(b), scratch)
    assert rms == pytest.approx(O.rms(O.residual(S, u, b, h, prm())), rel=1e-12)


@pytest.mark.parametrize("n", SIZES)
def test_diagnostics_df(n):
    """Energy, modified energy, mass and |grad a|^2 of df fields: every term
    and sum in double-float, so 1e-12 relative like the FP64 kernel."""
    h, b, c, u = case(n)
    a, b = from_df(to_df(u[0])), from_df(to_df(b))
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    out = B.pfc_op_diagnostics_df(n, h, EPS, dev_df(a), dev_df(b), scratch)
    assert out[0] == pytest.approx(O.energy(a, h, EPS), rel=1e-12)
    assert out[1] == pytest.approx(O.modified_energy(a, b, h, EPS), rel=1e-12)
    assert out[2] == pytest.approx(O.mass(a, h), rel=1e-12)
    assert out[3] == pytest.approx(O.grad_norm2_sq(a, h), rel=1e-12)


def guess_ref(b, c, h):
    """The extrapolated initial iterate written out from its definition:
    phi = 2b - c, omega = Lap(phi + b)/2 (row 3), mu from row 2."""
    S = O.source_S(b, c, h, prm())
    phi = 2 * b - c
    om = 0.5 * O.lap(phi + b, h)
    mu = S[1] + O.cubic_f(phi, b) + 0.5 * (1 - EPS) * phi + O.lap(om, h)
    return S, phi, mu, om


@pytest.mark.parametrize("n", SIZES)
def test_guess(n):
    h, b, c, _ = case(n)
    S, phi, mu, om = guess_ref(b, c, h)
    out = [empty(n) for _ in range(5)]
    B.pfc_op_guess(n, h, EPS, dev(b), dev(c), *out)
    for g, x, name in zip(out, [S[1], S[2], phi, mu, om], ("S2", "S3", "phi", "mu", "om")):
        assert_close_field(host(g), x, FP64_RTOL, name)
    # the iterate satisfies rows 2 and 3 of N(u) = S: only row 1 is left
    r = O.residual(S, [host(out[2]), host(out[3]), host(out[4])], b, h, prm())
    scale = max(float(np.abs(host(out[3])).max()), 1.0)
    assert float(np.abs(r[1]).max()) <= 1e-12 * scale
    assert float(np.abs(r[2]).max()) <= 1e-12 * scale


@pytest.mark.parametrize("n", SIZES)
def test_guess_df(n):
    h, b, c, _ = case(n)
    b, c = from_df(to_df(b)), from_df(to_df(c))
    S, phi, mu, om = guess_ref(b, c, h)
    out = [torch.empty((n, n, n, 2), dtype=torch.float32, device="cuda") for _ in range(5)]
    B.pfc_op_guess_df(n, h, EPS, dev_df(b), dev_df(c), *out)
    for g, x, name in zip(out, [S[1], S[2], phi, mu, om], ("S2", "S3", "phi", "mu", "om")):
        assert_close_field(host_df(g), x, DF_RTOL, name)


def test_integer_pipe_conversions():
    """FP64 -> FP32 rounding and FP32 -> FP64 widening formed from the bit
    fields: bit-exact against numpy's IEEE conversions (round to nearest,
    ties to even) on random values over the whole float range, exact ties
    (odd and even kept bits), carries into the exponent, overflow to
    infinity, the normal/subnormal boundary, zeros, infinities and NaN."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal(200000) * 10.0 ** rng.uniform(-45, 45, 200000)
    f = rng.standard_normal(2000).astype(np.float32)
    # exact halfway points between f and its neighbour away from zero
    ties = f.astype(np.float64) + np.spacing(f).astype(np.float64) / 2
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0 ** -126,
                        2.0 ** -126 * (1 - 2 ** -30), 2.0 ** -149, 2.0 ** -150, 1e-300,
                        3.4028234663852886e38, 3.4028235677973366e38, 3.5e38, 1e300,
                        1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 2.0 - 2.0 ** -25, 0.1, 1.0 / 3])
    xs = np.concatenate([x, ties, -ties, special])
    y = torch.empty(xs.size, dtype=torch.float32, device="cuda")
    B.pfc_op_round_f32(xs.size, dev(xs), y)
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):
        ref = xs.astype(np.float32)
    got = y.cpu().numpy()
    same = (got.view(np.uint32) == ref.view(np.uint32)) | (np.isnan(got) & np.isnan(ref))
    assert same.all(), xs[~same][:5]
    fs = np.concatenate([f, np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-40,
                                      1.1754944e-38, 3.4028235e38], np.float32),
                         (rng.standard_normal(50000) * 10.0 ** rng.uniform(-37, 37, 50000))
                         .astype(np.float32)])
    w = torch.empty(fs.size, dtype=torch.float64, device="cuda")
    B.pfc_op_widen_f64(fs.size, dev(fs, torch.float32), w)
    torch.cuda.synchronize()
    gw = w.cpu().numpy()
    rw = fs.astype(np.float64)
    same = (gw.view(np.uint64) == rw.view(np.uint64)) | (np.isnan(gw) & np.isnan(rw))
    assert same.all(), fs[~same][:5]


@pytest.mark.parametrize("n", [1, 2, 12, 32])
def test_df_conversions(n):
    """FP64 -> (hi, lo) pairs and back, out of place and in place: bit-exact
    against the same roundings on the host, over 40 decades of magnitude."""
    rng = np.random.default_rng(77 + n)
    x = rng.standard_normal((n,) * 3) * 10.0 ** rng.uniform(-20, 20, (n,) * 3)
    xd = dev(x)
    y = torch.empty((n, n, n, 2), dtype=torch.float32, device="cuda")
    B.pfc_op_df_from_f64(n ** 3, xd, y)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.cpu().numpy(), to_df(x))
    back = empty(n)
    B.pfc_op_df_to_f64(n ** 3, y, back)
    np.testing.assert_array_equal(host(back), from_df(to_df(x)))
    B.pfc_op_df_from_f64(n ** 3, xd, xd)            # in place, 8-byte slots
    torch.cuda.synchronize()
    np.testing.assert_array_equal(xd.view(torch.float32).reshape(n, n, n, 2).cpu().numpy(),
                                  to_df(x))
    B.pfc_op_df_to_f64(0, None, None)
    with pytest.raises(B.PFCError):
        B.pfc_op_df_to_f64(-1, y, back)


@pytest.mark.parametrize("n", SIZES)
def test_source_df(n):
    h, b, c, _ = case(n)
    S2 = torch.empty((n, n, n, 2), dtype=torch.float32, device="cuda")
    S3 = torch.empty_like(S2)
    B.pfc_op_source_df(n, h, EPS, dev_df(b), dev_df(c), S2, S3)
    ref = O.source_S(from_df(to_df(b)), from_df(to_df(c)), h, prm())
    assert_close_field(host_df(S2), ref[1], DF_RTOL, "S2")
    assert_close_field(host_df(S3), ref[2], DF_RTOL, "S3")


def check_defect(n, h, b, c, u):
    """pfc_op_defect against the oracle's FP64 residual (Eqs. 5.4-5.6) and
    Newton coefficient, both rounded to FP32, and the Laplacian of phi."""
    S = O.source_S(b, c, h, prm())
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    r = [empty(n, torch.float32) for _ in range(3)]
    q = empty(n, torch.float32)
    lap = empty(n)
    rms = B.pfc_op_defect(n, h, EPS, TAU, *[dev(x) for x in u], *[dev(s) for s in S], dev(b),
                          *r, q, scratch, lap=lap)
    ref = O.residual(S, u, b, h, prm())
    assert rms == pytest.approx(O.rms(ref), rel=1e-5)
    assert_close_field(host(lap), h * h * O.lap(u[0], h), FP64_RTOL, "lap")
    for g, x in zip(r, ref):
        assert_close_field(from_split(host(g)), x, 2 ** -23, "r32")
    # q feeds only the FP32 preconditioner and is formed in FP32 from phi and
    # b rounded to FP32: 2 input roundings (each doubled in the squares) and
    # five operation roundings of 2^-24 against terms that sum to at most
    # about twice q (q >= c1 > 0): below 16 * 2^-24 = 2^-20 of max |q|
    assert_close_field(from_split(host(q)), O.jacobian_coefficient(u[0], b, prm()), 2 ** -20,
                       "q32")


def check_start_extrap(n, h, b, c, u0, u1):
    """pfc_op_start_extrap against the oracle: the iterate 2 u^k - u^{k-1},
    S2, S3 (Eqs. 5.9-5.10), the residual of the iterate (Eqs. 5.4-5.6) and
    q rounded to FP32, and the iterate's Laplacians."""
    L = lambda x: h * h * O.lap(x, h)                     # unscaled Laplacian
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    r = [empty(n, torch.float32) for _ in range(3)]
    q = empty(n, torch.float32)
    S2, S3, phi, lap = empty(n), empty(n), empty(n), empty(n)
    mu1, om1, lmu1, lom1 = dev(u1[1]), dev(u1[2]), dev(L(u1[1])), dev(L(u1[2]))
    rms = B.pfc_op_start_extrap(n, h, EPS, TAU, dev(b), dev(c), dev(L(b)), dev(L(c)),
                                dev(u0[1]), dev(u0[2]), dev(L(u0[1])), dev(L(u0[2])),
                                mu1, om1, lmu1, lom1, S2, S3, phi, lap, *r, q, scratch)
    ug = [2 * b - c, 2 * u0[1] - u1[1], 2 * u0[2] - u1[2]]
    S = O.source_S(b, c, h, prm())
    ref = O.residual(S, ug, b, h, prm())
    assert rms == pytest.approx(O.rms(ref), rel=1e-5)
    assert_close_field(host(S2), S[1], FP64_RTOL, "S2")
    assert_close_field(host(S3), S[2], FP64_RTOL, "S3")
    for got, x, what in ((phi, ug[0], "phi"), (mu1, ug[1], "mu"), (om1, ug[2], "omega")):
        assert_close_field(host(got), x, FP64_RTOL, what)
    for got, x, what in ((lap, ug[0], "lap phi"), (lmu1, ug[1], "lap mu"),
                         (lom1, ug[2], "lap omega")):
        assert_close_field(host(got), L(x), FP64_RTOL, what)
    for g, x in zip(r, ref):
        assert_close_field(from_split(host(g)), x, 2 ** -23, "r32")
    assert_close_field(from_split(host(q)), O.jacobian_coefficient(ug[0], b, prm()), 2 ** -20,
                       "q32")


@pytest.mark.parametrize("n", SIZES + [48])
def test_start_extrap(n):
    """The pointwise start from the three-field extrapolation (the Laplacians
    of the iterate as combinations of the stored ones)."""
    h, b, c, u0 = case(n)
    _, _, _, u1 = case(n, seed=1)
    check_start_extrap(n, h, b, c, u0, u1)


def test_start_extrap_values_beyond_fixed_point_range():
    """A cell with phi^{k-1} = 33 (and so a Laplacian of phi^{k-1} beyond 32)
    takes the FP64 form of the fixed-point combinations; large mu^{k-1}
    (40) and Lap omega^k (48) enter FP64 arithmetic as always."""
    n = 12
    h, b, c, u0 = case(n, seed=4)
    _, _, _, u1 = case(n, seed=5)
    u1[1][3, 4:7, 5] = 40.0
    u0[2][7, 7, 7] = -8.0          # its unscaled Laplacian's centre term: -6 * -8 = 48
    c[1, 2, 3] = 33.0
    check_start_extrap(n, h, b, c, u0, u1)


def test_defect_values_beyond_fixed_point_range():
    """The defect's neighbour sums run in 64-bit fixed point for |v| < 32; a
    block that meets larger values (here mu = 40 in a few cells of one plane,
    phi = -50 in one cell of another, n = 48: partial x tiles and several
    z chunks) evaluates in FP64 from that plane on, with the same result."""
    n = 48
    h, b, c, u = case(n, seed=3)
    u[1][20, 5:9, 30] = 40.0
    u[0][7, 40, 2] = -50.0
    check_defect(n, h, b, c, u)


@pytest.mark.parametrize("n", [2, 4, 12, 32, 48])
def test_defect_and_correct(n):
    """FP64 outer loop (PFC_MIXED): FP64 residual and Newton coefficient
    rounded to FP32, FP64 update."""
    h, b, c, u = case(n)
    S = O.source_S(b, c, h, prm())
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    r = [empty(n, torch.float32) for _ in range(3)]
    q = empty(n, torch.float32)
    lap = empty(n)
    rms = B.pfc_op_defect(n, h, EPS, TAU, *[dev(x) for x in u], *[dev(s) for s in S], dev(b),
                          *r, q, scratch, lap=lap)
    ref = O.residual(S, u, b, h, prm())
    # |r|^2 of the FP32-rounded r, summed in FP32 within a block: ~1e-6
    assert rms == pytest.approx(O.rms(ref), rel=1e-5)
    # the unscaled Laplacian of phi kept for the sources and diagnostics
    assert_close_field(host(lap), h * h * O.lap(u[0], h), FP64_RTOL, "lap")
    for g, x in zip(r, ref):
        # FP64 residual rounded to FP32: half an FP32 ulp (colour-split layout)
        assert_close_field(from_split(host(g)), x, 2 ** -23, "r32")
    # q in FP32 from FP32-rounded phi and b (bound derived in check_defect)
    assert_close_field(from_split(host(q)), O.jacobian_coefficient(u[0], b, prm()), 2 ** -20,
                       "q32")
    # u += d: one FP64 rounding of the same sum on both sides -> bit-exact
    rng = np.random.default_rng(5)
    d = [rng.standard_normal((n,) * 3).astype(np.float32) for _ in range(3)]
    du = [dev(x) for x in u]
    B.pfc_op_correct(n, *du, *[dev(to_split(x), torch.float32) for x in d])
    for g, x, y in zip(du, u, d):
        np.testing.assert_array_equal(host(g), x + y.astype(np.float64))


@pytest.mark.parametrize("n", [2, 4, 12, 32])
def test_defect_and_correct_df(n):
    h, b, c, u = case(n)
    # the oracle sees exactly the values the df fields hold
    b = from_df(to_df(b))
    u = [from_df(to_df(x)) for x in u]
    S = [from_df(to_df(x)) for x in O.source_S(b, c, h, prm())]
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    r = [empty(n, torch.float32) for _ in range(3)]
    q = empty(n, torch.float32)
    lap = torch.empty((n, n, n, 2), dtype=torch.float32, device="cuda")
    rms = B.pfc_op_defect_df(n, h, EPS, TAU, *[dev_df(x) for x in u], *[dev_df(s) for s in S],
                          dev_df(b), *r, q, scratch, lap=lap)
    assert_close_field(host_df(lap), h * h * O.lap(u[0], h), DF_RTOL, "lap")
    ref = O.residual(S, u, b, h, prm())
    # |r|^2 summed in FP32 within a thread block: relative error ~1e-6
    assert rms == pytest.approx(O.rms(ref), rel=1e-5)
    for g, x in zip(r, ref):
        # df residual (error ~DF_RTOL) rounded to FP32: half an FP32 ulp
        assert_close_field(from_split(host(g)), x, 2 ** -23, "r32")
    # q = f'(phi) + (1-eps)/2 is formed in FP32 arithmetic: a few FP32 ulps
    assert_close_field(from_split(host(q)), O.jacobian_coefficient(u[0], b, prm()), 1e-6,
                       "q32")
    # u += d in double-float: |error| <= ~2u (|u| + |u + d|), u = 2^-48
    rng = np.random.default_rng(5)
    d = [rng.standard_normal((n,) * 3).astype(np.float32) for _ in range(3)]
    du = [dev_df(x) for x in u]
    B.pfc_op_correct_df(n, *du, *[dev(to_split(x), torch.float32) for x in d])
    for g, x, y in zip(du, u, d):
        exact = x + y.astype(np.float64)
        err = np.abs(host_df(g) - exact)
        assert np.all(err <= 4 * 2.0 ** -48 * (np.abs(x) + np.abs(exact)) + 1e-300)
    with pytest.raises(B.PFCError):
        B.pfc_op_correct_df(3, *du, *r)                  # n must be even


@pytest.mark.parametrize("n", [4, 12, 32])
@pytest.mark.parametrize("zero", [False, True])
def test_linear_residual_restrict_fp32(n, zero):
    """I (r - J d) in FP32 (block sums: the Laplacians' interior faces cancel
    over the eight children) against the oracle's restrict(r - J d) in FP64,
    colour-split on both levels; d = 0 for the zero-start variant."""
    h, b, c, u = case(n)
    p = prm()
    rng = np.random.default_rng(21 + n)
    q = O.jacobian_coefficient(u[0], b, p).astype(np.float32)
    r = [rng.standard_normal((n,) * 3).astype(np.float32) for _ in range(3)]
    d = [np.zeros((n,) * 3, np.float32) if zero else
         (0.1 * rng.standard_normal((n,) * 3)).astype(np.float32) for _ in range(3)]
    f64 = lambda xs: [x.astype(np.float64) for x in xs]
    ref = [O.restrict(x) for x in
           (np.array(rr) - jd for rr, jd in zip(f64(r), O.jacobian_apply(f64(d), q.astype(np.float64), h, p)))]
    nc = n // 2
    cc = [empty(nc, torch.float32) for _ in range(3)]
    dd = [dev(to_split(x), torch.float32) for x in d]
    B.pfc_op_lin_residual_restrict(n, h, EPS, TAU, zero, *(None, None, None) if zero else dd,
                                   *[dev(to_split(x), torch.float32) for x in r],
                                   None if zero else dev(to_split(q), torch.float32), *cc)
    # FP32 sums of O(1) terms scaled by up to 12/h^2 ~ 19: a few FP32 ulps of that
    for g, x in zip(cc, ref):
        assert_close_field(from_split(host(g)), x, 2e-6, "rho")


@pytest.mark.parametrize("n", [4, 12, 32, 72])
@pytest.mark.parametrize("assign", [False, True])
@pytest.mark.parametrize("skip0", [False, True])
def test_linear_prolong_fp32(n, assign, skip0):
    """d += P e (or d = P e) in FP32, three one-dimensional passes, against
    the oracle's trilinear prolongation in FP64 (colour-split layouts).  With
    PFC_PROLONG_SKIP_COLOUR0 the colour-1 cells are the same and the colour-0
    cells keep their input bits (NaN where d = P e: they are not read)."""
    rng = np.random.default_rng(31 + n)
    nc = n // 2
    e = [rng.standard_normal((nc,) * 3).astype(np.float32) for _ in range(3)]
    d0 = [rng.standard_normal((n,) * 3).astype(np.float32) for _ in range(3)]
    dd = [dev(to_split(x), torch.float32) for x in d0]
    if assign:
        for t in dd:
            t.fill_(float("nan"))            # must not be read
    before = [host(t).copy() for t in dd]
    flags = (B.PFC_PROLONG_ASSIGN if assign else 0) | (B.PFC_PROLONG_SKIP_COLOUR0 if skip0 else 0)
    B.pfc_op_lin_prolong(n, flags, *[dev(to_split(x), torch.float32) for x in e], *dd)
    i, j, k = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    colour1 = ((i + j + k) & 1) == 1                     # natural-order mask
    for g, x, y, b0 in zip(dd, d0, e, before):
        ref = O.prolong(y.astype(np.float64)) + (0.0 if assign else x.astype(np.float64))
        got = from_split(host(g))
        if not skip0:
            assert_close_field(got, ref, 1e-6, "d+Pe")
            continue
        assert_close_field(np.where(colour1, got, 0.0), np.where(colour1, ref, 0.0), 1e-6,
                           "colour 1 of d+Pe")
        # colour 0 untouched: the first half of every colour-split row
        half = n // 2
        gs = host(g).reshape(n * n, n)
        assert np.array_equal(gs[:, :half], b0.reshape(n * n, n)[:, :half], equal_nan=True)


@pytest.mark.parametrize("skip0", [False, True])
def test_linear_prolong_fp32_multiplane(skip0):
    """At 204^3 the kernel's blocks take eight coarse planes each (102 coarse
    planes: 12 full chunks and a ragged one of six), and the grid's last x
    tile (6 of 32 columns) and last y tile (2 of 4 rows) are ragged: d += P e
    against the oracle."""
    n, nc = 204, 102
    rng = np.random.default_rng(5)
    e = [rng.standard_normal((nc,) * 3).astype(np.float32) for _ in range(3)]
    d0 = [rng.standard_normal((n,) * 3).astype(np.float32) for _ in range(3)]
    dd = [dev(to_split(x), torch.float32) for x in d0]
    B.pfc_op_lin_prolong(n, B.PFC_PROLONG_SKIP_COLOUR0 if skip0 else 0,
                         *[dev(to_split(x), torch.float32) for x in e], *dd)
    i, j, k = np.indices((n,) * 3)
    colour1 = ((i + j + k) & 1) == 1
    for g, x, y in zip(dd, d0, e):
        ref = O.prolong(y.astype(np.float64)) + x.astype(np.float64)
        got = from_split(host(g))
        if skip0:
            assert_close_field(np.where(colour1, got, 0.0), np.where(colour1, ref, 0.0), 1e-6,
                               "colour 1 of d+Pe")
            assert np.array_equal(np.where(colour1, 0.0, got), np.where(colour1, 0.0, x))
        else:
            assert_close_field(got, ref, 1e-6, "d+Pe")


@pytest.mark.parametrize("n", [32, 64, 96, 128])
@pytest.mark.parametrize("kind", ["rb", "jacobi"])
@pytest.mark.parametrize("assign", [False, True])
def test_prolong_smooth_fused_equals_separate(n, kind, assign):
    """The fused way up (d (+)= P e formed in shared memory inside the first
    post-smoothing pass) against pfc_op_lin_prolong followed by one sweep of
    pfc_op_lin_smooth / pfc_op_lin_jacobi: equal bit for bit, including the
    periodic halo of every tile (32^3: 128-thread tiles of 32 x 4 x 2 cells;
    larger: 32 x 8 x 4; 96^3 has three tiles across)."""
    rng = np.random.default_rng(n + (7 if assign else 0) + (3 if kind == "rb" else 0))
    nc, h, w = n // 2, 32.0 / n, 0.7
    f32 = lambda a: dev(a.astype(np.float32).ravel(), torch.float32)
    e = [f32(rng.standard_normal(nc ** 3)) for _ in range(3)]
    d0 = [rng.standard_normal(n ** 3) for _ in range(3)]
    r = [f32(rng.standard_normal(n ** 3)) for _ in range(3)]
    q = f32(0.3 + 0.1 * rng.standard_normal(n ** 3))
    code = B.PFC_SWEEP_RB if kind == "rb" else B.PFC_SWEEP_JACOBI
    # separate entry points
    ds = [f32(x) for x in d0]
    ts = [torch.empty_like(x) for x in ds]
    B.pfc_op_lin_prolong(n, B.PFC_PROLONG_ASSIGN if assign else 0, *e, *ds)
    if kind == "rb":
        B.pfc_op_lin_smooth(n, h, EPS, TAU, 1, False, *ds, *r, q)
    else:
        B.pfc_op_lin_jacobi(n, h, EPS, TAU, 1, w, False, *ds, *ts, *r, q)
    # fused
    df = [f32(x) for x in d0]
    if assign:
        for t in df:
            t.fill_(float("nan"))             # d = P e: the old values are not read
    tf = [torch.empty_like(x) for x in df]
    B.pfc_op_lin_prolong_smooth(n, h, EPS, TAU, code, assign, w, *e, *df, *tf, *r, q)
    torch.cuda.synchronize()
    for a, b in zip(ds, df):
        assert torch.equal(a, b)
        assert torch.isfinite(a).all()


@pytest.mark.parametrize("n,sweeps", [(4, 1), (12, 1), (64, 2), (128, 1)])
def test_smooth_with_folded_correction_equals_separate(n, sweeps):
    """Red-black sweeps whose last colour-1 pass adds d to the FP64 state u
    (the last pass of a correction's last V-cycle) against pfc_op_lin_smooth
    followed by pfc_op_correct: u equal bit for bit, d's colour-0 cells
    equal (its colour-1 cells are not written by the folded pass)."""
    rng = np.random.default_rng(100 + n + sweeps)
    h = 32.0 / n
    f32 = lambda a: dev(a.astype(np.float32).ravel(), torch.float32)
    d0 = [rng.standard_normal(n ** 3) for _ in range(3)]
    r = [f32(rng.standard_normal(n ** 3)) for _ in range(3)]
    q = f32(0.3 + 0.1 * rng.standard_normal(n ** 3))
    u0 = [rng.standard_normal(n ** 3) for _ in range(3)]
    ds, us = [f32(x) for x in d0], [dev(x) for x in u0]
    B.pfc_op_lin_smooth(n, h, EPS, TAU, sweeps, False, *ds, *r, q)
    B.pfc_op_correct(n, *us, *ds)
    df, uf = [f32(x) for x in d0], [dev(x) for x in u0]
    B.pfc_op_lin_smooth_correct(n, h, EPS, TAU, sweeps, *df, *r, q, *uf)
    torch.cuda.synchronize()
    for a, b in zip(us, uf):
        assert torch.equal(a, b)
    half = n // 2
    for a, b in zip(ds, df):
        assert torch.equal(a.view(n * n, n)[:, :half], b.view(n * n, n)[:, :half])


def test_prolong_smooth_fused_checks_its_size():
    z = torch.zeros(48 ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(B.PFCError) as exc:
        B.pfc_op_lin_prolong_smooth(48, 1.0, EPS, TAU, B.PFC_SWEEP_RB, False, 0.7,
                                    *([z] * 13))
    assert exc.value.code == B.PFC_EINVAL


def test_linear_prolong_rejects_unknown_flags():
    z = torch.zeros(8 ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(B.PFCError):
        B.pfc_op_lin_prolong(8, 4, z[:64], z[:64], z[:64], z, z, z)


@pytest.mark.parametrize("n", [4, 12, 32])
@pytest.mark.parametrize("zero_init", [True, False])
def test_linear_smoother_fp32(n, zero_init):
    h, b, c, u = case(n)
    p = prm()
    q = O.jacobian_coefficient(u[0], b, p).astype(np.float32)
    rng = np.random.default_rng(9)
    r = [rng.standard_normal((n,) * 3).astype(np.float32) for _ in range(3)]
    d0 = [np.zeros((n,) * 3) if zero_init else 0.1 * rng.standard_normal((n,) * 3)
          for _ in range(3)]
    d0 = [x.astype(np.float32) for x in d0]
    dd = [dev(to_split(x), torch.float32) for x in d0]
    if zero_init:                       # contents must not matter
        for t in dd:
            t.fill_(float("nan"))
    B.pfc_op_lin_smooth(n, h, EPS, TAU, 2, zero_init, *dd,
                        *[dev(to_split(x), torch.float32) for x in r],
                        dev(to_split(q), torch.float32))
    ref = O.linear_smooth([x.astype(np.float64) for x in d0],
                          [x.astype(np.float64) for x in r], q.astype(np.float64), h, p, 2)
    for g, x in zip(dd, ref):
        assert_close_field(from_split(host(g)), x, 1e-5, "d32")


@pytest.mark.parametrize("n", [4, 12, 32])
@pytest.mark.parametrize("zero_init", [True, False])
@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_linear_jacobi_fp32(n, zero_init, sweeps):
    h, b, c, u = case(n)
    p = prm()
    q = O.jacobian_coefficient(u[0], b, p).astype(np.float32)
    rng = np.random.default_rng(19)
    r = [rng.standard_normal((n,) * 3).astype(np.float32) for _ in range(3)]
    d0 = [np.zeros((n,) * 3, np.float32) if zero_init
          else (0.1 * rng.standard_normal((n,) * 3)).astype(np.float32) for _ in range(3)]
    dd = [dev(to_split(x), torch.float32) for x in d0]
    if zero_init:
        for t_ in dd:
            t_.fill_(float("nan"))
    tt = [empty(n, torch.float32) for _ in range(3)]
    B.pfc_op_lin_jacobi(n, h, EPS, TAU, sweeps, 0.7, zero_init, *dd, *tt,
                        *[dev(to_split(x), torch.float32) for x in r],
                        dev(to_split(q), torch.float32))
    ref = O.linear_smooth([x.astype(np.float64) for x in d0], [x.astype(np.float64) for x in r],
                          q.astype(np.float64), h, p, sweeps, "jacobi")
    for g, x in zip(dd, ref):
        assert_close_field(from_split(host(g)), x, 1e-5, "d32")


@pytest.mark.parametrize("n", [2, 4, 12])
def test_split_layout_is_a_permutation(n):
    perm = split_perm(n)
    assert sorted(perm.tolist()) == list(range(n ** 3))
    x = np.arange(n ** 3, dtype=np.float64).reshape((n,) * 3)
    np.testing.assert_array_equal(from_split(to_split(x)), x)


@pytest.mark.parametrize("n,levels", [(32, 2), (64, 3), (96, 3)])
@pytest.mark.parametrize("zero", [False, True])
def test_restrict_chain_equals_separate_restrictions(n, levels, zero):
    """The V-cycle's descent without pre-smoothing in one launch: the first
    restriction I (r - J d) and one or two further 8-cell averages, bit for
    bit the separate restrictions (each coarser level from d = 0), and the
    first level against the oracle as in the single restriction's test."""
    h, b, c, u = case(n)
    p = prm()
    rng = np.random.default_rng(41 + n)
    q = O.jacobian_coefficient(u[0], b, p).astype(np.float32)
    r = [rng.standard_normal((n,) * 3).astype(np.float32) for _ in range(3)]
    d = [np.zeros((n,) * 3, np.float32) if zero else
         (0.1 * rng.standard_normal((n,) * 3)).astype(np.float32) for _ in range(3)]
    dd = [dev(to_split(x), torch.float32) for x in d]
    rd = [dev(to_split(x), torch.float32) for x in r]
    qd = dev(to_split(q), torch.float32)
    sizes = [n // 2, n // 4, n // 8][:levels]
    chain = [[empty(m, torch.float32) for _ in range(3)] for m in sizes]
    B.pfc_op_lin_restrict_chain(n, h, EPS, TAU, zero, levels, *(None, None, None) if zero else dd,
                                *rd, None if zero else qd, *chain[0], *chain[1],
                                *(chain[2] if levels == 3 else (None, None, None)))
    # separate launches: the first restriction, then zero-start restrictions
    sep = [[empty(m, torch.float32) for _ in range(3)] for m in sizes]
    B.pfc_op_lin_residual_restrict(n, h, EPS, TAU, zero, *(None, None, None) if zero else dd,
                                   *rd, None if zero else qd, *sep[0])
    for lv in range(1, levels):
        m = n >> lv
        B.pfc_op_lin_residual_restrict(m, 2.0 ** lv * h, EPS, TAU, True, None, None, None,
                                       *sep[lv - 1], None, *sep[lv])
    for lv in range(levels):
        for x, y in zip(chain[lv], sep[lv]):
            assert torch.equal(x, y), (lv, n)
    # the last level is the average of the first one's cells over blocks
    first = [from_split(host(x)).astype(np.float64) for x in sep[0]]
    k = 2 ** (levels - 1)
    for x, y in zip(first, sep[levels - 1]):
        m = x.shape[0] // k
        avg = x.reshape(m, k, m, k, m, k).mean(axis=(1, 3, 5))
        assert_close_field(from_split(host(y)), avg, 1e-6, "chained average")


def test_restrict_chain_rejects_bad_sizes():
    z = torch.zeros(48 ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(B.PFCError):           # n / 2 not a multiple of 16
        B.pfc_op_lin_restrict_chain(48, 0.5, EPS, TAU, True, 2, None, None, None, z, z, z, None,
                                    z, z, z, z, z, z)
    with pytest.raises(B.PFCError):           # levels out of range
        B.pfc_op_lin_restrict_chain(64, 0.5, EPS, TAU, True, 4, None, None, None, z, z, z, None,
                                    z, z, z, z, z, z, z, z, z)


def _restrict_f32(x):
    """8-cell average in float32, children summed in the kernels' order
    (x fastest, then y, then z), natural layout [k, j, i]."""
    acc = np.zeros(tuple(s // 2 for s in x.shape), np.float32)
    for s in range(8):
        acc = (acc + x[(s >> 2)::2, ((s >> 1) & 1)::2, (s & 1)::2]).astype(np.float32)
    return (np.float32(0.125) * acc).astype(np.float32)


@pytest.mark.parametrize("n,levels", [(12, 1), (32, 2), (64, 3), (128, 3)])
def test_restrict_q_chain_is_bit_exact(n, levels):
    """pfc_op_restrict_q (the one-launch restriction of the Newton coefficient
    q to the coarse levels of the FP32 correction solve) equals the chain of
    single-level float32 8-cell averages bit for bit."""
    rng = np.random.default_rng(40 + n)
    q = (0.2 + rng.random((n, n, n))).astype(np.float32)
    outs = [torch.empty((n >> (l + 1)) ** 3, dtype=torch.float32, device="cuda")
            for l in range(levels)]
    B.pfc_op_restrict_q(n, levels, dev(to_split(q), torch.float32).reshape(-1), *outs)
    torch.cuda.synchronize()
    want = q
    for l in range(levels):
        want = _restrict_f32(want)
        got = from_split(outs[l].cpu().numpy().reshape((n >> (l + 1),) * 3))
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), l
