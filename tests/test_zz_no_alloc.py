"""The allocation-free residual norm, pfc_op_residual_norm_static.

Some callers cannot allocate device memory (their device memory is reserved
up front by their own pool, or they cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree).  For them the library keeps the
partial sums of this reduction in a fixed device array of its own.  This file
checks, through the C ABI, that calls in a row -- a larger grid, a smaller
one, the larger again, and a grid at the array's limit of 256^3 cells -- give
the oracle's RMS residual and the value of pfc_op_residual_norm (caller
scratch), that both entry points check their arguments alike, and that a grid
beyond the limit is rejected.  It is named so that pytest collects it last.
"""

import numpy as np
import pytest
import torch

from gpu_helpers import dev
from oracle import pfc_oracle as O
from paper_1611_06288_gb300 import binding as B

pytestmark = pytest.mark.gpu

EPS, TAU = 0.1, 0.05


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    h = 0.8
    b = 0.2 + 0.1 * rng.standard_normal((n,) * 3)
    c = b + 0.01 * rng.standard_normal((n,) * 3)
    u = [b + 0.02 * rng.standard_normal((n,) * 3), rng.standard_normal((n,) * 3),
         rng.standard_normal((n,) * 3)]
    S = O.source_S(b, c, h, O.Params(eps=EPS, tau=TAU))
    want = O.rms(O.residual(S, u, b, h, O.Params(eps=EPS, tau=TAU)))
    return h, [dev(x) for x in u], [dev(x) for x in S], dev(b), want


def _check(n, seed):
    h, u, S, b, oracle = _inputs(n, seed)
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    other = B.pfc_op_residual_norm(n, h, EPS, TAU, *u, *S, b, scratch)
    got = B.pfc_op_residual_norm_static(n, h, EPS, TAU, *u, *S, b)
    # FP64 sums in another order than the oracle's: a few ulps of the norm
    assert got == pytest.approx(oracle, rel=1e-12)
    assert got == pytest.approx(other, rel=1e-12)


def test_static_scratch_matches_oracle_and_caller_scratch_in_a_row():
    # larger grid, then a smaller one (slots beyond its tiles still hold the
    # larger grid's partial sums), then the larger one again
    for n, seed in ((64, 1), (12, 2), (64, 3), (12, 4)):
        _check(n, seed)


def test_static_scratch_at_its_limit():
    _check(256, 5)
    _check(256, 6)


def test_both_entry_points_check_arguments_alike():
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(2), dtype=torch.uint8, device="cuda")
    for n, h in ((1, 1.0), (2, 0.0), (2, -1.0)):
        codes = []
        for fn, extra in ((B.pfc_op_residual_norm, (scratch,)),
                          (B.pfc_op_residual_norm_static, ())):
            with pytest.raises(B.PFCError) as e:
                fn(n, h, EPS, TAU, *([t] * 7), *extra)
            codes.append(e.value.code)
        assert codes == [B.PFC_EINVAL, B.PFC_EINVAL], (n, h, codes)


def test_static_scratch_rejects_grids_beyond_its_limit():
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PFCError) as e:
        B.pfc_op_residual_norm_static(257, 1.0, EPS, TAU, *([tiny] * 7))
    assert e.value.code == B.PFC_ESIZE
    assert "256^3" in str(e.value)
