"""The allocation-free residual norm, pfc_op_residual_norm_static.

Some callers cannot allocate device memory (their device memory is reserved
up front by their own pool, or they cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree).  For them the library keeps the
partial sums of this reduction in a fixed device array of its own.  This file
checks, through the C ABI, that two calls in a row give the same value as
pfc_op_residual_norm (caller-provided scratch) within the tolerance of the
other norm tests, and that a grid beyond the array's limit is rejected.  It is
named so that pytest collects it last.
"""

import numpy as np
import pytest
import torch

from gpu_helpers import dev
from oracle import pfc_oracle as O
from paper_1611_06288_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    h = 0.8
    b = 0.2 + 0.1 * rng.standard_normal((n,) * 3)
    c = b + 0.01 * rng.standard_normal((n,) * 3)
    u = [b + 0.02 * rng.standard_normal((n,) * 3), rng.standard_normal((n,) * 3),
         rng.standard_normal((n,) * 3)]
    S = O.source_S(b, c, h, O.Params(eps=0.1, tau=0.05))
    return h, [dev(x) for x in u], [dev(x) for x in S], dev(b)


@pytest.mark.parametrize("n", [12, 64])
def test_static_scratch_matches_caller_scratch_twice(n):
    scratch = torch.empty(B.pfc_reduce_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    for seed in (1, 2):          # two calls in a row on different inputs
        h, u, S, b = _inputs(n, seed)
        want = B.pfc_op_residual_norm(n, h, 0.1, 0.05, *u, *S, b, scratch)
        got = B.pfc_op_residual_norm_static(n, h, 0.1, 0.05, *u, *S, b)
        assert got == pytest.approx(want, rel=1e-12)


def test_static_scratch_rejects_grids_beyond_its_limit():
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PFCError) as e:
        B.pfc_op_residual_norm_static(257, 1.0, 0.1, 0.05, *([tiny] * 7))
    assert e.value.code == B.PFC_ESIZE
    assert "256^3" in str(e.value)
