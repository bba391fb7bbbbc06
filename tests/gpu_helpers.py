"""Shared helpers of the GPU tests: numpy <-> CUDA tensors and tolerances."""

import numpy as np
import torch


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def empty(n, dtype=torch.float64):
    return torch.empty((n, n, n), dtype=dtype, device="cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_close_field(got, ref, rtol, what=""):
    """max |got - ref| <= rtol * max(|ref|, 1): element by element."""
    scale = max(float(np.abs(ref).max()), 1.0)
    err = float(np.abs(got - ref).max())
    assert err <= rtol * scale, f"{what}: max err {err:.3e} > {rtol:.1e} * {scale:.3e}"


def split_perm(n):
    """Position of every natural-order cell in the colour-split FP32 layout:
    within each x-row the cells with (i+j+k) even come first (by i//2), then
    the odd ones."""
    k, j, i = np.indices((n, n, n))
    return ((k * n + j) * n + ((i + j + k) & 1) * (n // 2) + (i >> 1)).ravel()


def to_split(x):
    n = x.shape[0]
    y = np.empty(x.size, dtype=x.dtype)
    y[split_perm(n)] = x.ravel()
    return y.reshape(x.shape)


def from_split(y):
    n = y.shape[0]
    return y.ravel()[split_perm(n)].reshape(y.shape)


def to_df(x):
    """FP64 array -> double-float pairs (..., 2) float32: hi = FP32 rounding of
    x, lo = FP32 rounding of x - hi (the remainder is exact in FP64)."""
    x = np.asarray(x, dtype=np.float64)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return np.stack([hi, lo], axis=-1)


def from_df(y):
    """Double-float pairs -> FP64 values hi + lo (exact)."""
    y = np.asarray(y)
    return y[..., 0].astype(np.float64) + y[..., 1].astype(np.float64)


def dev_df(x):
    return torch.from_numpy(np.ascontiguousarray(to_df(x))).to("cuda")


def host_df(t):
    torch.cuda.synchronize()
    return from_df(t.detach().cpu().numpy())
