"""Host check of the fixed-point images used for exact stencil sums in the
FP64 defect kernel (csrc/pfc_fixed.cuh).

The header is plain C++ outside nvcc; this test compiles it with g++ into a
small shared library and compares its bit arithmetic with exact rational
arithmetic (fractions.Fraction): X = round(v 2^54) with halves away from
zero, X 2^-54 rounded to nearest-even binary64 (Python's float(Fraction) is
correctly rounded), and the exact integer Laplacian.
"""

import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_1611_06288_gb300", "csrc")
FRAC = 54

SRC = r"""
#include "pfc_fixed.cuh"
extern "C" {
long long t_fix_of(double v, int* ok) {
  bool b = true;
  long long x = (long long)pfc::fix_of(v, b);
  *ok = b ? 1 : 0;
  return x;
}
double t_fix_to_double(long long x) { return pfc::fix_to_double((int64_t)x); }
long long t_fix_lap(const long long* v) {
  return (long long)pfc::fix_lap(v[0], v[1], v[2], v[3], v[4], v[5], v[6]);
}
}
"""


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("fixed")
    src = d / "t.cpp"
    src.write_text(SRC)
    so = d / "t.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", HEADER_DIR,
                    str(src), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.t_fix_of.restype = ctypes.c_longlong
    lib.t_fix_of.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
    lib.t_fix_to_double.restype = ctypes.c_double
    lib.t_fix_to_double.argtypes = [ctypes.c_longlong]
    lib.t_fix_lap.restype = ctypes.c_longlong
    lib.t_fix_lap.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    return lib


def fix_of(lib, v):
    ok = ctypes.c_int(0)
    x = lib.t_fix_of(float(v), ctypes.byref(ok))
    return x, bool(ok.value)


def round_half_away(q: Fraction) -> int:
    a = abs(q)
    r = int(a)
    if a - r >= Fraction(1, 2):
        r += 1
    return r if q >= 0 else -r


def sample_values(rng, count):
    mags = 10.0 ** rng.uniform(-22, np.log10(31.999), count)
    vals = list(mags * rng.choice([-1.0, 1.0], count))
    # exact halves at the quantum, zeros, subnormals, the range edge
    q = 2.0 ** -FRAC
    vals += [0.0, -0.0, 5e-324, -5e-324, q / 2, -q / 2, 3 * q / 2, q / 4, q,
             31.999999999999996, -31.999999999999996, 1.0, -1.0, 0.1, 2.0 ** -53 + 1.0]
    return vals


def test_fix_of_matches_exact_rounding(fx):
    rng = np.random.default_rng(11)
    for v in sample_values(rng, 4000):
        x, ok = fix_of(fx, v)
        assert ok, v
        assert x == round_half_away(Fraction(v) * 2 ** FRAC), v


def test_fix_of_flags_out_of_range(fx):
    for v in [32.0, -32.0, 1e3, -7e300, float("inf"), float("-inf"), float("nan")]:
        _, ok = fix_of(fx, v)
        assert not ok, v


def test_fix_to_double_rounds_to_nearest_even(fx):
    rng = np.random.default_rng(12)
    xs = [int(x) for x in rng.integers(-(2 ** 62), 2 ** 62, 4000, dtype=np.int64)]
    xs += [int(x) >> int(s) for x, s in zip(rng.integers(-(2 ** 62), 2 ** 62, 2000,
                                                         dtype=np.int64),
                                           rng.integers(0, 62, 2000))]
    # ties: 53 significant bits followed by exactly a half (1000000000b, 63-bit
    # values), odd and even kept bits, and a carry into the exponent
    for top in [(1 << 52) + 1, (1 << 52) + 2, (1 << 53) - 1]:
        xs += [(top << 10) | 0x200, -((top << 10) | 0x200), (top << 10) | 0x201,
               (top << 10) | 0x1FF, (top << 3) | 0x4, (top << 3) | 0x5]
    xs += [1, -1, 2 ** 53, 2 ** 53 + 1, 2 ** 62 + 2 ** 61, 0]
    for x in xs:
        assert fx.t_fix_to_double(x) == float(Fraction(x, 2 ** FRAC)), x


def test_laplacian_is_exact_for_quantised_inputs(fx):
    rng = np.random.default_rng(13)
    arr = (ctypes.c_longlong * 7)()
    for _ in range(2000):
        vals = rng.uniform(-31.99, 31.99, 7) * 10.0 ** rng.integers(-6, 1)
        xs = []
        for k, v in enumerate(vals):
            x, ok = fix_of(fx, v)
            assert ok
            xs.append(x)
            arr[k] = x
        exact = sum(xs[:6]) - 6 * xs[6]
        assert fx.t_fix_lap(arr) == exact
        got = fx.t_fix_to_double(fx.t_fix_lap(arr))
        assert got == float(Fraction(exact, 2 ** FRAC))
        # within the stated bound of the true Laplacian of the FP64 inputs
        true = sum(Fraction(v) for v in vals[:6]) - 6 * Fraction(vals[6])
        assert abs(Fraction(got) - true) <= 12 * Fraction(1, 2 ** 55) + abs(true) * 2 ** -53
