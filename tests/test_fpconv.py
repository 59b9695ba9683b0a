"""The library's FP64 <-> FP32 conversions and double-FP32 arithmetic (csrc/tg_fpconv.cuh),
compiled for the host from the same header the kernels include, against numpy's hardware
conversions and extended-precision references.

The kernels of the mixed precision convert on the integer pipes because GB300's FP64 pipe,
which also executes the conversion instructions, issues ~2 lanes per clock per SM.  These
tests pin the bit-level replacements: round-to-nearest-even FP64 -> FP32 (ties, the carry
into the exponent, the zero and subnormal bands, infinities, NaN), exact FP32 -> FP64, the
split x = hi + lo, and the double-FP32 tanh used for the elasticity force (relative error
about 3e-14: some twenty double-FP32 operations of ~2^-46 each)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1810_05370_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "native", "fpconv_check.cpp")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("fpc") / "fpc.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I", CSRC, SRC, "-o", out], check=True)
    L = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    L.tgc_f32_of.argtypes = [dp, fp, ctypes.c_long]
    L.tgc_f64_of.argtypes = [fp, dp, ctypes.c_long]
    L.tgc_f64_of_scaled.argtypes = [fp, dp, dp, ctypes.c_long]
    L.tgc_df_split.argtypes = [dp, fp, fp, ctypes.c_long]
    L.tgc_df_value.argtypes = [fp, fp, dp, ctypes.c_long]
    L.tgc_df_tanh.argtypes = [dp, dp, ctypes.c_long]
    L.tgc_df_div_mul.argtypes = [dp, dp, dp, dp, ctypes.c_long]
    L.tgc_cs_dot.argtypes = [dp, dp, dp, dp, ctypes.c_long, ctypes.c_long]
    return L


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def f32_of(L, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(x.shape, np.float32)
    L.tgc_f32_of(_p(x, ctypes.c_double), _p(out, ctypes.c_float), x.size)
    return out


def same_bits32(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_f32_of_matches_round_to_nearest_even(lib):
    rng = np.random.default_rng(0)
    # random bit patterns over every exponent (all classes: zero, subnormal, normal, inf, NaN)
    x = rng.integers(0, 2**64, size=400_000, dtype=np.uint64).view(np.float64)
    # values around the FP32 range ends and the subnormal band
    e = rng.uniform(-160, 130, size=200_000)
    y = np.ldexp(rng.uniform(1, 2, size=e.size), np.floor(e).astype(int)) * rng.choice([-1, 1], e.size)
    # exact ties between neighbouring FP32 numbers, and one FP64 ulp either side of them
    f = rng.uniform(-1e30, 1e30, size=100_000).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + g.astype(np.float64)) / 2
    ties = np.concatenate([mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)])
    # carries into the exponent (all-ones FP32 significand rounding up), and the largest finite
    carry = np.nextafter(np.float32(2.0) ** rng.integers(-120, 127, 1000).astype(np.float32),
                         np.float32(0)).astype(np.float64) + 2.0 ** -60
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 2.0**-150, -2.0**-150,
                        np.nextafter(2.0**-150, 1), 2.0**-149, 2.0**-126, np.nextafter(2.0**-126, 0),
                        3.4028234663852886e38, 3.4028235677973366e38, 2.0**128, 1e-300, 5e-324])
    for v in (x, y, ties, carry, special):
        with np.errstate(all="ignore"):
            ref = v.astype(np.float32)
        got = f32_of(lib, v)
        nan = np.isnan(ref)
        assert np.array_equal(np.isnan(got), nan)
        assert same_bits32(got[~nan], ref[~nan])


def test_f64_of_is_exact(lib):
    rng = np.random.default_rng(1)
    f = rng.integers(0, 2**32, size=400_000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    f = np.concatenate([f, np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-40,
                                     1.1754942e-38, 3.4028235e38], np.float32)])
    out = np.empty(f.shape, np.float64)
    lib.tgc_f64_of(_p(f, ctypes.c_float), _p(out, ctypes.c_double), f.size)
    with np.errstate(all="ignore"):
        ref = f.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(out), nan)
    assert np.array_equal(out[~nan].view(np.uint64), ref[~nan].view(np.uint64))


def test_f64_of_scaled_is_exact(lib):
    """f * 2^k by moving the exponent field, FP64 multiplication where that would leave the
    normal range (the inner solves' power-of-two right-hand-side scaling)."""
    rng = np.random.default_rng(6)
    f = (rng.standard_normal(200_000) * 10.0 ** rng.uniform(-30, 30, 200_000)).astype(np.float32)
    f[:5] = [0.0, -0.0, np.inf, np.nan, 1e-40]
    k = rng.integers(-1100, 1000, f.size)
    s = np.ldexp(1.0, np.clip(k, -1022, 1023))
    out = np.empty(f.shape, np.float64)
    lib.tgc_f64_of_scaled(_p(f, ctypes.c_float), _p(s, ctypes.c_double), _p(out, ctypes.c_double), f.size)
    with np.errstate(all="ignore"):
        ref = f.astype(np.float64) * s
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(out), nan)
    assert np.array_equal(out[~nan].view(np.uint64), ref[~nan].view(np.uint64))


def test_df_split_is_the_rounded_head_and_tail(lib):
    rng = np.random.default_rng(2)
    e = rng.uniform(-140, 120, size=300_000)
    x = np.ldexp(rng.uniform(1, 2, size=e.size), np.floor(e).astype(int)) * rng.choice([-1, 1], e.size)
    x = np.concatenate([x, [0.0, -0.0, 1.0, 1.0 + 2.0**-30, 0.1, -0.7, 2.0**-150, 1e-200]])
    hi = np.empty(x.shape, np.float32)
    lo = np.empty(x.shape, np.float32)
    lib.tgc_df_split(_p(x, ctypes.c_double), _p(hi, ctypes.c_float), _p(lo, ctypes.c_float), x.size)
    assert same_bits32(hi, x.astype(np.float32))
    tail = x - hi.astype(np.float64)   # exact in FP64
    ref = tail.astype(np.float32)
    normal = np.abs(ref) >= np.float32(2.0**-126)
    zero = ref == 0
    assert np.array_equal(lo[normal | zero], ref[normal | zero])
    # where the tail is FP32-subnormal it may be rounded twice: one subnormal step at most
    sub = ~(normal | zero)
    assert np.all(np.abs(lo[sub].astype(np.float64) - tail[sub]) <= 2.0**-149)
    # the pair carries x to 2^-48 relative (normal range)
    big = np.abs(x) > 2.0**-100
    err = np.abs(hi[big].astype(np.float64) + lo[big].astype(np.float64) - x[big])
    assert np.all(err <= 2.0**-48 * np.abs(x[big]))


def test_df_value_is_one_rounded_sum(lib):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100_000) * 10.0 ** rng.integers(-20, 20, 100_000)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    out = np.empty(x.shape, np.float64)
    lib.tgc_df_value(_p(hi, ctypes.c_float), _p(lo, ctypes.c_float), _p(out, ctypes.c_double), x.size)
    assert np.array_equal(out, hi.astype(np.float64) + lo.astype(np.float64))


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 60, reason="needs extended-precision long double")
def test_df_tanh_relative_error(lib):
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(-20, 20, 200_000), rng.uniform(0, 3, 200_000),
                        10.0 ** rng.uniform(-12, 0, 50_000), -(10.0 ** rng.uniform(-12, 0, 50_000)),
                        [0.0, 1e-30, 16.999, 17.0, 30.0, -17.5]])
    out = np.empty(x.shape, np.float64)
    lib.tgc_df_tanh(_p(x, ctypes.c_double), _p(out, ctypes.c_double), x.size)
    # the reference at the pair's own value hi + lo (the split is the input's only rounding)
    hi = x.astype(np.float32)
    s = hi.astype(np.longdouble) + (x - hi.astype(np.float64)).astype(np.float32).astype(np.longdouble)
    ref = np.tanh(s)
    rel = np.abs((out.astype(np.longdouble) - ref) / np.where(ref == 0, 1, ref))
    assert float(rel.max()) <= 5e-14, float(rel.max())
    nan = np.empty(1, np.float64)
    lib.tgc_df_tanh(_p(np.array([np.nan]), ctypes.c_double), _p(nan, ctypes.c_double), 1)
    assert np.isnan(nan[0])


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 60, reason="needs extended-precision long double")
def test_df_div_and_mul_relative_error(lib):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(200_000) * 10.0 ** rng.uniform(-8, 8, 200_000)
    y = rng.standard_normal(200_000) * 10.0 ** rng.uniform(-8, 8, 200_000)
    quo = np.empty(x.shape, np.float64)
    prod = np.empty(x.shape, np.float64)
    lib.tgc_df_div_mul(_p(x, ctypes.c_double), _p(y, ctypes.c_double), _p(quo, ctypes.c_double),
                       _p(prod, ctypes.c_double), x.size)

    def pair(v):
        h = v.astype(np.float32)
        return h.astype(np.longdouble) + (v - h.astype(np.float64)).astype(np.float32).astype(np.longdouble)

    a, b = pair(x), pair(y)
    assert float(np.max(np.abs((quo - a / b) / (a / b)))) <= 1e-13
    assert float(np.max(np.abs((prod - a * b) / (a * b)))) <= 1e-13


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 60, reason="needs extended-precision long double")
def test_compensated_residual_sum(lib):
    """b - sum of products with heavy cancellation, as in the elasticity residual of a nearly
    converged iterate: the error stays at ~2^-48 of the terms' magnitudes, far below the
    residual itself."""
    rng = np.random.default_rng(7)
    rows, m = 20_000, 21
    x = rng.uniform(0.5, 2.0, (rows, m)) * rng.choice([-1, 1], (rows, m))
    y = 1.0 + 1e-3 * rng.standard_normal((rows, m))
    # b equal to the products' sum up to a residual 1e-9 of their size
    pairs = lambda v: (v.astype(np.float32).astype(np.longdouble)
                       + (v - v.astype(np.float32).astype(np.float64)).astype(np.float32).astype(np.longdouble))
    prod = pairs(x) * pairs(y)
    exact_sum = prod.sum(axis=1)
    b = (exact_sum + np.abs(prod).sum(axis=1) * 1e-9 * rng.standard_normal(rows)).astype(np.float64)
    out = np.empty(rows, np.float64)
    lib.tgc_cs_dot(_p(b, ctypes.c_double), _p(np.ascontiguousarray(-x), ctypes.c_double),
                   _p(np.ascontiguousarray(y), ctypes.c_double), _p(out, ctypes.c_double), rows, m)
    ref = pairs(b) - exact_sum
    scale = np.abs(prod).sum(axis=1) + np.abs(pairs(b))
    err = np.abs(out.astype(np.longdouble) - ref) / scale
    # measured: median 1.5e-15, max 4.8e-14 of the terms' magnitudes (a double-FP32 product
    # and addition per term: 4.4e-16 and 6.4e-15, at 2.4 times the operations)
    assert float(np.median(err)) <= 2.0 ** -47, float(np.median(err))
    assert float(err.max()) <= 2.0 ** -42, float(err.max())
