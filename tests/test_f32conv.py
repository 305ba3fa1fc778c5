"""The integer FP64 -> FP32 conversion (csrc/f32conv.h) against IEEE 754
round-to-nearest-even as numpy implements it, bit for bit, and the exact
FP32 -> FP64 widening beside it.  The header is host
and device code; here it is compiled for the host with the system C++ compiler."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_03110_gb300", "csrc")

SHIM = r'''
#include "f32conv.h"
extern "C" void conv(const double* x, float* y, long n)
{
    for (long i = 0; i < n; ++i) y[i] = mhe::f32_rn(x[i]);
}
extern "C" void widen(const float* x, double* y, long n)
{
    for (long i = 0; i < n; ++i) y[i] = mhe::f64_of(x[i]);
}
'''


@pytest.fixture(scope="module")
def conv():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "shim.cpp")
    so = os.path.join(d, "shim.so")
    open(src, "w").write(SHIM)
    subprocess.run([cxx, "-O2", "-shared", "-fPIC", "-I", CSRC, src, "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.conv.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long]
    L.widen.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long]

    def f(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(x.size, dtype=np.float32)
        L.conv(x.ctypes.data, y.ctypes.data, x.size)
        return y

    def g(x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.empty(x.size, dtype=np.float64)
        L.widen(x.ctypes.data, y.ctypes.data, x.size)
        return y
    f.widen = g
    yield f
    shutil.rmtree(d, ignore_errors=True)


def _same_bits(a, b):
    a, b = a.view(np.uint32), b.view(np.uint32)
    nan = np.isnan(a.view(np.float32)) & np.isnan(b.view(np.float32))
    return np.all((a == b) | nan)


def test_random_over_the_whole_exponent_range(conv):
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2**63, size=200000, dtype=np.uint64) | (rng.integers(0, 2, size=200000, dtype=np.uint64) << 63)
    x = bits.view(np.float64)
    with np.errstate(over="ignore", invalid="ignore"):
        assert _same_bits(conv(x), x.astype(np.float32))


def test_values_of_ordinary_size(conv):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(200000) * 10.0 ** rng.integers(-30, 30, size=200000)
    assert _same_bits(conv(x), x.astype(np.float32))


def test_ties_and_boundaries(conv):
    f = np.float32
    one = np.float64(1.0)
    ulp = 2.0 ** -23
    x = [0.0, -0.0, one, -one, one + ulp / 2, one + 3 * ulp / 2, one + ulp / 2 + 2.0 ** -40,
         one + ulp / 2 - 2.0 ** -40, float(np.finfo(f).max), float(np.finfo(f).max) * (1 + 2.0 ** -25),
         float(np.finfo(f).max) * (1 + 2.0 ** -24), float(np.finfo(f).tiny), float(np.finfo(f).tiny) * (1 - 2.0 ** -30),
         float(np.finfo(f).tiny) / 3, 2.0 ** -149, 2.0 ** -150, 2.0 ** -151, 1e-300, 1e300, -1e300,
         np.inf, -np.inf, np.nan, 2.0 ** 127 * (2 - 2.0 ** -24)]
    x = np.array(x, dtype=np.float64)
    with np.errstate(over="ignore"):
        assert _same_bits(conv(x), x.astype(np.float32))


def test_widening_is_exact(conv):
    rng = np.random.default_rng(2)
    bits = rng.integers(0, 2**32, size=200000, dtype=np.uint64).astype(np.uint32)
    x = np.concatenate([bits.view(np.float32),
                        np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan], dtype=np.float32),
                        np.array([2.0 ** -149, -(2.0 ** -126), 2.0 ** -126 * (1 - 2.0 ** -23)], dtype=np.float32),
                        np.finfo(np.float32).max.reshape(1)])
    y = conv.widen(x)
    with np.errstate(invalid="ignore"):
        ref = x.astype(np.float64)
    a, b = y.view(np.uint64), ref.view(np.uint64)
    assert np.all((a == b) | (np.isnan(y) & np.isnan(ref)))
