"""The integer FP64 -> FP32 conversion (csrc/f32conv.h) against IEEE 754
round-to-nearest-even as numpy implements it, bit for bit.  The header is host
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

    def f(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(x.size, dtype=np.float32)
        L.conv(x.ctypes.data, y.ctypes.data, x.size)
        return y
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
