"""The integer-only FP64 <-> FP32 conversions of the FP32 path, checked on the CPU.

The kernels convert the FP64 cell averages to FP32 and back with integer
operations on the IEEE-754 bit patterns (``f32_bits_of_f64`` and
``f64_words_of_f32`` in ``csrc/dg_physics.cuh``, host and device functions).
This test compiles those two functions for the host with nvcc and compares them
with numpy's IEEE conversions: rounding to nearest with ties away from zero,
non-finite values and out-of-range magnitudes keeping their class (a NaN stays a
NaN, |x| >= 2^128 after rounding becomes an infinity), subnormal results
flushed to a signed zero.  No GPU is needed.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1305_5536_gb300", "csrc")

_SRC = r"""
#include "dg_physics.cuh"
extern "C" void f64_to_f32_bits(const unsigned long long* x, unsigned* out, long n) {
  for (long i = 0; i < n; ++i)
    out[i] = dgk::f32_bits_of_f64((unsigned)(x[i] >> 32), (unsigned)(x[i] & 0xffffffffull));
}
extern "C" void f32_to_f64_bits(const unsigned* u, unsigned long long* out, long n) {
  for (long i = 0; i < n; ++i) {
    unsigned hi, lo;
    dgk::f64_words_of_f32(u[i], hi, lo);
    out[i] = ((unsigned long long)hi << 32) | lo;
  }
}
"""


@pytest.fixture(scope="module")
def conv(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and not shutil.which(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("cvt")
    src = d / "cvt.cu"
    src.write_text(_SRC)
    lib = d / "libcvt.so"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I", CSRC,
                    str(src), "-o", str(lib)], check=True, capture_output=True)
    L = ctypes.CDLL(str(lib))
    vp, cl = ctypes.c_void_p, ctypes.c_long
    L.f64_to_f32_bits.argtypes = [vp, vp, cl]
    L.f32_to_f64_bits.argtypes = [vp, vp, cl]

    def to32(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros(x.size, dtype=np.uint32)
        L.f64_to_f32_bits(x.ctypes.data, out.ctypes.data, x.size)
        return out.view(np.float32)

    def to64(f):
        f = np.ascontiguousarray(f, dtype=np.float32)
        out = np.zeros(f.size, dtype=np.uint64)
        L.f32_to_f64_bits(f.ctypes.data, out.ctypes.data, f.size)
        return out.view(np.float64)

    return to32, to64


def _round_half_away(x):
    """FP32 rounding of doubles to nearest with ties away from zero (reference):
    numpy rounds ties to even, so exact ties that went toward zero are moved one
    ulp away."""
    with np.errstate(over="ignore"):
        f = x.astype(np.float32)
    fd = f.astype(np.float64)
    away = np.nextafter(f, np.float32(np.inf) * np.sign(f)).astype(np.float64)
    tie = np.isfinite(fd) & (np.abs(x - fd) == np.abs(away - x)) & (np.abs(fd) < np.abs(x))
    return np.where(tie, away.astype(np.float32), f)


def test_special_values_keep_their_class(conv):
    to32, _ = conv
    with np.errstate(invalid="ignore"):
        snan = np.array([0x7ff0000000000001], dtype=np.uint64).view(np.float64)[0]
        nan_lo_only = np.array([0x7ff0000000000100], dtype=np.uint64).view(np.float64)[0]
    x = np.array([np.inf, -np.inf, np.nan, -np.nan, snan, nan_lo_only, 1e300, -1e300,
                  2.0 ** 128, -(2.0 ** 200), 0.0, -0.0, 1e-300, -1e-300, 5e-324])
    r = to32(x)
    assert r[0] == np.inf and r[1] == -np.inf
    assert np.isnan(r[2:6]).all()
    assert r[6] == np.inf and r[7] == -np.inf and r[8] == np.inf and r[9] == -np.inf
    # below the float range: signed zeros
    assert (r[10:] == 0).all()
    assert not np.signbit(r[10]) and np.signbit(r[11])
    assert np.signbit(r[13]) and not np.signbit(r[12])


def test_overflow_threshold(conv):
    to32, _ = conv
    fmax = float(np.finfo(np.float32).max)
    half_ulp = 2.0 ** (127 - 24)
    below = np.nextafter(fmax + half_ulp, 0.0)  # rounds down to FLT_MAX
    x = np.array([fmax, below, fmax + half_ulp, -fmax, -(fmax + half_ulp)])
    r = to32(x)
    assert r[0] == np.float32(fmax) and r[1] == np.float32(fmax)
    assert r[2] == np.inf  # the tie rounds away from zero, to 2^128
    assert r[3] == -np.float32(fmax) and r[4] == -np.inf


def test_normal_range_rounds_to_nearest_ties_away(conv):
    to32, _ = conv
    rng = np.random.default_rng(1305)
    e = rng.uniform(-125.0, 127.5, 400_000)
    x = np.sign(rng.uniform(-1, 1, e.size)) * 2.0 ** e
    # exact ties: a float plus half its ulp
    f = rng.uniform(1.0, 2.0, 50_000).astype(np.float32)
    ties = f.astype(np.float64) + np.spacing(f).astype(np.float64) / 2.0
    x = np.concatenate([x, ties, -ties, [2.0 ** -126, np.nextafter(2.0 ** -126, 0.0)]])
    got = to32(x)
    ref = _round_half_away(x)
    ref = np.where(np.abs(x) < 2.0 ** -126 * (1 - 2.0 ** -25), np.float32(0.0) * np.sign(x), ref)
    np.testing.assert_array_equal(got.view(np.uint32), ref.astype(np.float32).view(np.uint32))


def test_widening_is_exact_and_keeps_specials(conv):
    _, to64 = conv
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 2 ** 32, 400_000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    got = to64(f)
    fin = np.isfinite(f) & (np.abs(f) >= np.finfo(np.float32).tiny)
    np.testing.assert_array_equal(got[fin], f[fin].astype(np.float64))
    nan = np.isnan(f)
    assert np.isnan(got[nan]).all()
    inf = np.isinf(f)
    np.testing.assert_array_equal(got[inf], f[inf].astype(np.float64))
    sub = np.isfinite(f) & (np.abs(f) < np.finfo(np.float32).tiny)
    assert (got[sub] == 0).all()
    np.testing.assert_array_equal(np.signbit(got[sub]), np.signbit(f[sub]))
    special = np.array([np.inf, -np.inf, np.nan, 0.0, -0.0], dtype=np.float32)
    g = to64(special)
    assert g[0] == np.inf and g[1] == -np.inf and np.isnan(g[2]) and g[3] == 0 and g[4] == 0
