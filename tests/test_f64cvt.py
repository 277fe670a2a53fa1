"""The integer-pipe double-to-float rounding of `csrc/f64cvt.h`, checked on the CPU against
numpy's float32 conversion (IEEE round to nearest, ties to even).

The restriction kernels use it for every value of a residual they copy into FP32 local vectors, so
it must give exactly the bits of a conversion instruction wherever it claims a result, and it must
claim every double of magnitude in [2^-126, 2^128), the binary32 normal exponents (including the
rounding of the largest ones up to infinity).  The cases: random bit patterns over all doubles, random doubles across the float
range, exact ties in both parities, the normal range's edges, signed zeros, infinities and NaN."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_7227_gb300", "csrc")

SHIM = r'''
#include "f64cvt.h"
#include <cstring>
extern "C" void cvt_many(const double* in, unsigned* out, int* ok, long n) {
    for (long i = 0; i < n; i++) {
        unsigned long long b;
        std::memcpy(&b, &in[i], 8);
        unsigned f = 0;
        ok[i] = asm2::f64_to_f32_bits((unsigned)(b >> 32), (unsigned)b, f) ? 1 : 0;
        out[i] = f;
    }
}
'''


@pytest.fixture(scope="module")
def cvt(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("cvt")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    out = str(d / "libcvt.so")
    subprocess.run([cxx, "-std=c++17", "-O1", "-fPIC", "-shared", f"-I{CSRC}", str(src), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.cvt_many.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_long]

    def run(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        bits = np.zeros(x.size, np.uint32)
        ok = np.zeros(x.size, np.int32)
        lib.cvt_many(x.ctypes.data, bits.ctypes.data, ok.ctypes.data, x.size)
        return bits, ok.astype(bool)

    return run


def reference_bits(x):
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        return np.asarray(x, np.float64).astype(np.float32).view(np.uint32)


def must_claim(x):
    """doubles of magnitude in [2^-126, 2^128): biased binary64 exponent 897..1150"""
    e = (np.asarray(x).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
    return (e >= 897) & (e <= 1150)


def check(cvt, x):
    bits, ok = cvt(x)
    ref = reference_bits(x)
    assert np.array_equal(bits[ok], ref[ok]), np.asarray(x)[ok][bits[ok] != ref[ok]][:5]
    need = must_claim(x)
    assert np.all(ok[need]), np.asarray(x)[need & ~ok][:5]
    return ok


def test_random_bit_patterns(cvt):
    rng = np.random.default_rng(1)
    x = rng.integers(0, 2**64, size=400_000, dtype=np.uint64).view(np.float64)
    check(cvt, x)


def test_random_values_across_the_float_range(cvt):
    rng = np.random.default_rng(2)
    mag = 2.0 ** rng.uniform(-130, 130, size=400_000)
    x = np.where(rng.random(mag.size) < 0.5, -mag, mag)
    ok = check(cvt, x)
    assert ok.mean() > 0.95


def test_exact_ties_round_to_even(cvt):
    rng = np.random.default_rng(3)
    hi = rng.integers(0, 2**32, size=100_000, dtype=np.uint64)
    e = rng.integers(897, 1151, size=hi.size, dtype=np.uint64)
    hi = (hi & np.uint64(0x800FFFFF)) | (e << np.uint64(20))
    for low in (0x10000000, 0x10000001, 0x0FFFFFFF, 0x30000000, 0x1FFFFFFF, 0):
        lo = (rng.integers(0, 8, size=hi.size, dtype=np.uint64) << np.uint64(29)) | np.uint64(low)
        x = ((hi << np.uint64(32)) | lo).view(np.float64)
        ok = check(cvt, x)
        assert ok.all()


def test_edges_of_the_normal_range(cvt):
    f32 = np.finfo(np.float32)
    big = float(f32.max)
    tiny = float(f32.tiny)
    ulp_big = 2.0 ** 104
    x = np.array([big, -big, big + ulp_big / 2, big + ulp_big / 2 - 2.0 ** 75, big * 2, tiny, -tiny,
                  tiny * (1 - 2.0 ** -25), tiny * (1 - 2.0 ** -24), tiny / 2, 2.0 ** -150, 1.0, -1.0,
                  np.nextafter(1.0, 2.0), 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 0.0, -0.0, np.inf, -np.inf,
                  np.nan, 1e300, -1e-300, 5e-324])
    bits, ok = cvt(x)
    check(cvt, x)
    # zeros, magnitudes below 2^-126 (also those that round up to it), infinities, NaN and
    # magnitudes of 2^128 and more are left to the conversion instruction
    for v in (0.0, -0.0, np.inf, -np.inf, np.nan, 2.0 ** -150, tiny / 2, tiny * (1 - 2.0 ** -25), 1e300, 5e-324,
              big * 2):
        i = [k for k, y in enumerate(x) if (np.isnan(v) and np.isnan(y)) or y == v and np.signbit(y) == np.signbit(v)][0]
        assert not ok[i], v
    # rounding up from the largest float's exponent gives infinity, as the instruction does
    i = list(x).index(big + ulp_big / 2)
    assert ok[i] and bits[i] == np.float32(np.inf).view(np.uint32)
