"""The integer-pipe floating-point conversions of the CUDA kernels
(paper_2205_05840_gb300/csrc/fpbits.cuh), compiled as host C++ and checked bit
for bit against IEEE-754 conversions done by NumPy and exact integer arithmetic
in Python.  The FP64 fixed-point stencil (to_fixed, fixed_to_double) and the
mixed PCG's float right-hand side and float-to-double return (d2f_pow2,
f2d_pow2, f2d_bits) rely on them.  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_05840_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "fpbits.cuh"
using namespace ndmg;
template <typename T> std::vector<T> rd(const char* p) {
  FILE* f = fopen(p, "rb"); fseek(f, 0, SEEK_END); long n = ftell(f); fseek(f, 0, SEEK_SET);
  std::vector<T> v(n / sizeof(T)); if (n) fread(v.data(), sizeof(T), v.size(), f); fclose(f); return v;
}
template <typename T> void wr(const char* p, const std::vector<T>& v) {
  FILE* f = fopen(p, "wb"); fwrite(v.data(), sizeof(T), v.size(), f); fclose(f);
}
int main(int argc, char** argv) {
  const std::string d = argv[1];
  auto P = [&](const char* n) { return (d + "/" + n); };
  auto f32 = rd<float>(P("f32.bin").c_str());
  auto f64 = rd<double>(P("f64.bin").c_str());
  auto ks = rd<int>(P("k.bin").c_str());
  auto fx = rd<long long>(P("fx.bin").c_str());
  auto fxs = rd<int>(P("fxs.bin").c_str());
  auto i64 = rd<long long>(P("i64.bin").c_str());
  std::vector<double> o_f2d(f32.size()), o_f2dp(f32.size() * ks.size()), o_i2d(i64.size()), o_p2e(f64.size());
  std::vector<float> o_d2fp(f64.size() * ks.size());
  std::vector<long long> o_fix(fxs.size());
  for (size_t i = 0; i < f32.size(); ++i) o_f2d[i] = f2d_bits(f32[i]);
  for (size_t j = 0; j < ks.size(); ++j)
    for (size_t i = 0; i < f32.size(); ++i) o_f2dp[j * f32.size() + i] = f2d_pow2(f32[i], ks[j]);
  for (size_t j = 0; j < ks.size(); ++j)
    for (size_t i = 0; i < f64.size(); ++i) o_d2fp[j * f64.size() + i] = d2f_pow2(f64[i], ks[j]);
  for (size_t i = 0; i < f64.size(); ++i) o_p2e[i] = (double)pow2_exponent(f64[i]);
  // to_fixed on (value, shift) pairs: the value's bits come in fx
  for (size_t i = 0; i < fxs.size(); ++i) { double v; memcpy(&v, &fx[i], 8); o_fix[i] = to_fixed(v, fxs[i]); }
  for (size_t i = 0; i < i64.size(); ++i) o_i2d[i] = fixed_to_double(i64[i]);
  wr(P("o_f2d.bin").c_str(), o_f2d); wr(P("o_f2dp.bin").c_str(), o_f2dp); wr(P("o_d2fp.bin").c_str(), o_d2fp);
  wr(P("o_p2e.bin").c_str(), o_p2e); wr(P("o_fix.bin").c_str(), o_fix); wr(P("o_i2d.bin").c_str(), o_i2d);
  return 0;
}
"""

KS = np.array([-1100, -200, -60, -30, -3, -1, 0, 1, 2, 7, 40, 127, 300, -4096, 4096], dtype=np.int32)
F32_MIN_NORMAL = np.float32(2.0 ** -126)


def _bits64(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _bits32(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = str(tmp_path_factory.mktemp("fpbits"))
    src = os.path.join(d, "drv.cpp")
    with open(src, "w") as fh:
        fh.write(DRIVER.replace("#include <vector>", "#include <vector>\n#include <cstring>\n#include <string>"))
    exe = os.path.join(d, "drv")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)
    rng = np.random.default_rng(7)

    # floats: random normals over the whole exponent range, both signs, and
    # the special values
    f32 = np.concatenate([
        (rng.uniform(1, 2, 4000) * 2.0 ** rng.integers(-126, 128, 4000)).astype(np.float32)
        * np.where(rng.random(4000) < 0.5, -1, 1).astype(np.float32),
        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0 ** -126, -(2.0 ** -126), 2.0 ** -130,
                  -(2.0 ** -140), np.finfo(np.float32).max, np.finfo(np.float32).tiny], dtype=np.float32)])
    # doubles: random values, exact rounding ties (low 29 fraction bits = 2^28)
    # with even and odd kept parts, the carry out of the fraction, values
    # near the float limits, specials
    rnd = rng.uniform(1, 2, 4000) * 2.0 ** rng.integers(-200, 200, 4000) * np.where(rng.random(4000) < 0.5, -1, 1)
    base = _bits64(rng.uniform(1, 2, 400))
    ties = ((base & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000000)).view(np.float64)
    above = ((base & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000001)).view(np.float64)
    below = ((base & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x0FFFFFFF)).view(np.float64)
    carry = np.array([np.nextafter(2.0, 1.0), -np.nextafter(1.0, 0.0) * 2.0 ** 10, 1.9999999403953552,
                      1.999999970197677612], dtype=np.float64)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, 2.0 ** -126, 2.0 ** -127, 2.0 ** -149,
                        float(np.finfo(np.float32).max), 3.4028235677973366e38, 5e-324, 1e-310, 2.0 ** 1023,
                        0.5, 0.75, 0.375], dtype=np.float64)
    f64 = np.concatenate([rnd, ties, -ties * 4, above, below, carry, special])
    # to_fixed: |v| 2^s < 2^63, the regime of the stencil (max |u| 2^s < 2^55)
    v = rng.uniform(-1, 1, 3000) * 2.0 ** rng.integers(-60, 5, 3000)
    v = np.concatenate([v, [0.0, -0.0, 5e-324, -1e-310, 1.0, -1.0, 2.0 ** -80]])
    s = rng.integers(40, 56, v.size).astype(np.int32)
    # int64 -> double: magnitudes up to 2^63 with exact ties at 2^11 granularity
    i64 = np.concatenate([
        rng.integers(-(2 ** 62), 2 ** 62, 3000, dtype=np.int64),
        rng.integers(-(2 ** 30), 2 ** 30, 1000, dtype=np.int64),
        (rng.integers(2 ** 52, 2 ** 53, 500, dtype=np.int64) << 11) | (1 << 10),   # ties, 53-bit mantissas
        np.array([0, 1, -1, 2 ** 53 + 1, 2 ** 63 - 1, -(2 ** 63), -(2 ** 62) - 1], dtype=np.int64)])
    for name, arr in (("f32", f32), ("f64", f64), ("k", KS), ("fx", v.view(np.int64)), ("fxs", s), ("i64", i64)):
        arr.tofile(os.path.join(d, name + ".bin"))
    subprocess.run([exe, d], check=True)
    out = {n: np.fromfile(os.path.join(d, f"o_{n}.bin"), dtype=t)
           for n, t in (("f2d", np.float64), ("f2dp", np.float64), ("d2fp", np.float32), ("p2e", np.float64),
                        ("fix", np.int64), ("i2d", np.float64))}
    return dict(f32=f32, f64=f64, v=v, s=s, i64=i64, **out)


def _same(a, b):
    """bitwise equality, any NaN equal to any NaN"""
    a, b = np.asarray(a), np.asarray(b)
    nan = np.isnan(a) & np.isnan(b)
    if a.dtype == np.float64:
        eq = _bits64(a) == _bits64(b)
    else:
        eq = _bits32(a) == _bits32(b)
    return bool(np.all(eq | nan))


def test_f2d_bits_is_the_exact_widening(run):
    f = run["f32"]
    want = f.astype(np.float64)
    sub = (f != 0) & (np.abs(f) < F32_MIN_NORMAL)
    want[sub] = np.copysign(0.0, f[sub])            # subnormal floats flush to signed zero
    assert _same(run["f2d"], want)


def test_f2d_pow2_is_the_exact_scaled_widening(run):
    f = run["f32"]
    got = run["f2dp"].reshape(KS.size, f.size)
    for j, k in enumerate(KS):
        with np.errstate(over="ignore", under="ignore"):
            want = np.ldexp(f.astype(np.float64), int(np.clip(k, -2000, 2000)))
        sub = (f != 0) & (np.abs(f) < F32_MIN_NORMAL)
        tiny = np.isfinite(f) & (f != 0) & (np.abs(want) < 2.0 ** -1022)
        want[sub | tiny] = np.copysign(0.0, f[sub | tiny])   # below the normal double range: signed zero
        assert _same(got[j], want), k


def test_d2f_pow2_rounds_to_nearest_even(run):
    x = run["f64"]
    got = run["d2fp"].reshape(KS.size, x.size)
    for j, k in enumerate(KS):
        want = np.empty(x.size, dtype=np.float32)
        for i, xi in enumerate(x):
            if not np.isfinite(xi) or xi == 0 or abs(xi) < 2.0 ** -1022:
                want[i] = np.float32(xi) if not (xi != 0 and abs(xi) < 2.0 ** -1022) else np.copysign(0.0, xi)
                continue
            # the exact product as a rational, rounded by NumPy's IEEE
            # conversion of the correctly rounded double where that is exact,
            # else by hand (round to nearest, ties to even, on 24 bits)
            e = Fraction(xi) * (Fraction(2) ** int(k))
            a = abs(e)
            if a >= 2 ** 128:
                want[i] = np.copysign(np.inf, xi)
                continue
            ex = a.numerator.bit_length() - a.denominator.bit_length()
            if Fraction(2) ** ex > a:
                ex -= 1
            # a = m 2^(ex - 23), m in [2^23, 2^24)
            m = a / Fraction(2) ** (ex - 23)
            fl = m.numerator // m.denominator
            rem = m - fl
            if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
                fl += 1
            val = Fraction(fl) * Fraction(2) ** (ex - 23)
            if val >= Fraction(2) ** 128:
                w = np.inf
            elif val < Fraction(2) ** -126:
                w = 0.0                                   # below the normal float range: flushed
            else:
                w = float(val)
            want[i] = np.float32(np.copysign(w, xi))
        assert _same(got[j], want), k


def test_d2f_pow2_matches_numpy_inside_the_normal_range(run):
    # a second, independent expectation: NumPy's float64 -> float32 cast of
    # the (exact) double product
    x = run["f64"]
    got = run["d2fp"].reshape(KS.size, x.size)
    for j, k in enumerate(KS):
        if abs(int(k)) > 1000:
            continue
        with np.errstate(over="ignore", under="ignore", invalid="ignore"):
            prod = np.ldexp(x, int(k))
            ok = np.isfinite(x) & (np.abs(x) >= 2.0 ** -1022) & (np.abs(prod) >= 2.0 ** -1022) & \
                (np.abs(prod) >= 2.0 ** -126) & (np.abs(prod) < 3.0e38)
            want = prod.astype(np.float32)
        assert _same(got[j][ok], want[ok]), k


def test_pow2_exponent(run):
    x = run["f64"]
    got = run["p2e"]
    for xi, g in zip(x, got):
        b = int(_bits64(xi)) >> 52 & 0x7FF
        want = -4096 if b == 0 else (4096 if b == 0x7FF else b - 1023)
        assert g == want, (xi, g, want)


def test_to_fixed_truncates_exactly(run):
    for v, s, g in zip(run["v"], run["s"], run["fix"]):
        if v != 0 and abs(v) < 2.0 ** -1022:
            assert g == 0
            continue
        e = Fraction(float(v)) * Fraction(2) ** int(s)
        want = int(e)              # truncation toward zero
        assert int(g) == want, (v, s, g, want)


def test_fixed_to_double_rounds_to_nearest_even(run):
    for x, g in zip(run["i64"], run["i2d"]):
        assert _bits64(g) == _bits64(float(int(x))), (x, g)   # Python's int -> float rounds ties to even
