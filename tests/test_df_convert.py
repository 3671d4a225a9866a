"""The integer-path conversions between double and double-float pairs that
the FP64 sweep uses (csrc/df_convert.h), compiled on the host with g++ and
checked against exact arithmetic (long double holds hi + lo exactly):

* to_df: hi carries the leading 24 bits (hi is a float and |lo| < ulp(hi)),
  and hi + lo = x to 2^-47 relative, on the integer path (2^-74 <= |x| <
  2^115) and on the rounded fallback outside it, down to |x| = 2^-100 (the
  double-float range: below it lo is a float subnormal and the error is at
  most 2^-149 absolute); zero and FP64 subnormals give (0, 0).
* from_df: for pairs normalised as the sweep's arithmetic leaves them
  (hi = fl(hi + lo), the two-sum of two floats, and the pairs to_df makes)
  the result is hi + lo to 2^-52 relative, and round trips return x to
  2^-47.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2407_02100_gb300", "csrc")

PROG = r'''
#include "df_convert.h"
#include <cmath>
#include <cstdio>
#include <random>
using gmg::dfconv::to_df;
using gmg::dfconv::from_df;

static int fail(const char* what, double x, double a, double b) {
  std::printf("FAIL %s x=%.17g got=%.17g want=%.17g\n", what, x, a, b);
  return 1;
}

int main() {
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> mant(1.0, 2.0);
  std::uniform_int_distribution<int> ex(-140, 126);  // float range: |x| < 2^127
  long checked = 0, fast = 0;
  for (int t = 0; t < 2000000; ++t) {
    double x = std::ldexp(mant(rng), ex(rng));
    if (rng() & 1) x = -x;
    float hi, lo;
    to_df(x, hi, lo);
    const long double s = (long double)hi + (long double)lo;
    const long double err = std::fabs((long double)x - s);
    // double-float carries 2^-47 relative down to |x| = 2^-100; below, lo
    // is a float subnormal and the error is absolute, at most 2^-149
    const long double bound = std::fabs(x) >= std::ldexp(1.0, -100) ? std::ldexp((long double)std::fabs(x), -47)
                                                                      : std::ldexp((long double)1, -149);
    if (!(err <= bound)) return fail("to_df sum", x, (double)s, x);
    if (std::fabs(x) >= std::ldexp(1.0, -100) && std::fabs(x) < std::ldexp(1.0, 120)) {
      const float ulp = std::nextafter(std::fabs(hi), INFINITY) - std::fabs(hi);
      if (!(std::fabs(lo) <= ulp)) return fail("to_df |lo| <= ulp(hi)", x, lo, ulp);
      const double back = from_df(hi, lo);
      if (!(std::fabs(back - x) <= std::ldexp(std::fabs(x), -47))) return fail("round trip", x, back, x);
    }
    if (std::fabs(x) >= std::ldexp(1.0, -74) && std::fabs(x) < std::ldexp(1.0, 115)) ++fast;
    ++checked;
  }
  // pairs from the two-sum of two floats (the normalised form of df arithmetic)
  std::uniform_real_distribution<float> u(-1.f, 1.f);
  std::uniform_int_distribution<int> gap(24, 40), fe(-100, 100);
  for (int t = 0; t < 1000000; ++t) {
    const float a = std::ldexp(u(rng), fe(rng));
    const float b = std::ldexp(u(rng), std::ilogb(a) - gap(rng));
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    const long double want = (long double)s + (long double)e;
    const double got = from_df(s, e);
    if (!(std::fabs((long double)got - want) <= std::ldexp(std::fabs(want), -52))) return fail("from_df", (double)want, got, (double)want);
  }
  // special values
  float hi, lo;
  to_df(0.0, hi, lo);
  if (hi != 0.f || lo != 0.f) return fail("zero", 0, hi, lo);
  to_df(-0.0, hi, lo);
  if (hi != 0.f || lo != 0.f) return fail("-zero", 0, hi, lo);
  to_df(4.9e-324, hi, lo);
  if (hi != 0.f || lo != 0.f) return fail("subnormal", 4.9e-324, hi, lo);
  if (from_df(0.f, 0.f) != 0.0) return fail("from zero", 0, from_df(0.f, 0.f), 0);
  if (from_df(1.5f, 0.f) != 1.5) return fail("from exact", 1.5, from_df(1.5f, 0.f), 1.5);
  if (from_df(-3.0f, 0.f) != -3.0) return fail("from negative", -3, from_df(-3.0f, 0.f), -3);
  std::printf("ok %ld %ld\n", checked, fast);
  return 0;
}
'''


def test_double_float_conversions_against_exact_arithmetic(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("needs g++")
    src = tmp_path / "df_convert_test.cpp"
    exe = tmp_path / "df_convert_test"
    src.write_text(PROG)
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", f"-I{CSRC}", str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0 and res.stdout.startswith("ok"), res.stdout + res.stderr
    _, checked, fast = res.stdout.split()
    assert int(fast) > int(checked) // 2      # most samples take the integer path
