"""The integer-pipe helpers of the particle push (csrc/bits.cuh) against the
FP64 sequences they replace, bit for bit, on the CPU: the header's host build
runs both forms over random and edge-case inputs.

* split_cell(s): (int)s clamped to ncell - 1 and s - (double)k, for s in
  [0, ncell) (random, integers and their neighbours one ulp away, tiny
  values, 0) and for negative, clamped and non-finite s;
* fix44(w): round-to-nearest-even of w 2^44 (llrint), for w in [0, 1]
  (random, exact ties at the 2^-45 grid, the neighbours of ties, tiny, 0, 1)
  and outside that range;
* lt_zero, ge_pos: the IEEE comparisons x < 0 and x >= c over random,
  signed-zero, subnormal, infinite and NaN inputs;
* recip_refine(x, seed): within one ulp of 1.0 / x for seeds up to two FP32
  ulps from the rounded FP32 reciprocal (the device seed, PTX rcp.approx, is
  within one), x in [1, 4) and log-uniform over 1e-30 .. 1e30;
* recip2_refine(x, seed): bit for bit 2 recip_refine(x, seed) on the same x;
* to_cells / from_cells (positions between SI and cell units) on axes of 2 .. 4096
  cells of random lengths: x in [0, X) lands in [0, ncell), x >= X at or above ncell,
  x < 0 below 0, NaN stays NaN; from_cells lands in [0, X) and the round trip is within
  4 ulp of x (x of at least one cell; within 4 ulp of the cell width below that).
"""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_10727_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "bits.cuh"
using namespace pic;
static bool same(double a, double b) { uint64_t x, y; std::memcpy(&x, &a, 8); std::memcpy(&y, &b, 8); return x == y; }
static long long bad = 0, n = 0;
static void check_split(double s, int ncell) {
  int k1; double f1; split_cell(s, ncell, k1, f1);
  int k2 = (int)s; if (k2 > ncell - 1) k2 = ncell - 1; double f2 = s - (double)k2;
  ++n; if (k1 != k2 || !same(f1, f2)) { if (bad < 5) std::printf("split %.17g %d: %d %.17g vs %d %.17g\n", s, ncell, k1, f1, k2, f2); ++bad; }
}
static void check_fix(double w) {
  uint64_t a = fix44(w), b = (uint64_t)std::llrint(w * 17592186044416.0);
  ++n; if (a != b) { if (bad < 5) std::printf("fix %.17g: %llu vs %llu\n", w, (unsigned long long)a, (unsigned long long)b); ++bad; }
}
static void check_recip(double x) {
  const double want = 1.0 / x;
  float s = (float)(1.0 / x);
  float seeds[5] = {s, std::nextafterf(s, 0.0f), std::nextafterf(s, 1e30f),
                    std::nextafterf(std::nextafterf(s, 0.0f), 0.0f),
                    std::nextafterf(std::nextafterf(s, 1e30f), 1e30f)};
  for (float sd : seeds) {
    const double y = recip_refine(x, (double)sd);
    uint64_t a, b; std::memcpy(&a, &y, 8); std::memcpy(&b, &want, 8);
    const uint64_t ulps = a > b ? a - b : b - a;
    ++n; if (ulps > 1) { if (bad < 5) std::printf("recip %.17g: %.17g vs %.17g\n", x, y, want); ++bad; }
    ++n; if (!same(recip2_refine(x, (double)sd), 2.0 * y)) { if (bad < 5) std::printf("recip2 %.17g\n", x); ++bad; }
  }
}
static void check_cells(double x, double d, int ncell) {
  const double X = ncell * d, inv = 1.0 / d;
  const double s = to_cells(x, inv, ncell, X);
  bool ok;
  if (x != x) ok = s != s;
  else if (x < 0.0) ok = s < 0.0;
  else if (x >= X) ok = s >= (double)ncell;
  else {
    const double back = from_cells(s, d, X);
    const double tol = 4.0 * std::ldexp(1.0, -52) * (x > d ? x : d);
    ok = s >= 0.0 && s < (double)ncell && back >= 0.0 && back < X && std::fabs(back - x) <= tol;
  }
  ++n; if (!ok) { if (bad < 5) std::printf("cells %.17g %.17g %d -> %.17g\n", x, d, ncell, s); ++bad; }
}
static void check_cmp(double x, double c) {
  ++n; if (lt_zero(x) != (x < 0.0) || ge_pos(x, c) != (x >= c)) {
    if (bad < 5) std::printf("cmp %.17g %.17g\n", x, c); ++bad; }
}
int main() {
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> u(0.0, 1.0);
  for (int ncell : {1, 2, 7, 256, 512, 4096, 65536}) {
    for (int t = 0; t < 400000; ++t) check_split(u(g) * ncell, ncell);
    for (int k = 0; k <= ncell && k < 5000; ++k) {
      double s = k;
      check_split(s, ncell);
      check_split(std::nextafter(s, -1.0), ncell);
      check_split(std::nextafter(s, 1e9), ncell);
    }
    for (double s : {0.0, 1e-300, 5e-324, 1e-20, 0.5, -0.0, -1e-12, -0.75, -3.5,
                     (double)ncell + 0.25, 1e12, 3e9, (double)INFINITY})
      check_split(s, ncell);
  }
  for (int t = 0; t < 2000000; ++t) check_fix(u(g));
  for (int t = 0; t < 200000; ++t) {   // exact ties and their neighbours
    uint64_t j = g() & ((1ULL << 45) - 1);
    double w = std::ldexp((double)(2 * j + 1), -45);
    check_fix(w); check_fix(std::nextafter(w, 0.0)); check_fix(std::nextafter(w, 2.0));
  }
  for (double w : {0.0, -0.0, 5e-324, 1e-300, 1e-14, 2.842170943040401e-14, 5.684341886080802e-14,
                   0.5, 1.0, std::nextafter(1.0, 0.0), 1.0000000000000002, 200.0, 255.999, 256.0,
                   1e6, -1e-15, -0.5})
    check_fix(w);
  for (double c : {0.05, 1e-300, 3.5, 1e300}) {
    for (int t = 0; t < 200000; ++t) { double x = (u(g) - 0.5) * 4.0 * c; check_cmp(x, c); }
    for (double x : {0.0, -0.0, 5e-324, -5e-324, c, -c, std::nextafter(c, 0.0), std::nextafter(c, 1e308),
                     (double)INFINITY, -(double)INFINITY, (double)NAN, -(double)NAN, 1e308, -1e308})
      check_cmp(x, c);
  }
  for (int t = 0; t < 1000000; ++t) check_recip(1.0 + 3.0 * u(g));
  for (int t = 0; t < 1000000; ++t) check_recip(std::pow(10.0, -30.0 + 60.0 * u(g)));
  for (int ncell : {2, 32, 256, 512, 4096}) {
    for (int t = 0; t < 2000; ++t) {
      const double d = std::pow(10.0, -6.0 + 4.0 * u(g)) / ncell * 1000.0;
      const double X = ncell * d;
      for (int k = 0; k < 50; ++k) check_cells(u(g) * X, d, ncell);
      for (double x : {0.0, -0.0, X, std::nextafter(X, 0.0), std::nextafter(X, 1e300), 2.0 * X,
                       -1e-300, -X, d, std::nextafter(d, 0.0), 5e-324, (double)NAN})
        check_cells(x, d, ncell);
    }
  }
  std::printf("checked %lld mismatches %lld\n", n, bad);
  return bad != 0;
}
"""


def test_integer_pipe_helpers_match_fp64_sequences(tmp_path):
    src = tmp_path / "bits_check.cpp"
    exe = tmp_path / "bits_check"
    src.write_text(PROGRAM)
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert "mismatches 0" in r.stdout
