// bits.cuh -- integer-pipe forms of two FP64 steps of the particle push.
//
// GB300 runs FP64 arithmetic, FP64 comparisons and FP64 <-> integer
// conversions on two FP64 lanes per SM per clock, and the FP64 push spends
// most of its time there.  The two helpers below give bit for bit the results
// of short FP64 sequences (truncation + conversion + subtraction; scaling +
// rounding conversion) using integer operations on the bit pattern, which run
// on the wide integer pipes.  Each falls back to the FP64 sequence outside the
// range it handles.  Also here: the conversions of particle positions between SI
// and cell units (pic_set_particles / pic_get_particles).  Host and device
// versions are the same code, so the equivalences are checked on the CPU.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define PIC_HD __host__ __device__ __forceinline__
#else
#define PIC_HD inline
#endif

namespace pic {

PIC_HD uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}

PIC_HD double double_of(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}

PIC_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

constexpr uint64_t kMantMask = (1ULL << 52) - 1;

// Cell of coordinate s = x / d on an axis of `ncell` cells: k = (int)s clamped
// to ncell - 1 and f = s - k.  For 1 <= s < ncell the fraction is exact
// (k <= s < k + 1 <= 2k), so it is the low mantissa bits of s renormalised;
// 0 <= s < 1 gives k = 0, f = s.  Anything else (negative, clamped, huge or
// non-finite s) takes the FP64 sequence.
PIC_HD void split_cell(double s, int ncell, int& k, double& f) {
  const uint64_t b = bits_of(s);
  const int be = (int)(b >> 52);  // sign and biased exponent
  if (be < 1023) {                // 0 <= s < 1 (and +0, subnormals)
    k = 0;
    f = s;
    return;
  }
  if (be <= 1023 + 30) {          // 1 <= s < 2^31
    const uint64_t mant = (b & kMantMask) | (1ULL << 52);
    const int sh = 1075 - be;     // 52 - exponent: fraction bits, 22..52
    const int i = (int)(mant >> sh);
    if (i <= ncell - 1) {
      const uint64_t frac = mant & ((1ULL << sh) - 1);
      k = i;
      if (frac == 0) {
        f = 0.0;
      } else {
        const int p = 63 - clz64(frac);  // top bit of frac, p < sh
        f = double_of(((uint64_t)(p - sh + 1023) << 52) | ((frac << (52 - p)) & kMantMask));
      }
      return;
    }
  }
  int i = (int)s;
  if (i > ncell - 1) i = ncell - 1;
  k = i;
  f = s - (double)i;
}

// round(w * 2^44), ties to even, for 0 <= w < 2^8: w = m 2^(be - 1075) with
// the 53-bit significand m, so w 2^44 = m >> (1031 - be) plus the rounding of
// the bits shifted out.  Other w (negative, large, non-finite) take the FP64
// sequence.
PIC_HD uint64_t fix44(double w) {
  const uint64_t b = bits_of(w);
  const int be = (int)(b >> 52);
  if (be < 1031) {                  // 0 <= w < 2^8 (w >= 0: sign bit clear)
    const int d = 1031 - be;        // right shift, >= 1
    if (d >= 64) return 0ULL;       // w 2^44 < 2^-10 (also 0 and subnormals)
    const uint64_t mant = (b & kMantMask) | (1ULL << 52);
    const uint64_t q = mant >> d, rem = mant & ((1ULL << d) - 1), half = 1ULL << (d - 1);
    return q + ((rem > half || (rem == half && (q & 1ULL))) ? 1ULL : 0ULL);
  }
#ifdef __CUDA_ARCH__
  return (uint64_t)__double2ll_rn(w * 17592186044416.0);
#else
  return (uint64_t)std::llrint(w * 17592186044416.0);
#endif
}

// Comparisons on the bit patterns (integer pipes), with the IEEE outcome for
// every input, NaN included (all false).  x < 0: sign set, magnitude nonzero
// and not NaN.  x >= c for c > 0 finite: for non-negative x the bit patterns
// order like the values; negative x and NaN give false.
constexpr uint64_t kAbsMask = 0x7FFFFFFFFFFFFFFFULL;
constexpr uint64_t kInfBits = 0x7FF0000000000000ULL;
PIC_HD bool lt_zero(double x) {
  const uint64_t b = bits_of(x), a = b & kAbsMask;
  return (b >> 63) != 0 && a != 0 && a <= kInfBits;
}
PIC_HD bool ge_pos(double x, double c) {
  const uint64_t b = bits_of(x);
  return b >= bits_of(c) && b <= kInfBits;
}
// x > 0 for x known to be >= 0 or NaN (a sum of squares): true also for NaN
PIC_HD bool nonzero_sq(double x) { return bits_of(x) != 0; }

// 1 / x refined from a seed y whose relative error e satisfies |e| < 2^-20:
// a Newton-Raphson step y <- y + y (1 - x y) turns the error e into -e^2, so
// after two steps only the rounding of the last operations remains (within
// one ulp of the correctly rounded 1 / x).  Four FMAs replace the division.
PIC_HD double recip_refine(double x, double y) {
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// 2 / x, exactly 2 recip_refine(x, y): the last step is written for 2y, which
// is y with its exponent raised by one (an integer add; y is a positive normal
// number below 2^1023 after the first step for the x this is used on), so the
// doubling costs no FP64 operation.
PIC_HD double recip2_refine(double x, double y) {
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  const double y2 = double_of(bits_of(y) + (1ULL << 52));
  return fma(y2, e, y2);
}

// SI coordinate x on an axis of length X = ncell d -> cell units x / d (as
// x * inv_d).  The domain test is kept: x in [0, X) gives a value below
// ncell (a product rounded up to ncell is moved one ulp down), x >= X one of
// at least ncell; negative and NaN x stay negative / NaN.
// the next double toward zero of a positive finite x (nextafter(x, 0))
PIC_HD double next_down(double x) { return double_of(bits_of(x) - 1ULL); }

PIC_HD double to_cells(double x, double inv_d, int ncell, double X) {
  double s = x * inv_d;
  if (x < X) {
    if (s >= (double)ncell) s = next_down((double)ncell);
  } else if (x >= X && s < (double)ncell) {
    s = (double)ncell;
  }
  return s;
}

// cell units s in [0, ncell) -> SI s d, kept below X = ncell d (host and
// device give the same value: one rounded product and a clamp)
PIC_HD double from_cells(double s, double d, double X) {
  const double x = s * d;
  return x < X ? x : next_down(X);
}

}  // namespace pic
