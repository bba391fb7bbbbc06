// Exact 7-point neighbour sums of FP64 fields on the integer pipe.
//
// GB300 issues FP64 arithmetic at about 2 lanes per SM per clock, 1/32 to
// 1/64 of its integer rate, and the five additions and the centre term of a
// 7-point Laplacian are most of the FP64 work of a defect evaluation.  Here a
// value v with |v| < 2^kFixIntBits is mapped to the 64-bit integer
// X = round(v 2^kFixFrac) (binary64 layout: sign | 11-bit biased exponent |
// 52-bit fraction, bias 1023), the sum X_xm + X_xp + X_ym + X_yp + X_zm +
// X_zp - 6 X_c is formed exactly in int64 (|X| < 2^59, so |sum| < 12 2^59
// < 2^63), and the result is rounded once to binary64 (to nearest, ties to
// even).
//
// Accuracy: each input is quantised to 2^-kFixFrac (error <= 2^-55 with the
// constants below), so the Laplacian carries an absolute error <= 12 2^-55
// ~ 3.3e-16 plus one final rounding; a left-to-right FP64 sum of O(1) values
// rounds five partial sums of size up to ~6, about 5 * 2^-51 ~ 2.2e-15 in the
// worst case.  Values outside the range (|v| >= 2^kFixIntBits, Inf, NaN) are
// reported through `ok`; the caller then evaluates in FP64 instead.
//
// The functions are plain C++ on the host (for tests of the bit arithmetic)
// and use the device intrinsics under nvcc.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define PFC_HD __host__ __device__ __forceinline__
#else
#define PFC_HD inline
#endif

namespace pfc {

constexpr int kFixFrac = 54;      // fraction bits of the fixed-point image
constexpr int kFixIntBits = 5;    // |v| < 32; 12 * 2^(5 + 54) < 2^63
// largest biased binary64 exponent inside the range (|v| < 2^5)
constexpr unsigned kFixMaxBiasedExp = 1023u + kFixIntBits - 1u;

PFC_HD uint64_t fix_bits_of(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t u;
  memcpy(&u, &v, sizeof(u));
  return u;
#endif
}

PFC_HD double fix_double_of_bits(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double v;
  memcpy(&v, &u, sizeof(v));
  return v;
#endif
}

PFC_HD int fix_clz64(uint64_t a) {   // a != 0
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}

// X = round(v 2^kFixFrac), halves rounded away from zero (a symmetric
// rounding); ok is cleared when |v| >= 2^kFixIntBits or v is not finite.
// v = m 2^(e - 1075) with m the 53-bit significand and e the biased exponent,
// so X = m 2^(e - 1075 + kFixFrac): a left shift by s = e - 1021 >= 0, else a
// rounded right shift by -s (zero and subnormal inputs shift out to 0).
PFC_HD int64_t fix_of(double v, bool& ok) {
  const uint64_t u = fix_bits_of(v);
  const unsigned e = (unsigned)(u >> 52) & 0x7FFu;
  ok = ok && e <= kFixMaxBiasedExp;
  const uint64_t m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int s = (int)e - (1075 - kFixFrac);
  uint64_t a;
  if (s >= 0) {
    a = m << (s & 7);                      // s <= kFixIntBits + 1 inside the range
  } else {
    const int r = -s;
    a = r < 60 ? (m + (1ull << (r - 1))) >> r : 0ull;
  }
  return (u >> 63) ? -(int64_t)a : (int64_t)a;
}

// X 2^-kFixFrac rounded to binary64, to nearest with ties to even.  The top
// set bit of |X| at position p = 63 - clz gives the biased exponent
// p - kFixFrac + 1023 (never subnormal: p >= 0); the 53 bits below and
// including it form the significand, the 11 dropped bits decide the
// rounding, and a carry out of the significand moves into the exponent
// field.
PFC_HD double fix_to_double(int64_t X) {
  if (X == 0) return 0.0;
  const uint64_t sign = (uint64_t)X & 0x8000000000000000ull;
  const uint64_t a = sign ? (uint64_t)(-X) : (uint64_t)X;
  const int lz = fix_clz64(a);
  const uint64_t norm = a << lz;                          // top bit at 63
  const uint64_t mant = norm >> 11;                       // bit 52 = implicit one
  const uint64_t rest = norm & 0x7FFull;
  const uint64_t up = (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
  const uint64_t ebias = (uint64_t)(63 - lz - kFixFrac + 1023);
  return fix_double_of_bits(sign | (((ebias - 1ull) << 52) + mant + up));
}

// Unscaled 7-point Laplacian of fixed-point images: sum of six neighbours
// minus 6 x the centre, exact.
PFC_HD int64_t fix_lap(int64_t xm, int64_t xp, int64_t ym, int64_t yp, int64_t zm, int64_t zp,
                       int64_t c) {
  return ((xm + xp) + (ym + yp)) + (zm + zp) - c * 6;
}

}  // namespace pfc
