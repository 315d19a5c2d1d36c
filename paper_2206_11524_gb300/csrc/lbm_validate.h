// lbm_validate.h -- host-side checks of the arrays a caller hands to the
// library (geometry and initial densities), kept apart from the CUDA code so
// that they can be compiled and tested on their own.
#pragma once

#include <cstdint>
#include <cstring>

namespace hmcsc {

// The checks look at a float's IEEE-754 bits, which turns them into integer
// compares without branches (NaNs included) that the compiler vectorizes.
inline std::uint32_t float_bits(float v) {
  std::uint32_t u;
  std::memcpy(&u, &v, sizeof u);
  return u;
}
// A bounce-back fraction outside [0, 1], or NaN: valid are +0 .. 1.0f
// (bits 0 .. 0x3f800000) and -0.
struct BadFraction {
  bool operator()(float v) const {
    const std::uint32_t u = float_bits(v);
    return (u > 0x3f800000u) & (u != 0x80000000u);
  }
};
// Not a finite number (exponent bits all set: an infinity or a NaN).
struct BadFinite {
  bool operator()(float v) const { return (float_bits(v) & 0x7f800000u) == 0x7f800000u; }
};
// Not a finite number > 0 (a component density): valid are the bits
// 1 .. 0x7f7fffff (the smallest denormal up to the largest finite float).
struct BadDensity {
  bool operator()(float v) const { return float_bits(v) - 1u > 0x7f7ffffeu; }
};

// Index of the first element of x[0, n) for which bad(x[i]) holds, or n.
// The first pass has no branch on the data; the second pass, which finds
// the index, runs only when something is bad.
template <typename Bad>
inline long long first_bad(const float *x, long long n, Bad bad) {
  std::uint32_t any = 0;
  for (long long i = 0; i < n; ++i) any |= static_cast<std::uint32_t>(bad(x[i]));
  if (!any) return n;
  for (long long i = 0; i < n; ++i)
    if (bad(x[i])) return i;
  return n;
}

inline bool bad_fraction(float v) { return BadFraction{}(v); }
inline bool bad_finite(float v) { return BadFinite{}(v); }
inline bool bad_density(float v) { return BadDensity{}(v); }

}  // namespace hmcsc
