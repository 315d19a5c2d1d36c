// Checks the library's host-side input checks (lbm_validate.h) against the
// same conditions written plainly, on special values and on long arrays
// with bad values planted.  Built and run by test_validate_helpers.py.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <limits>
#include <random>
#include <vector>

#include "lbm_validate.h"

static int failures = 0;
#define CHECK(c)                                                   \
  do {                                                             \
    if (!(c)) {                                                    \
      std::printf("FAIL line %d: %s\n", __LINE__, #c);             \
      ++failures;                                                  \
    }                                                              \
  } while (0)

static bool ref_fraction(float v) { return !(v >= 0.0f && v <= 1.0f); }
static bool ref_finite(float v) { return !std::isfinite(v); }
static bool ref_density(float v) { return !(v > 0.0f) || !std::isfinite(v); }

int main() {
  const float nan = std::numeric_limits<float>::quiet_NaN();
  const float inf = std::numeric_limits<float>::infinity();
  const float denorm = std::numeric_limits<float>::denorm_min();
  const float special[] = {0.0f, -0.0f, 1.0f, std::nextafter(1.0f, 2.0f),
                           std::nextafter(0.0f, -1.0f), denorm, -denorm, 0.5f, nan,
                           -nan, inf, -inf, FLT_MAX, -FLT_MAX, FLT_MIN, -FLT_MIN,
                           2.0f, -2.0f, 1e-30f, 1e30f};
  for (float v : special) {
    CHECK(hmcsc::bad_fraction(v) == ref_fraction(v));
    CHECK(hmcsc::bad_finite(v) == ref_finite(v));
    CHECK(hmcsc::bad_density(v) == ref_density(v));
  }
  std::mt19937 rng(2206);
  std::uniform_real_distribution<float> unit(0.0f, 1.0f);
  for (long long n : {0LL, 1LL, 7LL, 1000LL, 100003LL}) {
    std::vector<float> x(n);
    for (auto &v : x) v = 0.05f + 0.9f * unit(rng);
    CHECK(hmcsc::first_bad(x.data(), n, hmcsc::BadFraction{}) == n);
    CHECK(hmcsc::first_bad(x.data(), n, hmcsc::BadFinite{}) == n);
    CHECK(hmcsc::first_bad(x.data(), n, hmcsc::BadDensity{}) == n);
    if (n == 0) continue;
    for (float badv : {nan, inf, -inf, -0.5f, 1.5f}) {
      for (long long at : {0LL, n / 2, n - 1}) {
        std::vector<float> y = x;
        y[at] = badv;
        if (at + 3 < n) y[at + 3] = badv;  // a later one does not hide the first
        long long want = n;
        for (long long i = 0; i < n && want == n; ++i)
          if (ref_fraction(y[i])) want = i;
        CHECK(hmcsc::first_bad(y.data(), n, hmcsc::BadFraction{}) == want);
        want = n;
        for (long long i = 0; i < n && want == n; ++i)
          if (ref_finite(y[i])) want = i;
        CHECK(hmcsc::first_bad(y.data(), n, hmcsc::BadFinite{}) == want);
        want = n;
        for (long long i = 0; i < n && want == n; ++i)
          if (ref_density(y[i])) want = i;
        CHECK(hmcsc::first_bad(y.data(), n, hmcsc::BadDensity{}) == want);
      }
    }
  }
  if (failures) return 1;
  std::printf("ok\n");
  return 0;
}
