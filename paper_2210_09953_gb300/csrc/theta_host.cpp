// Host construction of the 256 integer levels of Theta and its scale.
//
// T[t] = round(44 * Phi^{-1}((t + 1/2) / 256)), t = 0..255, where Phi is the
// standard normal CDF.  Phi^{-1} is found here by bisection on
// Phi(x) = erfc(-x / sqrt 2) / 2 (C99 erfc), to full double precision; the
// levels are then rounded half away from zero (no level lies near a tie).
#include <cmath>
#include <mutex>

#include "rcqr_internal.h"

namespace rcqr {

static double normal_quantile(double p) {
  double lo = -40.0, hi = 40.0;
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    const double cdf = 0.5 * std::erfc(-mid / std::sqrt(2.0));
    if (cdf < p)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

const ThetaTable &theta_table() {
  static ThetaTable table;
  static std::once_flag once;
  std::call_once(once, [] {
    for (int t = 0; t < 256; ++t) {
      const double x = 44.0 * normal_quantile((t + 0.5) / 256.0);
      const double r = x >= 0 ? std::floor(x + 0.5) : -std::floor(-x + 0.5);
      table.level[t] = (int8_t)r;
    }
  });
  return table;
}

double theta_scale(int64_t k) {
  const ThetaTable &T = theta_table();
  long long s = 0;
  for (int t = 0; t < 256; ++t) s += (long long)T.level[t] * T.level[t];
  const double v = (double)s / 256.0;
  return 1.0 / std::sqrt((double)k * v);
}

}  // namespace rcqr
