// Host-side constant tables of the decision rule: the 4096 noise levels z(m) and the
// activation values tau_t(I).  These are the only transcendental evaluations of the
// library; everything per sweep runs on the device from integer tables built from them.
#include "host_tables.h"

#include <cmath>
#include <cstdint>

namespace pim {

// Standard normal CDF through the complementary error function of the C library:
// Phi(x) = erfc(-x / sqrt 2) / 2, accurate in the lower tail where it is used.
static double normal_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

// Phi^-1(p) for 0 < p < 1/2 by bisection on Phi over [-40, 0] until the bracket stops
// shrinking, then the bracket end whose CDF is closer to p.  Phi is strictly increasing,
// so the bracket always holds the root; the result is within a few units in the last
// place of double, far below the float32 rounding applied afterwards.
static double normal_quantile_lower(double p) {
  double lo = -40.0, hi = 0.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (normal_cdf(mid) < p)
      lo = mid;
    else
      hi = mid;
  }
  return (std::fabs(normal_cdf(lo) - p) <= std::fabs(normal_cdf(hi) - p)) ? lo : hi;
}

void noise_levels(int kind, float* out) {
  if (kind == 0) {  // Gaussian quantiles, exactly antisymmetric
    for (int m = 0; m < kNoiseLevels / 2; ++m) {
      const double p = (m + 0.5) / kNoiseLevels;
      const float v = static_cast<float>(normal_quantile_lower(p));
      out[m] = v;
      out[kNoiseLevels - 1 - m] = -v;
    }
  } else {  // uniform grid (2m - 4095) / 4096
    for (int m = 0; m < kNoiseLevels; ++m)
      out[m] = static_cast<float>((2.0 * m - (kNoiseLevels - 1)) / kNoiseLevels);
  }
}

// L-level staircase on [-1, 1]: output levels -1 + 2k/(L-1), input breakpoints
// -1 + 2k/L; saturates outside [-1, 1].
static double staircase(double x, int levels) {
  if (x < -1.0) return -1.0;
  if (x > 1.0) return 1.0;
  int k = 0;
  for (int kk = 1; kk < levels; ++kk)
    if (x >= -1.0 + 2.0 * kk / levels) k = kk;
  return -1.0 + 2.0 * k / (levels - 1);
}

void activation_levels(float b_t, int imax, int act, int lut_levels, float* out) {
  const double b = static_cast<double>(b_t);
  for (int I = -imax; I <= imax; ++I) {
    const double x = b * static_cast<double>(I);  // exact: 24-bit b times |I| < 2^20
    const double tau = (act == 0) ? std::tanh(x) : staircase(x, lut_levels);
    out[I + imax] = static_cast<float>(tau);
  }
}

float scaled_beta(float beta, double c) {
  return static_cast<float>(static_cast<double>(beta) * c);
}

namespace {

// ap_fixed<W, I, AP_TRN_ZERO, AP_SAT> value of v: drop the bits below 2^-(W-I) toward
// zero, then clamp to the signed range.  All inputs here are small multiples of powers of
// two or doubles whose truncation is exact in double arithmetic.
struct FixedFormat {
  double step, lo, hi;
  FixedFormat(int total_bits, int int_bits)
      : step(std::ldexp(1.0, int_bits - total_bits)),
        lo(-std::ldexp(1.0, int_bits - 1)),
        hi(std::ldexp(1.0, int_bits - 1) - std::ldexp(1.0, int_bits - total_bits)) {}
  double operator()(double v) const {
    const double q = std::trunc(v / step) * step;
    return q < lo ? lo : (q > hi ? hi : q);
  }
};

}  // namespace

void fixed_thresholds(double c, float beta_t, float eta_t, float xi, int act, int lut_levels,
                      int total_bits, int int_bits, const float* z, int imax, uint32_t* word) {
  const FixedFormat Q(total_bits, int_bits);
  const double qxi = Q(static_cast<double>(xi));
  const double qeta = Q(static_cast<double>(eta_t));
  // quantized noise term per key, non-decreasing in the key
  static thread_local double noise[kNoiseLevels];
  for (int m = 0; m < kNoiseLevels; ++m) noise[m] = Q(qeta * Q(static_cast<double>(z[m])));
  for (int I = -imax; I <= imax; ++I) {
    const double u = Q(c * static_cast<double>(I));          // scaling after the MAC
    const double x = Q(static_cast<double>(beta_t) * u);     // inverse temperature
    const double tau = Q(act == 0 ? std::tanh(x) : staircase(x, lut_levels));
    uint32_t w = 0;
    for (int s = 0; s < 2; ++s) {
      const double a = Q(tau + (s ? qxi : -qxi));
      // least key m with Q(a + noise[m]) >= 0, by bisection (the decision is monotone)
      int lo = 0, hi = kNoiseLevels;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (Q(a + noise[mid]) >= 0.0)
          hi = mid;
        else
          lo = mid + 1;
      }
      w |= static_cast<uint32_t>(lo) << (16 * s);
    }
    word[I + imax] = w;
  }
}

int32_t fixed_units(double v, int total_bits, int int_bits) {
  const FixedFormat Q(total_bits, int_bits);
  return static_cast<int32_t>(std::llround(Q(v) / Q.step));  // exact: Q(v) is on the grid
}

void fixed_real_tables(int total_bits, int int_bits, int act, int lut_levels, float xi,
                       const float* z, int32_t* tau, int32_t* qz, int32_t* qxi) {
  const FixedFormat Q(total_bits, int_bits);
  const long long half = 1ll << (total_bits - 1);
  for (long long m = -half; m < half; ++m) {
    const double x = static_cast<double>(m) * Q.step;
    const double v = Q(act == 0 ? std::tanh(x) : staircase(x, lut_levels));
    tau[m + half] = static_cast<int32_t>(std::llround(v / Q.step));
  }
  for (int k = 0; k < kNoiseLevels; ++k) qz[k] = fixed_units(static_cast<double>(z[k]), total_bits, int_bits);
  *qxi = fixed_units(static_cast<double>(xi), total_bits, int_bits);
}

}  // namespace pim
