// Host constant tables of the decision rule (noise levels and activation values).
#pragma once
#include <cstdint>

namespace pim {

constexpr int kNoiseLevels = 4096;  // 12-bit noise key

// 4096 noise levels: kind 0 = Gaussian quantiles Phi^-1((m+0.5)/4096) (antisymmetric),
// kind 1 = uniform grid (2m-4095)/4096.
void noise_levels(int kind, float* out);

// tau(I) for I = -imax..imax: act 0 = fl32(tanh(b_t * I)) in float64, act 1 = L-level
// staircase.
void activation_levels(float b_t, int imax, int act, int lut_levels, float* out);

// b_t = fl32(beta_t * c), the coupling scale folded into the inverse temperature.
float scaled_beta(float beta, double c);

// Decision thresholds of the fixed-point datapath (ap_fixed<total_bits, int_bits>,
// truncation toward zero, saturation) for one schedule step: for I = -imax..imax,
// word[I + imax] = M(s=-1) | M(s=+1) << 16 with M the least noise key whose quantized
// decision is +1 (4096 = never).  z: the 4096 noise levels.
void fixed_thresholds(double c, float beta_t, float eta_t, float xi, int act, int lut_levels,
                      int total_bits, int int_bits, const float* z, int imax, uint32_t* word);

// ap_fixed<total_bits, int_bits> value of v (truncation toward zero, then saturation) in
// units of its step 2^-(total_bits - int_bits): an integer in [-2^(W-1), 2^(W-1) - 1].
int32_t fixed_units(double v, int total_bits, int int_bits);

// Integer tables of the fixed-point datapath for real couplings (values in units of the
// step 2^-F, F = total_bits - int_bits): tau[m + 2^(W-1)] = Q(act(m 2^-F)) for every
// representable x = m 2^-F (act 0 = tanh, 1 = L-level staircase); qz[k] = Q(z[k]) for the
// 4096 noise levels; *qxi = Q(xi).  tau has 2^W entries.
void fixed_real_tables(int total_bits, int int_bits, int act, int lut_levels, float xi,
                       const float* z, int32_t* tau, int32_t* qz, int32_t* qxi);

}  // namespace pim
