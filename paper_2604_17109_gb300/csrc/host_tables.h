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

}  // namespace pim
