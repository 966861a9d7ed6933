// Host constant tables of the decision rule (noise levels and activation values).
#pragma once

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

}  // namespace pim
