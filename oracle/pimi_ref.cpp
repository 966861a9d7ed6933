// Plain C++17 oracle of the PIMI anneal -- TEST INFRASTRUCTURE ONLY.
//
// A second, independent CPU statement of the update rule that oracle/pimi.py restates in
// numpy: only the tests, the smoke check and the CPU-baseline legs of the benchmark load
// it.  It shares no code with the CUDA library (no header, table or helper of the library is
// included) and the library never loads it.  Built with -O2 -ffp-contract=off, so every
// float32 operation below rounds once, in the order written.
//
// What it computes (paper section / equation):
//   local field     I_i(t) = sum_j J_ij s_j(t) + h_i ....................... Eq. 2
//   energy          H(s) = -1/2 sum_i s_i (I_i + h_i) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i
//                   for symmetric J with zero diagonal ........................ Eq. 1
//   PIMI update     s_i(t+1) = sign[tanh(beta(t) c I_i(t)) + xi s_i(t) + eta(t) z] for all i
//                   at once, from s(t) .................................. Eq. 4, Box 1 (blue)
//   LUT activation  L levels -1 + 2k/(L-1), breakpoints -1 + 2k/L, saturating at +-1
//                   ........................ Algorithm "LUT-based tanh approximation"
//   bookkeeping     best energy over s(t_begin) .. s(t_begin + sweeps) (strict <, so the
//                   earliest minimum wins), its step and state; first step whose energy is
//                   <= target (success criterion of the supplementary CCTS section)
// with the same readings as the numpy oracle: the coupling scale c is applied after the
// multiply-accumulate through b_t = fl32(beta_t c) and x = b_t I in float64; tau = fl32 of the
// C library tanh; the decision a = fl32(tau + (s > 0 ? xi : -xi)), n = fl32(eta_t z),
// delta = fl32(a + n), s' = +1 iff delta >= 0; the N(0,1) term is z = Q[d >> 4] with
// Q[m] = fl32(Phi^-1((m + 0.5)/4096)) (exactly antisymmetric) and d a 16-bit draw of
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key (seed lo, seed hi) and counter
// (i >> 3, r, t, q), word (i & 7) >> 1, low half for even i; uniform noise of Eq. 3 uses
// (2m - 4095)/4096; initial spins, when not given, are bit 15 of the draw at step field
// 0xFFFFFFFF.
//
// Replicas are independent (counter-based noise), so they are split over threads.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr int kLevels = 4096;

// Philox4x32-10 from its published definition: ten rounds; a round multiplies counter words
// 0 and 2 by the two fixed multipliers, and the new counter is
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key advances by the
// two Weyl constants after every round.
void philox(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = M0 * c0;
    const uint64_t p1 = M1 * c2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = static_cast<uint32_t>(p1);
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = static_cast<uint32_t>(p0);
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// The 16-bit draws of one replica and step for spins 0 .. n-1 (one Philox block per 8).
void draws(uint64_t seed, uint32_t q, uint32_t r, uint32_t t, int n, uint16_t* d) {
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int b = 0; 8 * b < n; ++b) {
    const uint32_t ctr[4] = {static_cast<uint32_t>(b), r, t, q};
    uint32_t w[4];
    philox(ctr, k0, k1, w);
    for (int k = 0; k < 8 && 8 * b + k < n; ++k) {
      const uint32_t word = w[k >> 1];
      d[8 * b + k] = static_cast<uint16_t>((k & 1) ? (word >> 16) : (word & 0xFFFFu));
    }
  }
}

// Standard normal CDF through the complementary error function.
double normal_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

// Phi^-1(p) for 0 < p <= 1/2 by Newton's method from x = 0: Phi is increasing and convex on
// x <= 0, so the iterates decrease monotonically onto the root.
double normal_quantile_lower(double p) {
  const double inv_sqrt_2pi = 0.39894228040143267794;
  double x = 0.0;
  for (int it = 0; it < 200; ++it) {
    const double f = normal_cdf(x) - p;
    const double dens = inv_sqrt_2pi * std::exp(-0.5 * x * x);
    const double nx = x - f / dens;
    if (nx == x) break;
    x = nx;
  }
  return x;
}

void gauss_table(float* z) {
  for (int m = 0; m < kLevels / 2; ++m) {
    const float v = static_cast<float>(normal_quantile_lower((m + 0.5) / kLevels));
    z[m] = v;
    z[kLevels - 1 - m] = -v;
  }
}

void uniform_table(float* z) {
  for (int m = 0; m < kLevels; ++m)
    z[m] = static_cast<float>((2.0 * m - (kLevels - 1)) / kLevels);
}

double lut_staircase(double x, int levels) {
  if (x < -1.0) return -1.0;
  if (x > 1.0) return 1.0;
  int k = 0;
  for (int kk = 1; kk < levels; ++kk)
    if (x >= -1.0 + 2.0 * kk / levels) k = kk;
  return -1.0 + 2.0 * k / (levels - 1);
}

struct Problem {
  int n;
  int real;
  const int8_t* J8;
  const double* Jd;
  const int32_t* h32;
  const double* hd;
  double c;
  const float* beta;
  const float* eta;
  float xi;
  int act;
  int lut_levels;
  const float* z;
  int t_begin, sweeps;
  uint64_t seed;
  uint32_t q;
  int has_target;
  double target;
};

// Field I = J s + h of one state, and the energy -1/2 sum_i s_i (I_i + h_i).
double field_energy(const Problem& P, const int8_t* s, double* I) {
  const int n = P.n;
  if (!P.real) {
    long long tot = 0;
    for (int i = 0; i < n; ++i) {
      long long acc = P.h32 ? P.h32[i] : 0;
      const int8_t* row = P.J8 + static_cast<size_t>(i) * n;
      for (int j = 0; j < n; ++j) acc += static_cast<long long>(row[j]) * s[j];
      I[i] = static_cast<double>(acc);
      tot += s[i] * (acc + (P.h32 ? P.h32[i] : 0));
    }
    return static_cast<double>(-(tot / 2));  // s^T J s is even for zero-diagonal symmetric J
  }
  double tot = 0.0;
  for (int i = 0; i < n; ++i) {
    double acc = P.hd ? P.hd[i] : 0.0;
    const double* row = P.Jd + static_cast<size_t>(i) * n;
    for (int j = 0; j < n; ++j) acc += row[j] * s[j];
    I[i] = acc;
    tot += s[i] * (acc + (P.hd ? P.hd[i] : 0.0));
  }
  return -0.5 * tot;
}

// One replica: sweeps t_begin .. t_begin + sweeps - 1 from state s, with the records.
void run_replica(const Problem& P, uint32_t r, int8_t* s, double* best_E, int32_t* best_t,
                 int32_t* first_hit, double* final_E, int8_t* best_state) {
  const int n = P.n;
  std::vector<double> I(n);
  std::vector<uint16_t> d(n);
  std::vector<int8_t> next(n);
  auto bookkeep = [&](double E, int t) {
    if (E < *best_E) {
      *best_E = E;
      *best_t = t;
      std::memcpy(best_state, s, n);
    }
    if (P.has_target && *first_hit < 0 && E <= P.target) *first_hit = t;
  };
  for (int t = P.t_begin; t < P.t_begin + P.sweeps; ++t) {
    const double E = field_energy(P, s, I.data());  // Eq. 2 and Eq. 1 of s(t)
    bookkeep(E, t);
    draws(P.seed, P.q, r, static_cast<uint32_t>(t), n, d.data());
    const float b_t = static_cast<float>(static_cast<double>(P.beta[t]) * P.c);
    const float eta_t = P.eta[t];
    for (int i = 0; i < n; ++i) {  // Eq. 4 for every spin, all reading s(t)
      const double x = static_cast<double>(b_t) * I[i];
      const float tau = P.act == 0 ? static_cast<float>(std::tanh(x))
                                   : static_cast<float>(lut_staircase(x, P.lut_levels));
      const float a = tau + (s[i] > 0 ? P.xi : -P.xi);
      const float noise = eta_t * P.z[d[i] >> 4];
      const float delta = a + noise;
      next[i] = delta >= 0.0f ? 1 : -1;
    }
    std::memcpy(s, next.data(), n);
  }
  const double E = field_energy(P, s, I.data());
  bookkeep(E, P.t_begin + P.sweeps);
  *final_E = E;
}

}  // namespace

extern "C" {

// The 4096 noise levels (noise 0: Gaussian quantiles, 1: uniform grid).
void pimi_oracle_noise_levels(int noise, float* out) {
  if (noise == 0)
    gauss_table(out);
  else
    uniform_table(out);
}

// One Philox4x32-10 block.
void pimi_oracle_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out) {
  philox(ctr, k0, k1, out);
}

// Anneal of one instance.
//   real = 0: J int8 n x n, h int32[n] or NULL;  real = 1: J double n x n, h double[n] or NULL.
//   R replicas with indices replica_ids[0..R) (NULL: 0 .. R-1).
//   Start state: cont != 0 -> final_state holds s(t_begin) and best_E / best_t / first_hit /
//   best_state hold the previous records; else init (R x n, or NULL for the Philox draw).
//   Outputs per replica: best_E, best_t, first_hit (-1: none), final_E, best_state and
//   final_state (R x n int8).  threads <= 0: all hardware threads.  Returns 0, or -1 for
//   bad arguments.
int pimi_oracle_anneal(int n, int real, const void* J, const void* h, double c, const float* beta,
                       const float* eta, float xi, int noise, int act, int lut_levels, int R,
                       const int64_t* replica_ids, int t_begin, int sweeps, uint64_t seed,
                       uint32_t q, const int8_t* init, int cont, int has_target, double target,
                       int threads, double* best_E, int32_t* best_t, int32_t* first_hit,
                       double* final_E, int8_t* best_state, int8_t* final_state) {
  if (n < 1 || R < 1 || sweeps < 0 || t_begin < 0 || !J || !beta || !eta || !best_E || !best_t ||
      !first_hit || !final_E || !best_state || !final_state || (act == 1 && lut_levels < 2))
    return -1;
  std::vector<float> z(kLevels);
  if (noise == 0)
    gauss_table(z.data());
  else
    uniform_table(z.data());
  Problem P{};
  P.n = n;
  P.real = real;
  P.J8 = real ? nullptr : static_cast<const int8_t*>(J);
  P.Jd = real ? static_cast<const double*>(J) : nullptr;
  P.h32 = real ? nullptr : static_cast<const int32_t*>(h);
  P.hd = real ? static_cast<const double*>(h) : nullptr;
  P.c = c;
  P.beta = beta;
  P.eta = eta;
  P.xi = xi;
  P.act = act;
  P.lut_levels = lut_levels;
  P.z = z.data();
  P.t_begin = t_begin;
  P.sweeps = sweeps;
  P.seed = seed;
  P.q = q;
  P.has_target = has_target;
  P.target = target;

  auto work = [&](int r0, int r1) {
    std::vector<uint16_t> d(n);
    for (int k = r0; k < r1; ++k) {
      const uint32_t r = static_cast<uint32_t>(replica_ids ? replica_ids[k] : k);
      int8_t* s = final_state + static_cast<size_t>(k) * n;
      int8_t* bs = best_state + static_cast<size_t>(k) * n;
      if (!cont) {
        if (init) {
          std::memcpy(s, init + static_cast<size_t>(k) * n, n);
        } else {
          draws(seed, q, r, 0xFFFFFFFFu, n, d.data());
          for (int i = 0; i < n; ++i) s[i] = ((d[i] >> 15) & 1) ? 1 : -1;
        }
        best_E[k] = INFINITY;
        best_t[k] = -1;
        first_hit[k] = -1;
        std::memcpy(bs, s, n);
      }
      run_replica(P, r, s, &best_E[k], &best_t[k], &first_hit[k], &final_E[k], bs);
    }
  };
  int nt = threads > 0 ? threads : static_cast<int>(std::thread::hardware_concurrency());
  nt = std::max(1, std::min(nt, R));
  if (nt == 1) {
    work(0, R);
    return 0;
  }
  std::vector<std::thread> pool;
  for (int k = 0; k < nt; ++k) {
    const int r0 = static_cast<int>(static_cast<long long>(R) * k / nt);
    const int r1 = static_cast<int>(static_cast<long long>(R) * (k + 1) / nt);
    pool.emplace_back(work, r0, r1);
  }
  for (auto& th : pool) th.join();
  return 0;
}

}  // extern "C"
