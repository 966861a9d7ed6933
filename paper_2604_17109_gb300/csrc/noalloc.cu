// pim_anneal_noalloc: the fused sweep path for callers that cannot allocate device memory.
//
// Everything the path needs besides the caller's inputs and outputs (staged couplings,
// activation values, decision tables, launch descriptors, the device error word) lives in
// one file-scope device array of fixed size.  Host-side staging uses file-scope host
// arrays.  No call here allocates.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "host_tables.h"
#include "kernels.h"
#include "pim.h"

#define PIM_API extern "C" __attribute__((visibility("default")))

namespace {

using namespace pim;

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxN = PIM_NOALLOC_MAX_N;
constexpr int kMaxSteps = PIM_NOALLOC_MAX_STEPS;
constexpr int kMaxReplicas = PIM_NOALLOC_MAX_REPLICAS;
constexpr int kTableImax = 255;                     // field range covered by the tables
constexpr int kTauWidth = 2 * kTableImax + 1;       // tau entries per step
constexpr int kStrideWords = (kTauWidth + 3) & ~3;  // general table words per step
constexpr int kMaxDevices = 64;

// The scratch array.  In host code its name is only a stand-in: the device address comes
// from cudaGetSymbolAddress, taken once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host staging (file scope, reused by every call under g_mu).
float g_tau[static_cast<size_t>(kMaxSteps) * kTauWidth];
float g_z[kNoiseLevels];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
int g_err_host = 0;  // error word read back after each call

// Byte offsets of the regions inside the scratch array (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffErr = 0;
constexpr size_t kOffProb = align256(kOffErr + sizeof(int));
constexpr size_t kOffWork = align256(kOffProb + sizeof(Problem));
constexpr size_t kOffJ = align256(kOffWork + sizeof(WorkItem) * (kMaxReplicas / 128));
constexpr size_t kOffImg = align256(kOffJ + size_t(kMaxN) * kMaxN);
constexpr size_t kOffZ = align256(kOffImg + size_t(kMaxN) * kMaxN);
constexpr size_t kOffEta = align256(kOffZ + sizeof(float) * kNoiseLevels);
constexpr size_t kOffTau = align256(kOffEta + sizeof(float) * kMaxSteps);
constexpr size_t kOffThr = align256(kOffTau + sizeof(float) * kMaxSteps * kTauWidth);
constexpr size_t kOffDiag = align256(kOffThr + sizeof(uint32_t) * kMaxSteps * kStrideWords);
constexpr size_t kEnd = kOffDiag + size_t(2) * 1024 * kMaxSteps;
static_assert(kEnd <= kScratchBytes, "scratch layout exceeds the static array");

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

}  // namespace

#define CKN(call, what)                                                              \
  do {                                                                               \
    const cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                           \
      return fail(PIM_ERR_CUDA, "pim_anneal_noalloc: %s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

PIM_API int pim_anneal_noalloc(int n, const int8_t* J, double scale_c, int steps,
                               const float* beta, const float* eta, float xi, int replicas,
                               uint64_t seed, uint32_t instance_id, double target_energy,
                               double* best_E, int32_t* best_t, int32_t* first_hit_t,
                               double* final_E, uint32_t* best_bits, uint32_t* final_bits,
                               void* cuda_stream) {
  if (n < 1 || n > kMaxN)
    return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: n = %d outside [1, %d]", n, kMaxN);
  if (steps < 1 || steps > kMaxSteps)
    return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: steps = %d outside [1, %d]", steps, kMaxSteps);
  if (replicas < 1 || replicas > kMaxReplicas)
    return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: replicas = %d outside [1, %d]", replicas,
                kMaxReplicas);
  if (!J || !beta || !eta || !best_E || !best_t || !first_hit_t || !final_E || !best_bits ||
      !final_bits)
    return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: NULL input or output pointer");
  if (!(scale_c > 0.0) || !std::isfinite(scale_c) || !std::isfinite(xi) || xi < 0.0f)
    return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: scale_c must be > 0 and xi >= 0, finite");
  if (!std::isnan(target_energy) && !std::isfinite(target_energy))
    return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: target must be finite or NaN");
  int imax = 0;
  for (int i = 0; i < n; ++i) {
    if (J[static_cast<size_t>(i) * n + i] != 0)
      return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: J[%d][%d] != 0", i, i);
    int row = 0;
    for (int j = 0; j < n; ++j) {
      const int v = J[static_cast<size_t>(i) * n + j];
      if (v != J[static_cast<size_t>(j) * n + i])
        return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: J not symmetric at (%d, %d)", i, j);
      if (v < -16 || v > 16)
        return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: |J[%d][%d]| > 16", i, j);
      row += v < 0 ? -v : v;
    }
    if (row > imax) imax = row;
  }
  if (imax > kTableImax)
    return fail(PIM_ERR_INVALID,
                "pim_anneal_noalloc: max_i sum_j |J_ij| = %d exceeds %d", imax, kTableImax);
  for (int t = 0; t < steps; ++t)
    if (!std::isfinite(beta[t]) || beta[t] < 0.0f || !std::isfinite(eta[t]) || eta[t] < 0.0f)
      return fail(PIM_ERR_INVALID, "pim_anneal_noalloc: beta/eta[%d] must be finite, >= 0", t);

  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  CKN(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return fail(PIM_ERR_UNSUPPORTED, "pim_anneal_noalloc: device %d out of range", dev);
  if (!g_scratch_addr[dev]) {
    void* addr = nullptr;
    CKN(cudaGetSymbolAddress(&addr, g_noalloc_scratch), "cudaGetSymbolAddress");
    g_scratch_addr[dev] = addr;
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* d_err = reinterpret_cast<int*>(base + kOffErr);
  Problem* d_prob = reinterpret_cast<Problem*>(base + kOffProb);
  WorkItem* d_work = reinterpret_cast<WorkItem*>(base + kOffWork);
  int8_t* d_J = reinterpret_cast<int8_t*>(base + kOffJ);
  uint8_t* d_img = base + kOffImg;
  float* d_z = reinterpret_cast<float*>(base + kOffZ);
  float* d_eta = reinterpret_cast<float*>(base + kOffEta);
  float* d_tau = reinterpret_cast<float*>(base + kOffTau);
  uint32_t* d_thr = reinterpret_cast<uint32_t*>(base + kOffThr);
  uint32_t* d_diag = reinterpret_cast<uint32_t*>(base + kOffDiag);

  // Host-side constant tables for this schedule.
  for (int t = 0; t < steps; ++t)
    activation_levels(scaled_beta(beta[t], scale_c), kTableImax, 0, 0,
                      &g_tau[static_cast<size_t>(t) * kTauWidth]);
  noise_levels(0, g_z);

  const int npad = n <= 128 ? 128 : 256;
  const int words = ((n + 63) / 64) * 2;
  Problem P{};
  P.jimg = d_img;
  P.thr = d_thr;
  P.thr_diag = d_diag;
  P.diag_img = 1;
  P.best_E = best_E;
  P.final_E = final_E;
  P.best_t = best_t;
  P.first_hit = first_hit_t;
  P.best_bits = best_bits;
  P.cur_bits = final_bits;
  P.n = n;
  P.npad = npad;
  P.words = words;
  P.imax = kTableImax;
  P.stride_words = kStrideWords;
  P.R = replicas;
  P.q = instance_id;
  P.has_target = std::isnan(target_energy) ? 0 : 1;
  P.target = std::isnan(target_energy) ? 0 : static_cast<long long>(std::floor(target_energy));
  WorkItem work[kMaxReplicas / 128];
  int nwork = 0;
  for (int rb = 0; rb < replicas; rb += 128) work[nwork++] = WorkItem{0, rb};

  // The error word must start at zero; every other region is fully rewritten below.
  CKN(cudaMemsetAsync(d_err, 0, sizeof(int), st), "clear error word");
  CKN(cudaMemcpyAsync(d_J, J, static_cast<size_t>(n) * n, cudaMemcpyHostToDevice, st), "upload J");
  CKN(cudaMemcpyAsync(d_prob, &P, sizeof(P), cudaMemcpyHostToDevice, st), "upload descriptor");
  CKN(cudaMemcpyAsync(d_work, work, sizeof(WorkItem) * nwork, cudaMemcpyHostToDevice, st),
      "upload work list");
  CKN(cudaMemcpyAsync(d_z, g_z, sizeof(g_z), cudaMemcpyHostToDevice, st), "upload noise levels");
  CKN(cudaMemcpyAsync(d_eta, eta, sizeof(float) * steps, cudaMemcpyHostToDevice, st), "upload eta");
  CKN(cudaMemcpyAsync(d_tau, g_tau, sizeof(float) * kTauWidth * steps, cudaMemcpyHostToDevice, st),
      "upload activation values");
  CKN(launch_stage_fp8_image(d_J, n, npad, 256, d_img, st), "stage couplings");
  CKN(launch_thresholds(d_tau, d_eta, d_z, xi, steps, kTableImax, kStrideWords, d_thr, st),
      "decision thresholds");
  CKN(launch_diag_thresholds(d_thr, steps, kTableImax, kStrideWords, 256, d_diag, st),
      "diagonal thresholds");
  CKN(launch_init_bits(d_prob, 1, replicas, words, nullptr, static_cast<uint32_t>(seed),
                       static_cast<uint32_t>(seed >> 32), st),
      "initial spins");
  Launch L{};
  L.probs = d_prob;
  L.work = d_work;
  L.nwork = nwork;
  L.t_begin = 0;
  L.sweeps = steps;
  L.key_lo = static_cast<uint32_t>(seed);
  L.key_hi = static_cast<uint32_t>(seed >> 32);
  philox_round_keys(seed, L.round_keys);
  L.cont = 0;
  L.stride_words_max = kStrideWords;
  L.err = d_err;
  CKN(launch_sweep_tc(L, npad, nwork, st, true), "fused sweep kernel");
  // The error word comes back on the caller's stream (a copy on the legacy default stream
  // would also wait for unrelated work on every other blocking stream of the device).
  g_err_host = 0;
  CKN(cudaMemcpyAsync(&g_err_host, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "read error word");
  CKN(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  const int h_err = g_err_host;
  if (h_err & kDevErrTimeout)
    return fail(PIM_ERR_TIMEOUT, "pim_anneal_noalloc: a device-side bounded wait gave up");
  if (h_err) return fail(PIM_ERR_CUDA, "pim_anneal_noalloc: device error bits 0x%x", h_err);
  return PIM_OK;
}
