// Measurement probes of the GB300 units the sweep kernels are bound by (not part of any
// anneal): the tcgen05 tensor-pipe rate of each operand kind the kernels use, and the rate
// at which one SM takes in cp.async.bulk copies from L2 while every SM does the same.
// The roofline of a kernel uses the measured BF16 rate and a nominal ratio for FP8 / E2M1;
// these probes put a measured number beside it.
//
//   MMA probe     one CTA per SM; one thread issues `iters` MMAs of M = 128, N = 256 and the
//                 kind's K (FP8 E4M3 kind::f8f6f4: 32, BF16 kind::f16: 16, E2M1
//                 kind::mxf4.block_scale with unit scales: 64) back to back on operands in
//                 shared memory, accumulating into one TMEM accumulator, then commits and
//                 waits (bounded).  Rate = all CTAs' flops / the longest CTA time.
//   ingest probe  one CTA per SM; a producer thread streams `iters` copies of `bytes` from
//                 an L2-resident source through a 4-stage shared-memory ring, a consumer
//                 thread releases each stage as soon as it lands (no compute).  Mode 0: every
//                 CTA reads its own region; mode 1: all CTAs read the same region (as the
//                 tiles of one spin image are read by every column block).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "kernels.h"
#include "pim.h"
#include "sm100_ptx.cuh"

#define PIM_API extern "C" __attribute__((visibility("default")))

namespace pim {
namespace {

constexpr int kProbeThreads = 128;
constexpr int kABytes = 128 * 128;   // one 128-byte-wide K-block of A (128 rows)
constexpr int kBBytes = 256 * 128;   // one K-block of B (256 rows)
constexpr int kRing = 4;

// out[cta] = nanoseconds from the first MMA issue to the completion of the last one, or
// 0 when a wait gave up.
template <int KIND>  // 0 FP8 E4M3, 1 BF16, 2 E2M1 block-scaled
__global__ void __launch_bounds__(kProbeThreads, 1) probe_mma_kernel(int iters,
                                                                   unsigned long long* out) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + kABytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + kBBytes);
  uint32_t* sT = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < (kABytes + kBBytes) / 16; i += kProbeThreads)
    reinterpret_cast<uint4*>(sA)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    tmem_alloc(smem_u32(sT), 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(smem_u32(bar), 1);
    fence_mbar_init();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sT;
  if (KIND == 2) {  // unit scale factors in columns 256..511
    for (int c = 256; c < 512; c += 32)
      tmem_fill32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c, 0x7F7F7F7Fu);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    const uint32_t idesc = KIND == 0 ? idesc_e4m3(128, 256)
                                     : (KIND == 1 ? idesc_bf16(128, 256) : idesc_mxf4(128, 256));
    const uint64_t t0 = global_ns();
    for (int i = 0; i < iters; ++i) {
      const uint32_t ks = static_cast<uint32_t>(i & 3) * 32;
      const uint64_t a = sw128_desc(smem_u32(sA) + ks), b = sw128_desc(smem_u32(sB) + ks);
      if (KIND == 0)
        mma_e4m3(tmem, a, b, idesc, i > 0 ? 1u : 0u);
      else if (KIND == 1)
        mma_bf16(tmem, a, b, idesc, i > 0 ? 1u : 0u);
      else
        mma_mxf4(tmem, a, b, idesc, tmem + 256, tmem + 256, i > 0 ? 1u : 0u);
    }
    mma_commit(smem_u32(bar));
    const bool ok = mbar_wait_bounded(smem_u32(bar), 0, 2000000000ull);
    out[blockIdx.x] = ok ? global_ns() - t0 : 0ull;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// out[cta] = nanoseconds for `iters` copies of `bytes` each, or 0 when a wait gave up.
__global__ void __launch_bounds__(kProbeThreads, 1) probe_ingest_kernel(const uint8_t* src,
                                                                      size_t region, int bytes,
                                                                      int iters, int shared,
                                                                      unsigned long long* out) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kRing * static_cast<size_t>(bytes));
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kRing]);
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kRing; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const size_t base = shared ? 0 : static_cast<size_t>(blockIdx.x) * region;
  const size_t per_region = region / static_cast<size_t>(bytes);
  bool ok = true;
  const uint64_t t0 = global_ns();
  if (tid == 0) {
    for (int i = 0; i < iters && ok; ++i) {
      const uint32_t s = i % kRing, use = i / kRing;
      if (use > 0 && !mbar_wait_bounded(empty0 + 8 * s, (use - 1) & 1, 2000000000ull)) ok = false;
      if (!ok) break;
      mbar_expect_tx(full0 + 8 * s, static_cast<uint32_t>(bytes));
      bulk_g2s(smem_u32(smem + s * static_cast<size_t>(bytes)),
               src + base + (static_cast<size_t>(i) % per_region) * bytes, static_cast<uint32_t>(bytes),
               full0 + 8 * s);
    }
  } else if (tid == 32) {
    for (int i = 0; i < iters && ok; ++i) {
      const uint32_t s = i % kRing, use = i / kRing;
      if (!mbar_wait_bounded(full0 + 8 * s, use & 1, 2000000000ull)) ok = false;
      if (!ok) break;
      mbar_arrive(empty0 + 8 * s);
    }
    out[blockIdx.x] = ok ? global_ns() - t0 : 0ull;
  }
  // every issued copy has landed before the CTA exits
  if (tid == 0)
    for (int i = iters > kRing ? iters - kRing : 0; i < iters; ++i)
      mbar_wait_bounded(full0 + 8 * (i % kRing), (i / kRing) & 1, 2000000000ull);
  __syncthreads();
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, sms);
}

// Longest per-CTA time of a probe launch (ns), 0 on failure.
unsigned long long longest(unsigned long long* d_out, int n) {
  std::vector<unsigned long long> h(n);
  if (cudaMemcpy(h.data(), d_out, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
    return 0;
  unsigned long long m = 0;
  for (unsigned long long v : h) {
    if (v == 0) return 0;
    m = std::max(m, v);
  }
  return m;
}

}  // namespace
}  // namespace pim

using namespace pim;

PIM_API int pim_probe_tensor(int kind, int iters, double* tflops) {
  if (kind < 0 || kind > 2 || iters < 1 || !tflops) {
    set_last_error("pim_probe_tensor: kind must be 0 (FP8), 1 (BF16) or 2 (E2M1), iters >= 1");
    return PIM_ERR_INVALID;
  }
  const int sms = sm_count();
  const int smem = 1024 + kABytes + kBBytes + 64;
  const int force_one = 120 * 1024;  // one CTA per SM
  const int dyn = std::max(smem, force_one);
  unsigned long long* d_out = nullptr;
  if (cudaMalloc(&d_out, sms * sizeof(unsigned long long)) != cudaSuccess) {
    set_last_error("pim_probe_tensor: cudaMalloc failed");
    return PIM_ERR_NOMEM;
  }
  cudaError_t e = cudaSuccess;
  auto run = [&](auto kernel) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e == cudaSuccess) {
      kernel<<<sms, kProbeThreads, dyn>>>(iters, d_out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  };
  if (kind == 0) run(probe_mma_kernel<0>);
  if (kind == 1) run(probe_mma_kernel<1>);
  if (kind == 2) run(probe_mma_kernel<2>);
  const unsigned long long ns = e == cudaSuccess ? longest(d_out, sms) : 0;
  cudaFree(d_out);
  if (e != cudaSuccess || ns == 0) {
    set_last_error("pim_probe_tensor: probe launch failed or a wait gave up");
    return e != cudaSuccess ? PIM_ERR_CUDA : PIM_ERR_TIMEOUT;
  }
  const double k = kind == 0 ? 32.0 : (kind == 1 ? 16.0 : 64.0);
  *tflops = 2.0 * 128 * 256 * k * iters * sms / (static_cast<double>(ns) * 1e-9) / 1e12;
  return PIM_OK;
}

PIM_API int pim_probe_ingest(int bytes, int iters, int shared, double* gbs_per_sm) {
  if (bytes < 16 || bytes % 16 || bytes > 32768 || iters < 1 || !gbs_per_sm) {
    set_last_error("pim_probe_ingest: bytes a multiple of 16 in [16, 32768], iters >= 1");
    return PIM_ERR_INVALID;
  }
  const int sms = sm_count();
  const size_t region = size_t(256) << 10;  // 256 KB per CTA (L2-resident: 38 MB in all)
  const size_t total = shared ? region : region * sms;
  uint8_t* d_src = nullptr;
  unsigned long long* d_out = nullptr;
  if (cudaMalloc(&d_src, total) != cudaSuccess ||
      cudaMalloc(&d_out, sms * sizeof(unsigned long long)) != cudaSuccess) {
    if (d_src) cudaFree(d_src);
    set_last_error("pim_probe_ingest: cudaMalloc failed");
    return PIM_ERR_NOMEM;
  }
  cudaError_t e = cudaMemset(d_src, 1, total);
  const int dyn = std::max(1024 + kRing * bytes + 2 * kRing * 8, 120 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(probe_ingest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // pass 0 brings the source into L2
    probe_ingest_kernel<<<sms, kProbeThreads, dyn>>>(d_src, region, bytes, iters, shared, d_out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  const unsigned long long ns = e == cudaSuccess ? longest(d_out, sms) : 0;
  cudaFree(d_src);
  cudaFree(d_out);
  if (e != cudaSuccess || ns == 0) {
    set_last_error("pim_probe_ingest: probe launch failed or a wait gave up");
    return e != cudaSuccess ? PIM_ERR_CUDA : PIM_ERR_TIMEOUT;
  }
  *gbs_per_sm = static_cast<double>(bytes) * iters / static_cast<double>(ns);
  return PIM_OK;
}
