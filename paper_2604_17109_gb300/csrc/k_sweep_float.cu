// Fused PIMI sweep kernel for real-valued couplings (n <= 256): BF16 operands on the
// tcgen05 tensor path (kind::f16, FP32 accumulation), decision in FP32.
//
// Same structure as the integer kernel (one CTA = one instance x 128-replica tile, all
// sweeps inside, TMEM lane = replica, 4 lane quadrants x 2 column halves of threads), with:
//   operands  A = spins as BF16 +-1 (exact), B = J rounded to BF16, both K-major with the
//             128-byte swizzle; K advances 16 elements (32 bytes) per MMA.
//   decision  Eq. 4 evaluated directly: x = b_t (I + h), tau = tanh(x) (or the L-level
//             staircase of Algorithm "LUT-based tanh approximation"),
//             delta = (tau + xi s) + eta_t z(key), s' = +1 iff delta >= 0, with the same
//             Philox draws and 4096 noise levels as the integer path.
//   energy    H = -1/2 sum_i s_i (I_i + h_i) accumulated in FP32.
// Fixed-point datapath (P.fix_w > 0, npad 128): the couplings are Q(c J) in
// ap_fixed<W, W - F> (supplementary quantization section), held as two BF16 images whose sum
// is exact (high part + low part), so the two MMA chains give the exact field I in FP32
// (|I| 2^F < 2^24).  The decision then follows the datapath on integers in units of 2^-F:
//   u = sat(I), x = Q(fl32(beta_t) u), tau = table(x), a = sat(tau + s Q(xi)),
//   n = sat(trunc(Q(eta_t) Q(z) / 2^F)), s' = +1 iff sat(a + n) >= 0,
// and the energy is summed exactly in integers.
#include <cfloat>

#include "kernels.h"
#include "philox.cuh"
#include "sm100_ptx.cuh"

namespace pim {
namespace {

constexpr int kThreads = 256;
constexpr int kTileM = 128;

// Fixed-point decision of one spin (see the header): integers in units of 2^-F.
__device__ __forceinline__ uint32_t fixed_decide(float I, uint32_t s, float beta, int eta_q,
                                                 int z_q, int xi_q, int F, int half_range,
                                                 const int32_t* __restrict__ tau_tab) {
  const int lo = -half_range, hi = half_range - 1;
  const int mI = __float2int_rz(__fmul_rn(I, __int_as_float((127 + F) << 23)));  // I 2^F, exact
  const int mu = min(max(mI, lo), hi);
  // Q(beta u): the product of a 24-bit and a 16-bit integer is exact in double
  long long mx = static_cast<long long>(__dmul_rn(static_cast<double>(beta), static_cast<double>(mu)));
  mx = mx < lo ? lo : (mx > hi ? hi : mx);
  const int mt = __ldg(tau_tab + (mx + half_range));
  const int ma = min(max(mt + (s ? xi_q : -xi_q), lo), hi);
  const int mn = min(max((eta_q * z_q) / (1 << F), lo), hi);  // truncation toward zero
  const int md = min(max(ma + mn, lo), hi);
  return md >= 0 ? 1u : 0u;
}

__device__ __forceinline__ uint32_t ld_acquire_sys(const unsigned int* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys(unsigned int* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Serving kernel, one thread: the next request of the queue, or -1 when the queue stayed
// empty for Q.idle_ns or the host asked the kernel to stop (the reason goes to exit_status).
__device__ int serve_claim(const ServeQueue& Q) {
  const uint64_t t0 = global_ns();
  for (;;) {
    const uint32_t h = *reinterpret_cast<volatile unsigned int*>(Q.head);
    const uint32_t tl = ld_acquire_sys(Q.tail);
    if (h < tl) {
      if (atomicCAS(Q.head, h, h + 1) == h) return static_cast<int>(h);
      continue;
    }
    if (*reinterpret_cast<const volatile unsigned int*>(Q.stop) != 0) {
      atomicCAS(Q.exit_status, 0, 2);
      return -1;
    }
    if (global_ns() - t0 > Q.idle_ns) {
      atomicCAS(Q.exit_status, 0, 1);
      return -1;
    }
    __nanosleep(256);
  }
}

// SERVE = false: CTA b runs work item b of L (one instance x 128-replica tile).
// SERVE = true: persistent CTAs take requests from the queue Q one after another (each a
// whole instance of at most 128 replicas, initial spins from Philox, float32 decisions);
// the request's descriptor, couplings and bias are read from mapped host memory with loads
// that bypass the caches (a slot is rewritten for later requests), and the results go back
// there before the slot's done flag.
template <int NPAD, bool SERVE>
__global__ void __launch_bounds__(kThreads, 1) sweep_float_kernel(const Launch L, const ServeQueue Q) {
  constexpr int kMaxSlots = NPAD / 32;
  constexpr int kWordsPerThread = kMaxSlots / 2;
  constexpr int kRowBytes = 2 * NPAD;  // bytes of one operand row (K = NPAD BF16 values)
  constexpr bool kCanFix = NPAD == 128 && !SERVE;  // room for the second coupling image
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sJ = smem;                                  // NPAD x kRowBytes (x2: high | low part)
  uint8_t* sA = sJ + (NPAD == 128 ? 2 : 1) * NPAD * kRowBytes;  // 128 x kRowBytes
  float* sZ = reinterpret_cast<float*>(sA + kTileM * kRowBytes);  // 4096
  float* sH = sZ + 4096;                               // NPAD
  float* sPart = sH + NPAD;                            // [2][2][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sPart + 2 * 2 * kTileM);
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + 2);
  int* sAbort = reinterpret_cast<int*>(sTmem + 1);     // [0] abort, [1] request
  Problem* sProb = reinterpret_cast<Problem*>(bars + 4);  // SERVE: the request's descriptor

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane;
  const uint32_t bar_mma = smem_u32(&bars[0]);
  const uint32_t bar_j = smem_u32(&bars[1]);

  if (warp == 0) {
    tmem_alloc(smem_u32(sTmem), NPAD);
    tmem_relinquish();
  }
  if (tid == 32) {
    mbar_init(bar_mma, 1);
    mbar_init(bar_j, 1);
    fence_mbar_init();
    sAbort[0] = 0;
  }
  if constexpr (SERVE)
    for (int k = tid; k < 4096; k += kThreads) sZ[k] = Q.zlev[k];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t tmem_warp = tmem + (static_cast<uint32_t>(quad * 32) << 16);
  uint32_t phase = 0, jphase = 0;
  bool aborted = false;

  for (int unit = 0; !aborted; ++unit) {
    // ---- unit: this CTA's work item, or the next request of the queue -----------------
    int req = 0;
    if constexpr (SERVE) {
      if (tid == 0) sAbort[1] = serve_claim(Q);
      __syncthreads();
      req = sAbort[1];
      if (req < 0) break;
      const volatile int* src = reinterpret_cast<const volatile int*>(
          Q.slots + static_cast<size_t>(req % Q.nslots) * Q.slot_bytes);
      for (int k = tid; k < static_cast<int>(sizeof(Problem) / 4); k += kThreads)
        reinterpret_cast<int*>(sProb)[k] = src[k];
      __syncthreads();
    } else {
      if (unit > 0) break;
    }
    const WorkItem wk = SERVE ? WorkItem{0, 0} : L.work[blockIdx.x];
    const Problem& P = SERVE ? *sProb : L.probs[wk.prob];
    const int n = P.n, R = P.R;
    const uint32_t q = P.q;
    const int rg = wk.rbase + row;
    const bool row_valid = rg < R;
    const bool warp_active = (wk.rbase + quad * 32) < R;
    const int nch = (n + 15) >> 4;
    const int split = (n + 16) >> 5;
    const int c0 = half == 0 ? 0 : split;
    const int myc = half == 0 ? split : nch - split;
    const int ksteps = (n + 15) >> 4;      // 16 BF16 values per MMA
    const int mma_n = (n + 15) & ~15;
    const int t_begin = L.t_begin, t_end = L.t_begin + L.sweeps;
    const float xi = P.xi;
    const int act = P.act, levels = P.lut_levels;
    const bool fixed = kCanFix && P.fix_w > 0;
    const int fix_f = P.fix_f, fix_half = fixed ? 1 << (P.fix_w - 1) : 0, fix_xi = P.fix_xi;
    const float fix_scale = __int_as_float((127 + fix_f) << 23);  // 2^F

    // ---- prologue: zeroed A operand, noise levels, bias, coupling image -----------------
    for (int k = tid; k < kTileM * kRowBytes / 16; k += kThreads)
      reinterpret_cast<uint4*>(sA)[k] = make_uint4(0, 0, 0, 0);
    if constexpr (SERVE) {
      for (int k = tid; k < NPAD; k += kThreads)
        sH[k] = (P.hf != nullptr && k < n) ? __ldcv(P.hf + k) : 0.0f;
      const uint4* jsrc = reinterpret_cast<const uint4*>(P.jimg);
      for (int k = tid; k < NPAD * kRowBytes / 16; k += kThreads)
        reinterpret_cast<uint4*>(sJ)[k] = __ldcv(jsrc + k);
    } else {
      for (int k = tid; k < 4096; k += kThreads) sZ[k] = fixed ? __int_as_float(P.fix_z[k]) : P.zlev[k];
      for (int k = tid; k < NPAD; k += kThreads) sH[k] = (P.hf != nullptr && k < n) ? P.hf[k] : 0.0f;
    }
    __syncthreads();
    if (!SERVE && tid == 0) {
      constexpr uint32_t kJBytes = NPAD * kRowBytes;
      mbar_expect_tx(bar_j, fixed ? 2 * kJBytes : kJBytes);
      for (int part = 0; part < (fixed ? 2 : 1); ++part) {
        const uint8_t* src = part ? P.jimg_lo : P.jimg;
        for (uint32_t off = 0; off < kJBytes; off += 16384)
          bulk_g2s(smem_u32(sJ + part * kJBytes + off), src + off,
                   16384u < kJBytes - off ? 16384u : kJBytes - off, bar_j);
      }
    }

    uint32_t cur[kWordsPerThread], best[kWordsPerThread];
#pragma unroll
    for (int w = 0; w < kWordsPerThread; ++w) cur[w] = 0;
    if constexpr (SERVE) {
      // initial spins: bit 15 of the draw at step field 0xFFFFFFFF (one Philox block per 8)
      if (row_valid) {
#pragma unroll
        for (int k = 0; k < kMaxSlots; ++k)
          if (k < myc) {
            const int c = c0 + k;
            uint32_t nb = 0;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              const PhiloxOut o = philox4x32_10_rk(2u * c + g, static_cast<uint32_t>(rg), 0xFFFFFFFFu,
                                                   q, L.round_keys);
#pragma unroll
              for (int e = 0; e < 8; ++e) nb |= ((philox_half(o, e) >> 15) & 1u) << (8 * g + e);
            }
            const int valid = n - c * 16;
            if (valid < 16) nb &= (1u << valid) - 1u;
            cur[k >> 1] |= nb << ((k & 1) * 16);
          }
      }
    } else {
      const uint16_t* cur_in = reinterpret_cast<const uint16_t*>(P.cur_bits);
      if (row_valid) {
#pragma unroll
        for (int k = 0; k < kMaxSlots; ++k)
          if (k < myc) cur[k >> 1] |= static_cast<uint32_t>(cur_in[static_cast<size_t>(rg) * P.words * 2 + (c0 + k)]) << ((k & 1) * 16);
      }
    }
    double best_E = DBL_MAX;  // float32 energies (float mode) or exact ones (fixed mode)
    int best_t = -1, first_hit = -1;
    const bool has_target = P.has_target != 0;
    const double target = P.target_f;
    if (!SERVE && L.cont && row_valid) {
      best_E = P.best_E[rg];
      best_t = P.best_t[rg];
      first_hit = P.first_hit[rg];
      const uint16_t* best_in = reinterpret_cast<const uint16_t*>(P.best_bits);
#pragma unroll
      for (int w = 0; w < kWordsPerThread; ++w) best[w] = 0;
#pragma unroll
      for (int k = 0; k < kMaxSlots; ++k)
        if (k < myc) best[k >> 1] |= static_cast<uint32_t>(best_in[static_cast<size_t>(rg) * P.words * 2 + (c0 + k)]) << ((k & 1) * 16);
    } else {
#pragma unroll
      for (int w = 0; w < kWordsPerThread; ++w) best[w] = cur[w];
    }

    // Spins of 16 columns (chunk c) -> 32 bytes of the A operand row.
    auto write_chunk = [&](int c, uint32_t nb) {
      const int kbyte = c * 32;
      *reinterpret_cast<uint4*>(sA + sw128_offset(row, kbyte, kTileM)) = bf16x8_from_bits(nb & 0xFFu);
      *reinterpret_cast<uint4*>(sA + sw128_offset(row, kbyte + 16, kTileM)) = bf16x8_from_bits(nb >> 8);
    };
    if (warp_active) {
#pragma unroll
      for (int k = 0; k < kMaxSlots; ++k)
        if (k < myc) write_chunk(c0 + k, (cur[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu);
    }
    fence_proxy_async_smem();  // the A operand (and, serving, the coupling image)
    __syncthreads();

    const uint32_t idesc = idesc_bf16(kTileM, mma_n);
    const uint32_t sA_addr = smem_u32(sA), sJ_addr = smem_u32(sJ);
    auto issue_fields = [&]() {
      for (int part = 0; part < (fixed ? 2 : 1); ++part)  // fixed mode: high part, then low part
        for (int ks = 0; ks < ksteps; ++ks) {
          const uint32_t kb = ks >> 2, ko = (ks & 3) * 32;
          mma_bf16(tmem, sw128_desc(sA_addr + kb * (kTileM * 128) + ko),
                   sw128_desc(sJ_addr + part * (NPAD * kRowBytes) + kb * (NPAD * 128) + ko), idesc,
                   (ks > 0 || part > 0) ? 1u : 0u);
        }
      mma_commit(bar_mma);
    };
    if (tid == 0) {
      if (!SERVE && !mbar_wait_bounded(bar_j, jphase, L.wait_ns)) {
        atomicOr(L.err, kDevErrTimeout);
        sAbort[0] = 1;
      } else if (L.inject != 1) {  // injected fault: the first wait below cannot complete
        tc_fence_after();
        issue_fields();
      }
    }
    jphase ^= 1u;
    __syncthreads();
    aborted = sAbort[0] != 0;

    for (int t = t_begin; t <= t_end && !aborted; ++t) {
      const bool last = t == t_end;
      if (!mbar_wait_bounded(bar_mma, phase, L.wait_ns)) {
        atomicOr(L.err, kDevErrTimeout);
        sAbort[0] = 1;
      }
      phase ^= 1;
      tc_fence_after();
      const float b = last ? 0.0f : P.sched_b[t];
      const float eta = last ? 0.0f : P.sched_eta[t];
      const int eta_q = (fixed && !last) ? P.fix_eta[t] : 0;
      float* dump = (!SERVE && P.fields_out != nullptr && t == t_begin && !last && row_valid)
                        ? P.fields_out + static_cast<size_t>(rg) * n
                        : nullptr;
      uint32_t nxt[kWordsPerThread];
#pragma unroll
      for (int w = 0; w < kWordsPerThread; ++w) nxt[w] = 0;
      float eacc = 0.0f;
      int ieacc = 0;  // fixed mode: sum_i s_i (I_i + h_i) in units of 2^-F, exact
      if (warp_active) {
#pragma unroll
        for (int k = 0; k < kMaxSlots; ++k) {
          if (k < myc) {
            const int c = c0 + k;
            uint32_t v[16];
            tmem_ld16(tmem_warp + c * 16, v);
            PhiloxOut o0{}, o1{};
            if (!last) {
              o0 = philox4x32_10_rk(2u * c, static_cast<uint32_t>(rg), static_cast<uint32_t>(t), q,
                                    L.round_keys);
              o1 = philox4x32_10_rk(2u * c + 1u, static_cast<uint32_t>(rg), static_cast<uint32_t>(t),
                                    q, L.round_keys);
            }
            tmem_wait_ld(v);
            const uint32_t rw[8] = {o0.x0, o0.x1, o0.x2, o0.x3, o1.x0, o1.x1, o1.x2, o1.x3};
            const uint32_t ob = (cur[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu;
            uint32_t nb = 0;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float hv = sH[c * 16 + e];
              const float I = __fadd_rn(__uint_as_float(v[e]), hv);
              if (dump != nullptr && c * 16 + e < n) dump[c * 16 + e] = I;
              const uint32_t s = (ob >> e) & 1u;
              if (fixed) {
                const int term = __float2int_rz(__fmul_rn(__fadd_rn(I, hv), fix_scale));
                ieacc += s ? term : -term;
                if (!last) {
                  const uint32_t word = rw[e >> 1];
                  const uint32_t key = (e & 1) ? (word >> 20) : ((word >> 4) & 0xFFFu);
                  nb |= fixed_decide(I, s, b, eta_q, __float_as_int(sZ[key]), fix_xi, fix_f, fix_half,
                                     P.fix_tau)
                        << e;
                }
                continue;
              }
              const float term = __fadd_rn(I, hv);
              eacc += s ? term : -term;
              if (!last) {
                const float x = __fmul_rn(b, I);
                const float tau = act == 0 ? tanhf(x) : staircase(x, levels);
                const float a = __fadd_rn(tau, s ? xi : -xi);
                const uint32_t word = rw[e >> 1];
                const uint32_t key = (e & 1) ? (word >> 20) : ((word >> 4) & 0xFFFu);
                const float delta = __fadd_rn(a, __fmul_rn(eta, sZ[key]));
                nb |= (delta >= 0.0f ? 1u : 0u) << e;
              }
            }
            const int valid = n - c * 16;
            if (valid < 16) nb &= (1u << valid) - 1u;
            nxt[k >> 1] |= nb << ((k & 1) * 16);
            if (!last) write_chunk(c, nb);
          }
        }
      }
      sPart[(t & 1) * 2 * kTileM + half * kTileM + row] = fixed ? __int_as_float(ieacc) : eacc;
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      aborted = sAbort[0] != 0;
      if (aborted) break;
      if (tid == 0 && !last) {
        tc_fence_after();
        issue_fields();
      }
      const float other = sPart[(t & 1) * 2 * kTileM + (half ^ 1) * kTileM + row];
      // the quadratic form is even in units of 2^-F: symmetric couplings, zero diagonal
      const double E = fixed ? -static_cast<double>((ieacc + __float_as_int(other)) / 2) / fix_scale
                             : static_cast<double>(-0.5f * (eacc + other));
      if (E < best_E) {
        best_E = E;
        best_t = t;
#pragma unroll
        for (int w = 0; w < kWordsPerThread; ++w) best[w] = cur[w];
      }
      if (has_target && first_hit < 0 && E <= target) first_hit = t;
      if (last) {
        if (row_valid) {
          uint16_t* cur_out = reinterpret_cast<uint16_t*>(P.cur_bits);
          uint16_t* best_out = reinterpret_cast<uint16_t*>(P.best_bits);
#pragma unroll
          for (int k = 0; k < kMaxSlots; ++k)
            if (k < myc) {
              const size_t o = static_cast<size_t>(rg) * P.words * 2 + (c0 + k);
              cur_out[o] = static_cast<uint16_t>(cur[k >> 1] >> ((k & 1) * 16));
              best_out[o] = static_cast<uint16_t>(best[k >> 1] >> ((k & 1) * 16));
            }
          if (half == 0) {
            P.best_E[rg] = best_E;
            P.best_t[rg] = best_t;
            P.first_hit[rg] = first_hit;
            P.final_E[rg] = E;
          }
        }
      } else {
#pragma unroll
        for (int w = 0; w < kWordsPerThread; ++w) cur[w] = nxt[w];
      }
    }
    if (aborted) break;
    if constexpr (SERVE) {
      // every thread's results are written: make them visible to the host, then the flag
      __threadfence_system();
      __syncthreads();
      if (tid == 0) st_release_sys(Q.done + (req % Q.nslots), static_cast<uint32_t>(req) + 1u);
    }
  }
  if (aborted && tid == 0) mbar_wait_bounded(bar_mma, phase, L.wait_ns);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NPAD);
}

template <int NPAD, bool SERVE>
cudaError_t launch_float_variant(const Launch& L, const ServeQueue& Q, int blocks, cudaStream_t st) {
  const int smem = sweep_float_smem_bytes(NPAD);
  cudaError_t e = cudaFuncSetAttribute(sweep_float_kernel<NPAD, SERVE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  sweep_float_kernel<NPAD, SERVE><<<blocks, kThreads, smem, st>>>(L, Q);
  return cudaGetLastError();
}

}  // namespace

int sweep_float_smem_bytes(int npad) {
  return 1024 + (npad <= 128 ? 2 : 1) * npad * 2 * npad + kTileM * 2 * npad + 4096 * 4 +
         npad * 4 + 2 * 2 * kTileM * 4 + 64 + static_cast<int>(sizeof(Problem));
}

cudaError_t launch_sweep_float(const Launch& L, int npad, int blocks, cudaStream_t st) {
  const ServeQueue none{};
  return npad <= 128 ? launch_float_variant<128, false>(L, none, blocks, st)
                     : launch_float_variant<256, false>(L, none, blocks, st);
}

cudaError_t launch_serve_float(const Launch& L, const ServeQueue& Q, int npad, int blocks,
                               cudaStream_t st) {
  return npad <= 128 ? launch_float_variant<128, true>(L, Q, blocks, st)
                     : launch_float_variant<256, true>(L, Q, blocks, st);
}

// J (BF16 bits, row-major n x n) -> BF16 operand image (rows npad, K = npad values, 2 bytes
// each, K-major with the 128-byte swizzle); zero outside n x n.  One thread per element.
// chunk_major: the 16 KB blocks (128 rows x one K-block) ordered [row block][K-block].
__global__ void stage_bf16_image_kernel(const uint16_t* __restrict__ J, int n, int npad,
                                        int chunk_major, uint8_t* __restrict__ img) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= static_cast<uint32_t>(npad) * npad) return;
  const int i = e / npad, j = e % npad;
  const uint16_t v = (i < n && j < n) ? J[static_cast<size_t>(i) * n + j] : 0;
  uint32_t off = sw128_offset(i, 2 * j, npad);  // K-block-major position
  if (chunk_major) {
    const uint32_t kblocks = static_cast<uint32_t>(npad) * 2u / 128u, block_bytes = npad * 128u;
    const uint32_t kb = off / block_bytes, rem = off % block_bytes;
    off = ((rem >> 14) * kblocks + kb) * 16384u + (rem & 16383u);
  }
  *reinterpret_cast<uint16_t*>(img + off) = v;
}

cudaError_t launch_stage_bf16_image(const uint16_t* d_J, int n, int npad, uint8_t* d_img,
                                    cudaStream_t st, bool chunk_major) {
  if (chunk_major && npad % 128 != 0) return cudaErrorInvalidValue;
  const uint32_t total = static_cast<uint32_t>(npad) * npad;
  stage_bf16_image_kernel<<<(total + 255) / 256, 256, 0, st>>>(d_J, n, npad, chunk_major ? 1 : 0, d_img);
  return cudaGetLastError();
}

}  // namespace pim
