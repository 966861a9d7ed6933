// Fused PIMI sweep kernel for sm_103a: tcgen05 field GEMM into TMEM, fused decision,
// spin write-back and energy / best-state tracking, consecutive sweeps of a replica tile
// inside one CTA (all of them, or one chunk of them when persistent CTAs share the units
// through the launch's queue).
//
// Per sweep t (Box 1, PIMI loop; Eq. 2 then Eq. 4):
//   fields   D[r, i] = sum_j S[r, j] J[i, j]   (tcgen05.mma kind::f8f6f4, M = 128 replicas,
//            N = n spins rounded up to 16, K in steps of 32; FP8 E4M3 operands hold the
//            integer couplings and the +-1 spins exactly, FP32 accumulation is exact)
//   energy   H(s(t)) = -1/2 sum_i s_i (I_i + h_i) from the same fields (Eq. 1)
//   decision s_i(t+1) = +1 iff key(i, r, t) >= M_t[s_i(t)][I_i], the threshold form of the
//            float32 rule tau_t(I) + xi s + eta_t z(key) >= 0 (Eq. 4)
//   write    s(t+1) back into the shared-memory A operand, then the next sweep's MMA.
// The GEMM is transposed with respect to the paper's J s: TMEM lane = replica, column =
// spin, so that one thread owns one replica row of one column group and the energy of that
// replica is a thread-local sum plus the partial sums of the other column groups' threads.
#include <climits>

#include "kernels.h"
#include "philox.cuh"
#include "sm100_ptx.cuh"

namespace pim {
namespace {

constexpr int kGroups = 2;               // column groups of a replica row (2 or 3)
constexpr int kThreads = 128 * kGroups;  // 4 TMEM lane quadrants x kGroups column groups
constexpr int kTileM = 128;              // replicas per CTA (MMA M)

// The integer value I of an exactly integral float f (|f| < 2^22) appears in the low
// mantissa bits of f + 1.5 * 2^23.
constexpr float kMagic = 12582912.0f;
constexpr uint32_t kMagicBits = 0x4B400000u;
constexpr uint64_t kMagicPair = 0x4B4000004B400000ull;  // two FP32 1.5 * 2^23

// Two decision modes.
//  kModeDiag: h = 0 and |I| <= 255.  The couplings are staged with 256 on the diagonal, so
//    the MMA returns D = I + 256 s (sign(D) = s).  One 16-bit table entry per D gives the
//    key threshold for (s, I) at once, and |D| = s I + 256 gives the energy by an add.
//  kModeBias: general h; the table is indexed by I and holds both thresholds per word.
constexpr int kModeDiag = 0;
constexpr int kModeBias = 1;
constexpr int kDiagOffset = 256;
constexpr int kDiagEntries = 1024;  // D = -512 .. 511
constexpr int kMaxPrefetch = 1;     // 16-byte table pieces per thread: >= 256 x 16 B covers 4 KB

// First 16-column chunk of column group g (g = kGroups: the end), so that every group holds
// about n / kGroups spins.
__device__ __forceinline__ int group_begin(int g, int n, int nch) {
  return g == 0 ? 0 : g == kGroups ? nch : (g * n + 8 * kGroups) / (16 * kGroups);
}

// Most chunks one group holds, n <= NPAD (checked exhaustively for 2 and 3 groups).
template <int NPAD>
__host__ __device__ constexpr int max_group_chunks() {
  return (NPAD / 16 + kGroups - 1) / kGroups;
}
static_assert(kGroups == 2 || kGroups == 3, "column split checked for 2 and 3 groups only");

// One chunk of W = 16 or 8 consecutive spins of one replica in kModeDiag: load the fields
// D from tensor memory, draw the noise block(s), decide, and add |D| to the energy sum.
// Returns the new spins as bits (bit e = spin c*16+e is +1).
template <int W>
__device__ __forceinline__ uint32_t diag_chunk(uint32_t taddr, uint32_t c, uint32_t rg,
                                               uint32_t t, uint32_t q, const uint32_t* rk,
                                               uint32_t diag_bias, float& eacc) {
  uint32_t v[W];
  if constexpr (W == 16)
    tmem_ld16(taddr, v);
  else
    tmem_ld8(taddr, v);
  // The tensor-memory load runs while the noise block is generated.
  const PhiloxOut o0 = philox4x32_10_rk(2u * c, rg, t, q, rk);
  uint32_t rw[W / 2];
  rw[0] = o0.x0;
  rw[1] = o0.x1;
  rw[2] = o0.x2;
  rw[3] = o0.x3;
  if constexpr (W == 16) {
    const PhiloxOut o1 = philox4x32_10_rk(2u * c + 1u, rg, t, q, rk);
    rw[4] = o1.x0;
    rw[5] = o1.x1;
    rw[6] = o1.x2;
    rw[7] = o1.x3;
  }
  tmem_wait_ld(v);
  // Sign bits of (draw - 16 M) are shifted in from the top: after the last step bit e is set
  // iff key(e) < M, i.e. the new spin is -1.  Two shift chains and two energy sums keep the
  // dependent sequences short.
  uint32_t neg_hi = 0, neg_lo = 0;
  float e_a = 0.0f, e_b = 0.0f;
  // bits of D + 1.5 * 2^23 for two spins per instruction (packed FP32 add, round to nearest:
  // exact for these integers, identical to two scalar adds)
  uint32_t ibv[W];
#pragma unroll
  for (int e = 0; e < W; e += 2) {
    uint64_t pr, rr;
    asm("mov.b64 %0, {%1, %2};" : "=l"(pr) : "r"(v[e]), "r"(v[e + 1]));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rr) : "l"(pr), "l"(kMagicPair));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(ibv[e]), "=r"(ibv[e + 1]) : "l"(rr));
  }
#pragma unroll
  for (int e = W - 1; e >= 0; --e) {
    const float f = __uint_as_float(v[e]);
    const uint32_t ib = ibv[e];
    uint32_t m;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(m) : "r"(ib * 2u + diag_bias));
    const uint32_t w = rw[e >> 1];
    const uint32_t d = (e & 1) ? (w >> 16) : (w & 0xFFFFu);
    const uint32_t diff = d + m * 0xFFFFFFF0u;  // d - 16 m
    if (e >= W / 2)
      neg_hi = __funnelshift_l(diff, neg_hi, 1);
    else
      neg_lo = __funnelshift_l(diff, neg_lo, 1);
    if (e & 1)
      e_a += fabsf(f);
    else
      e_b += fabsf(f);
  }
  eacc += e_a + e_b;
  return ~((neg_hi << (W / 2)) | neg_lo) & ((1u << W) - 1u);
}

// QUEUE = false: CTA b runs work item b, all sweeps.  QUEUE = true: persistent CTAs take
// (chunk, item) segments from the launch's counter until none is left; a segment with
// chunk c > 0 starts from the state that chunk c-1 of its item (taken earlier from the
// counter, hence by a CTA already running) published.
template <int NPAD, int MODE, bool QUEUE>
__global__ void __launch_bounds__(kThreads, 2) sweep_tc_kernel(const Launch L) {
  constexpr int kMaxSlots = max_group_chunks<NPAD>();  // 16-column chunks per column group
  constexpr int kWordsPerThread = (kMaxSlots + 1) / 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int SW = MODE == kModeDiag ? kDiagEntries / 2 : L.stride_words_max;  // words per table
  uint8_t* sJ = smem;
  uint8_t* sA = sJ + NPAD * NPAD;
  uint32_t* sT = reinterpret_cast<uint32_t*>(sA + kTileM * NPAD);
  float* sPart = reinterpret_cast<float*>(sT + 2 * SW);
  int* sH = reinterpret_cast<int*>(sPart + 2 * kGroups * kTileM);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sH + (MODE == kModeBias ? NPAD : 0));
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + 2);
  int* sAbort = reinterpret_cast<int*>(sTmem + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, grp = warp >> 2;
  const int row = quad * 32 + lane;

  const uint32_t bar_mma = smem_u32(&bars[0]);
  const uint32_t bar_j = smem_u32(&bars[1]);

  // ---- per-CTA set-up: tensor memory and barriers, kept across the CTA's segments -----
  if (warp == 0) {
    tmem_alloc(smem_u32(sTmem), NPAD);
    tmem_relinquish();
  }
  if (tid == 32) {
    mbar_init(bar_mma, 1);
    mbar_init(bar_j, 1);
    fence_mbar_init();
    *sAbort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t tmem_warp = tmem + (static_cast<uint32_t>(quad * 32) << 16);
  uint32_t phase = 0, jphase = 0;
  bool aborted = false;
  const int nseg = QUEUE ? L.nwork * L.chunks : 1;

  for (int iter = 0; !aborted; ++iter) {
    // ---- segment: work item, chunk and sweep range ------------------------------------
    int seg = static_cast<int>(blockIdx.x);
    if (QUEUE) {
      if (tid == 0) sAbort[1] = static_cast<int>(atomicAdd(&L.ready[L.nwork], 1u));
      __syncthreads();
      seg = sAbort[1];
      if (seg >= nseg) break;
    } else if (iter > 0) {
      break;
    }
    const int item = QUEUE ? seg % L.nwork : seg;
    const int chunk = QUEUE ? seg / L.nwork : 0;
    const WorkItem wk = L.work[item];
    const Problem& P = L.probs[wk.prob];
    const int n = P.n;
    const int imax = P.imax;
    const int stride = MODE == kModeDiag ? kDiagEntries / 2 : P.stride_words;
    const uint32_t* thr = MODE == kModeDiag ? P.thr_diag : P.thr;
    const int R = P.R;
    const uint32_t q = P.q;
    const int rg = wk.rbase + row;
    const bool row_valid = rg < R;
    const bool warp_active = (wk.rbase + quad * 32) < R;
    // Column groups: contiguous ranges of 16-column chunks, about n / kGroups spins each.
    const int nch = (n + 15) >> 4;
    const int c0 = group_begin(grp, n, nch);
    const int myc = group_begin(grp + 1, n, nch) - c0;
    const int ksteps = (n + 31) >> 5;
    const int mma_n = (n + 15) & ~15;
    const int t_begin =
        QUEUE ? L.t_begin + static_cast<int>(static_cast<long long>(chunk) * L.sweeps / L.chunks) : L.t_begin;
    const int t_end = QUEUE ? L.t_begin + static_cast<int>(static_cast<long long>(chunk + 1) * L.sweeps /
                                                           L.chunks)
                            : L.t_begin + L.sweeps;
    const bool cont = L.cont != 0 || chunk > 0;

    // The item's previous chunk publishes its state first.
    if (QUEUE && chunk > 0) {
      if (tid == 0) {
        const uint64_t limit = L.wait_ns ? L.wait_ns : 2000000000ull;
        const uint64_t w0 = global_ns();
        while (ld_acquire_gpu(&L.ready[item]) < static_cast<uint32_t>(chunk)) {
          if (global_ns() - w0 > limit) {
            atomicOr(L.err, kDevErrTimeout);
            *sAbort = 1;
            break;
          }
          __nanosleep(128);
        }
      }
      __syncthreads();
      if (*sAbort != 0) {
        aborted = true;
        break;
      }
    }

    // ---- segment prologue: zeroed A operand, bias, first threshold table, J image -----
    for (int k = tid; k < kTileM * NPAD / 16; k += kThreads)
      reinterpret_cast<uint4*>(sA)[k] = make_uint4(0, 0, 0, 0);
    if (MODE == kModeBias)
      for (int k = tid; k < NPAD; k += kThreads) sH[k] = (P.h != nullptr && k < n) ? P.h[k] : 0;
    if (t_end > t_begin) {
      const uint4* src = reinterpret_cast<const uint4*>(thr + static_cast<size_t>(t_begin) * stride);
      uint4* dst = reinterpret_cast<uint4*>(sT + (t_begin & 1) * SW);
      for (int k = tid; k < stride / 4; k += kThreads) dst[k] = __ldg(src + k);
    }
    __syncthreads();  // the zeroed operand is complete before any row writes its spins
    if (tid == 0) {
      constexpr uint32_t kJBytes = NPAD * NPAD;
      mbar_expect_tx(bar_j, kJBytes);
      for (uint32_t off = 0; off < kJBytes; off += 16384)
        bulk_g2s(smem_u32(sJ + off), P.jimg + off, 16384u < kJBytes - off ? 16384u : kJBytes - off,
                 bar_j);
    }

    // ---- per-thread replica state: 16-bit spin chunks of this thread's column group ---
    // (L2 loads: a later chunk's state was written by another CTA of this launch)
    uint32_t cur[kWordsPerThread], best[kWordsPerThread];
    const uint16_t* cur_in = reinterpret_cast<const uint16_t*>(P.cur_bits);
#pragma unroll
    for (int w = 0; w < kWordsPerThread; ++w) cur[w] = 0;
    if (row_valid) {
#pragma unroll
      for (int k = 0; k < kMaxSlots; ++k)
        if (k < myc) {
          const uint32_t v = __ldcg(cur_in + static_cast<size_t>(rg) * P.words * 2 + (c0 + k));
          cur[k >> 1] |= v << ((k & 1) * 16);
        }
    }
    int best_E = INT_MAX, best_t = -1, first_hit = -1;
    const long long target = P.target;
    const bool has_target = P.has_target != 0;
    if (cont && row_valid) {
      best_E = static_cast<int>(__ldcg(P.best_E + rg));
      best_t = __ldcg(P.best_t + rg);
      first_hit = __ldcg(P.first_hit + rg);
      const uint16_t* best_in = reinterpret_cast<const uint16_t*>(P.best_bits);
#pragma unroll
      for (int w = 0; w < kWordsPerThread; ++w) best[w] = 0;
#pragma unroll
      for (int k = 0; k < kMaxSlots; ++k)
        if (k < myc) {
          const uint32_t v = __ldcg(best_in + static_cast<size_t>(rg) * P.words * 2 + (c0 + k));
          best[k >> 1] |= v << ((k & 1) * 16);
        }
    } else {
#pragma unroll
      for (int w = 0; w < kWordsPerThread; ++w) best[w] = cur[w];
    }

    // Write s(t_begin) into the A operand (row = replica, K = spin).
    if (warp_active) {
#pragma unroll
      for (int k = 0; k < kMaxSlots; ++k)
        if (k < myc) {
          const int c = c0 + k;
          const uint32_t nb = (cur[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu;
          *reinterpret_cast<uint4*>(sA + sw128_offset(row, c * 16, kTileM)) = fp8x16_from_bits(nb);
        }
    }
    fence_proxy_async_smem();
    __syncthreads();

    const uint32_t idesc = idesc_e4m3(kTileM, mma_n);
    const uint32_t sA_addr = smem_u32(sA), sJ_addr = smem_u32(sJ);
    auto issue_fields = [&]() {
      for (int ks = 0; ks < ksteps; ++ks) {
        const uint32_t kb = ks >> 2, ko = (ks & 3) * 32;
        mma_e4m3(tmem, sw128_desc(sA_addr + kb * (kTileM * 128) + ko),
                 sw128_desc(sJ_addr + kb * (NPAD * 128) + ko), idesc, ks > 0 ? 1u : 0u);
      }
      mma_commit(bar_mma);
    };

    if (tid == 0) {
      if (!mbar_wait_bounded(bar_j, jphase, L.wait_ns)) {
        atomicOr(L.err, kDevErrTimeout);
        *sAbort = 1;
      } else if (L.inject != 1) {  // injected fault: the first wait below cannot complete
        tc_fence_after();
        issue_fields();
      }
    }
    jphase ^= 1u;
    __syncthreads();
    aborted = *sAbort != 0;
    // kModeBias: word index of field I is (bits of I + 1.5*2^23) - (0x4B400000 - imax).
    const uint32_t ioff = kMagicBits - static_cast<uint32_t>(imax);

    // ---- sweep loop ----------------------------------------------------------------------
    for (int t = t_begin; t < t_end && !aborted; ++t) {
      if (!mbar_wait_bounded(bar_mma, phase, L.wait_ns)) {
        atomicOr(L.err, kDevErrTimeout);
        *sAbort = 1;
      }
      phase ^= 1;
      tc_fence_after();
      // Next step's thresholds: loaded into registers now, stored to the other table buffer
      // after this sweep's epilogue (so the load latency overlaps the epilogue).
      uint4 pre[kMaxPrefetch];
      const uint4* pre_src = reinterpret_cast<const uint4*>(thr + static_cast<size_t>(t + 1) * stride);
      const bool do_pre = t + 1 < t_end;
#pragma unroll
      for (int j = 0; j < kMaxPrefetch; ++j) {
        const int k = tid + j * kThreads;
        if (do_pre && k < stride / 4) pre[j] = __ldg(pre_src + k);
      }
      const uint32_t* tab = sT + (t & 1) * SW;
      // kModeDiag: byte address of entry D is 2 * (bits of D + 1.5*2^23) + this bias (mod 2^32).
      const uint32_t diag_bias = smem_u32(tab) + 2u * (kDiagEntries / 2) - 2u * kMagicBits;
      uint32_t nxt[kWordsPerThread];
#pragma unroll
      for (int w = 0; w < kWordsPerThread; ++w) nxt[w] = 0;
      float eacc = 0.0f;
      if (warp_active) {
#pragma unroll
        for (int k = 0; k < kMaxSlots; ++k) {
          if (k < myc) {
            const int c = c0 + k;
            const int valid = n - c * 16;
            uint32_t nb;
            if (MODE == kModeDiag) {
              if (valid > 8) {
                nb = diag_chunk<16>(tmem_warp + c * 16, c, rg, t, q, L.round_keys, diag_bias, eacc);
                if (valid < 16) nb &= (1u << valid) - 1u;
                *reinterpret_cast<uint4*>(sA + sw128_offset(row, c * 16, kTileM)) =
                    fp8x16_from_bits(nb);
              } else {  // last chunk with at most 8 spins: half the work
                nb = diag_chunk<8>(tmem_warp + c * 16, c, rg, t, q, L.round_keys, diag_bias, eacc);
                if (valid < 8) nb &= (1u << valid) - 1u;
                *reinterpret_cast<uint2*>(sA + sw128_offset(row, c * 16, kTileM)) =
                    make_uint2(fp8x4_from_bits(nb & 0xFu), fp8x4_from_bits((nb >> 4) & 0xFu));
              }
            } else {
              uint32_t v[16];
              tmem_ld16(tmem_warp + c * 16, v);
              const PhiloxOut o0 = philox4x32_10_rk(2u * c, static_cast<uint32_t>(rg),
                                                    static_cast<uint32_t>(t), q, L.round_keys);
              const PhiloxOut o1 = philox4x32_10_rk(2u * c + 1u, static_cast<uint32_t>(rg),
                                                    static_cast<uint32_t>(t), q, L.round_keys);
              tmem_wait_ld(v);
              const uint32_t rw[8] = {o0.x0, o0.x1, o0.x2, o0.x3, o1.x0, o1.x1, o1.x2, o1.x3};
              const uint32_t ob = (cur[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu;
              nb = 0;
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int hv = sH[c * 16 + e];
                const uint32_t ib = __float_as_uint(__fadd_rn(__uint_as_float(v[e]), kMagic)) + hv;
                const uint32_t w = tab[ib - ioff];
                const uint32_t s = (ob >> e) & 1u;
                const uint32_t th = s ? (w >> 16) : (w & 0xFFFFu);
                const uint32_t word = rw[e >> 1];
                const uint32_t key = (e & 1) ? (word >> 20) : ((word >> 4) & 0xFFFu);
                nb |= (key >= th ? 1u : 0u) << e;
                const int term = static_cast<int>(ib - kMagicBits) + hv;
                eacc += static_cast<float>(s ? term : -term);
              }
              if (valid < 16) nb &= (1u << valid) - 1u;
              *reinterpret_cast<uint4*>(sA + sw128_offset(row, c * 16, kTileM)) =
                  fp8x16_from_bits(nb);
            }
            nxt[k >> 1] |= nb << ((k & 1) * 16);
          }
        }
      }
      sPart[((t & 1) * kGroups + grp) * kTileM + row] = eacc;
      {
        uint4* pre_dst = reinterpret_cast<uint4*>(sT + ((t + 1) & 1) * SW);
#pragma unroll
        for (int j = 0; j < kMaxPrefetch; ++j) {
          const int k = tid + j * kThreads;
          if (do_pre && k < stride / 4) pre_dst[k] = pre[j];
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      aborted = *sAbort != 0;
      if (aborted) break;
      if (tid == 0) {
        tc_fence_after();
        issue_fields();  // fields of s(t+1)
      }
      float etot = 0.0f;
#pragma unroll
      for (int g = 0; g < kGroups; ++g) etot += sPart[((t & 1) * kGroups + g) * kTileM + row];
      const int E = MODE == kModeDiag
                        ? -((static_cast<int>(etot) - kDiagOffset * n) / 2)
                        : -(static_cast<int>(etot) / 2);
      if (E < best_E) {
        best_E = E;
        best_t = t;
#pragma unroll
        for (int w = 0; w < kWordsPerThread; ++w) best[w] = cur[w];
      }
      if (has_target && first_hit < 0 && E <= target) first_hit = t;
#pragma unroll
      for (int w = 0; w < kWordsPerThread; ++w) cur[w] = nxt[w];
    }
    if (aborted) break;

    // ---- energy of the state s(t_end) -------------------------------------------------
    if (!mbar_wait_bounded(bar_mma, phase, L.wait_ns)) {
      atomicOr(L.err, kDevErrTimeout);
      *sAbort = 1;
    }
    phase ^= 1u;
    tc_fence_after();
    float eacc = 0.0f;
    if (warp_active) {
#pragma unroll
      for (int k = 0; k < kMaxSlots; ++k) {
        if (k < myc) {
          const int c = c0 + k;
          uint32_t v[16];
          tmem_ld16(tmem_warp + c * 16, v);
          tmem_wait_ld(v);
          const uint32_t ob = (cur[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            if (MODE == kModeDiag) {
              eacc += fabsf(__uint_as_float(v[e]));
            } else {
              const int term = static_cast<int>(__float_as_uint(__fadd_rn(__uint_as_float(v[e]), kMagic)) -
                                                kMagicBits) + 2 * sH[c * 16 + e];
              eacc += static_cast<float>(((ob >> e) & 1u) ? term : -term);
            }
          }
        }
      }
    }
    sPart[((t_end & 1) * kGroups + grp) * kTileM + row] = eacc;
    tc_fence_before();
    __syncthreads();
    aborted = *sAbort != 0;
    float etot = 0.0f;
#pragma unroll
    for (int g = 0; g < kGroups; ++g) etot += sPart[((t_end & 1) * kGroups + g) * kTileM + row];
    const int E = MODE == kModeDiag
                      ? -((static_cast<int>(etot) - kDiagOffset * n) / 2)
                      : -(static_cast<int>(etot) / 2);
    if (E < best_E) {
      best_E = E;
      best_t = t_end;
#pragma unroll
      for (int w = 0; w < kWordsPerThread; ++w) best[w] = cur[w];
    }
    if (has_target && first_hit < 0 && E <= target) first_hit = t_end;
    if (row_valid && !aborted) {
      uint16_t* cur_out = reinterpret_cast<uint16_t*>(P.cur_bits);
      uint16_t* best_out = reinterpret_cast<uint16_t*>(P.best_bits);
#pragma unroll
      for (int k = 0; k < kMaxSlots; ++k)
        if (k < myc) {
          const size_t o = static_cast<size_t>(rg) * P.words * 2 + (c0 + k);
          cur_out[o] = static_cast<uint16_t>(cur[k >> 1] >> ((k & 1) * 16));
          best_out[o] = static_cast<uint16_t>(best[k >> 1] >> ((k & 1) * 16));
        }
      if (grp == 0) {
        P.best_E[rg] = static_cast<double>(best_E);
        P.best_t[rg] = best_t;
        P.first_hit[rg] = first_hit;
        P.final_E[rg] = static_cast<double>(E);
      }
    }
    // Publish the state to the item's next chunk; the barrier also keeps every thread's
    // reads of this segment's shared memory ahead of the next segment's writes.
    __syncthreads();
    if (QUEUE && !aborted && tid == 0 && chunk + 1 < L.chunks) {
      __threadfence();
      st_release_gpu(&L.ready[item], static_cast<uint32_t>(chunk + 1));
    }
  }

  if (aborted && tid == 0) {
    // A wait gave up: give an in-flight MMA and J copy a bounded chance to land before the
    // tensor and shared memory are released.
    mbar_wait_bounded(bar_mma, phase, L.wait_ns);
    mbar_wait_bounded(bar_j, jphase ^ 1u, L.wait_ns);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NPAD);
}

// Without a queue (L.chunks == 0): one CTA per work item.  With one: `blocks` persistent
// CTAs, the counter and ready flags zeroed first.  The queue needs no co-residency: a CTA
// only waits for a chunk that an already running CTA took from the counter before it.
template <int NPAD, int MODE, bool QUEUE>
cudaError_t launch_one(const Launch& L, int blocks, cudaStream_t st) {
  const int smem = sweep_tc_smem_bytes(NPAD, MODE == kModeDiag ? kDiagEntries / 2 : L.stride_words_max) +
                   (MODE == kModeBias ? NPAD * 4 : 0);
  cudaError_t e = cudaFuncSetAttribute(sweep_tc_kernel<NPAD, MODE, QUEUE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (QUEUE) {
    e = cudaMemsetAsync(L.ready, 0, (static_cast<size_t>(L.nwork) + 1) * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
  }
  sweep_tc_kernel<NPAD, MODE, QUEUE><<<blocks, kThreads, smem, st>>>(L);
  return cudaGetLastError();
}

template <int NPAD, int MODE>
cudaError_t launch_variant(const Launch& L, int blocks, cudaStream_t st) {
  return L.chunks > 0 ? launch_one<NPAD, MODE, true>(L, blocks, st)
                      : launch_one<NPAD, MODE, false>(L, blocks, st);
}

}  // namespace

int sweep_tc_smem_bytes(int npad, int stride_words_max) {
  return 1024 /* alignment slack */ + npad * npad + kTileM * npad + 2 * stride_words_max * 4 +
         2 * kGroups * kTileM * 4 + 64;
}

cudaError_t launch_sweep_tc(const Launch& L, int npad_max, int blocks, cudaStream_t st,
                            bool diag) {
  if (npad_max <= 128)
    return diag ? launch_variant<128, kModeDiag>(L, blocks, st) : launch_variant<128, kModeBias>(L, blocks, st);
  return diag ? launch_variant<256, kModeDiag>(L, blocks, st) : launch_variant<256, kModeBias>(L, blocks, st);
}

}  // namespace pim
