// Mid-N PIMI sweep kernel (integer couplings, n <= 1024): persistent, one CTA per SM.
// Serves any integer instance with n <= 1024 (plain or diagonal-encoded FP8 image).  Each
// CTA takes (instance, 128-replica panel) units from a global counter, in the order the host
// sorted them (largest first), and runs every sweep of a unit before it takes the next, so
// instances of any size and replica count share one launch with no inter-CTA
// synchronisation.
//
// Per unit, per sweep t (Box 1, PIMI loop; Eq. 2 then Eq. 4):
//   spins    the panel's spins s(t) stay in tensor memory as the A operand of the field
//            GEMM (128 replicas = TMEM lanes, npad FP8 +-1 along the columns, four per
//            32-bit column), written by the epilogue threads that own the rows;
//   fields   the couplings stream from L2 through a 3-stage cp.async.bulk ring (four
//            K-blocks of 128 coupling rows per stage, one copy when the image is chunk-major)
//            in chunks of 128 output spins (all shared memory but the step table is ring);
//            chunk c accumulates D[r, i] = sum_j S[r, j] J[i, j] into one of two TMEM
//            buffers (tcgen05.mma kind::f8f6f4, A from TMEM), so the MMAs of chunk c+1 run
//            while the epilogue decides chunk c;
//   decision 16 epilogue warps (4 TMEM lane quadrants x 4 groups of 32 columns): each
//            thread owns one replica and 32 spins of every chunk, keeps their old / new
//            bits in registers, draws the Philox blocks and looks the threshold up in the
//            step's table at I = D + h; after the last chunk it writes the new spins into
//            the tensor-memory A image (all MMAs of the sweep have completed by then);
//   energy   E(s(t)) = -1/2 sum_i s_i (I_i + h_i), exact in int32, reduced over the four
//            column groups in shared memory; best state (written to the output array when
//            it improves) and first hit per replica.
#include <climits>

#include "kernels.h"
#include "philox.cuh"
#include "sm100_ptx.cuh"

namespace pim {
namespace {

constexpr int kNT = 128;                    // output spins per chunk (MMA N)
constexpr int kMaxNpad = 1024;
constexpr int kMaxChunks = kMaxNpad / kNT;
constexpr int kStages = 3;                  // coupling ring depth
constexpr int kBufs = 2;                    // TMEM accumulators of kNT columns
constexpr int kTabWords = 4096;             // threshold table of one step in shared memory
constexpr int kEpiWarps = 16;
constexpr int kGroups = kEpiWarps / 4;      // column groups per chunk
constexpr int kCols = kNT / kGroups;        // columns of a chunk per epilogue thread
constexpr int kWordsPT = kCols / 32;        // 32-bit spin words per thread and chunk
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = kEpiThreads + 64;  // + producer warp + MMA warp
constexpr int kTmemA = kBufs * kNT;         // first TMEM column of the spin image (npad / 4 columns)
constexpr int kTmemCols = kTmemA + kMaxNpad / 4;
constexpr int kBlockBytes = kNT * 128;      // one K-block of 128 coupling rows
// K-blocks per ring stage: a bulk copy costs about the same producer and copy-engine time
// whatever its size, so fewer, larger copies stream the couplings faster (measured: 4 x 3
// stages beat 2 x 6, 3 x 4 and 6 x 2 on the uneven batch).
constexpr int kKPS = 4;
constexpr int kStageBytes = kKPS * kBlockBytes;
constexpr int kBarCount = 2 * kStages + 2 * kBufs + 2;

// Bounded wait with the common case (phase already complete) inline; the out-of-line wait
// sleeps inside try_wait between checks.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  return mbar_try_wait(bar, parity) || mbar_wait_sleep(bar, parity, limit_ns);
}

// 32 spins -> their FP8 bytes in the thread's TMEM lane: K index col .. col + 31 = columns
// col / 4 .. col / 4 + 7 of the spin image (four K values per 32-bit column, lowest byte
// first).  Warp-collective.
__device__ __forceinline__ void put_spins32_tm(uint32_t tlane, int col, uint32_t bits, uint32_t neg) {
  const uint4 lo = fp8x16_from_bits(bits & 0xFFFFu, neg), hi = fp8x16_from_bits(bits >> 16, neg);
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
                   tlane + static_cast<uint32_t>(kTmemA + col / 4)),
               "r"(lo.x), "r"(lo.y), "r"(lo.z), "r"(lo.w), "r"(hi.x), "r"(hi.y), "r"(hi.z), "r"(hi.w)
               : "memory");
}

// D (+)= A B with A (128 x 32 FP8, K-major) in tensor memory at a_tmem.
__device__ __forceinline__ void mma_f8_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

constexpr float kMagic = 12582912.0f;      // 1.5 * 2^23: integer D in the low mantissa bits
constexpr uint32_t kMagicBits = 0x4B400000u;

// Bits of (a + 1.5 * 2^23) and (b + 1.5 * 2^23) for two exactly integral fields in one
// packed FP32 add (round to nearest: identical to two scalar adds, exact for |D| < 2^22).
__device__ __forceinline__ void magic_add2(uint32_t a, uint32_t b, uint32_t& va, uint32_t& vb) {
  uint64_t pr, rr;
  asm("mov.b64 %0, {%1, %2};" : "=l"(pr) : "r"(a), "r"(b));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rr) : "l"(pr), "l"(0x4B4000004B400000ull));
  asm("mov.b64 {%0, %1}, %2;" : "=r"(va), "=r"(vb) : "l"(rr));
}

// Sixteen spins of one replica, general-bias table without bias (h = 0, plain image):
// vb = bits(D + 1.5 * 2^23) = 0x4B400000 + I, the 16-bit threshold of (s, I) at shared
// address tab_c + 4 vb + 2 s (tab_c = table + 4 (imax - 0x4B400000), mod 2^32), and
// key >= M  <=>  d >= 16 M for the 16-bit draw d (key = d >> 4); the sign bits of d - 16 M
// (new spin -1) are shifted in by two chains.  sum_all / sum_up collect vb over all spins /
// the +1 spins for the energy.  Returns the new spins as bits 0..15.
template <bool DECIDE>
__device__ __forceinline__ uint32_t bias_chunk16(const uint32_t (&v)[16], const uint32_t (&rw)[8],
                                                 uint32_t cw16, uint32_t tab_c, uint32_t& sum_all,
                                                 uint32_t& sum_up) {
  uint32_t neg_hi = 0, neg_lo = 0, sa = 0, su = 0;
  uint32_t vpair = 0;
#pragma unroll
  for (int e = 15; e >= 0; --e) {
    uint32_t vb;
    if (e & 1)
      magic_add2(v[e - 1], v[e], vpair, vb);
    else
      vb = vpair;
    const uint32_t s = (cw16 >> e) & 1u;
    sa += vb;
    su += s * vb;
    if constexpr (DECIDE) {
      uint32_t m;
      asm volatile("ld.shared.u16 %0, [%1];" : "=r"(m) : "r"(tab_c + 4u * vb + 2u * s));
      const uint32_t w = rw[e >> 1];
      const uint32_t d = (e & 1) ? (w >> 16) : (w & 0xFFFFu);
      const uint32_t diff = d + m * 0xFFFFFFF0u;  // d - 16 m
      if (e >= 8)
        neg_hi = __funnelshift_l(diff, neg_hi, 1);
      else
        neg_lo = __funnelshift_l(diff, neg_lo, 1);
    }
  }
  sum_all += sa;
  sum_up += su;
  return ~((neg_hi << 8) | neg_lo) & 0xFFFFu;
}

// Sixteen spins of one replica, diagonal-encoded image (D = I + dk s, |I| < dk, h = 0): the
// 16-bit threshold of (s, I) is the table entry of D at shared address 2 vb + tab_d
// (vb = bits(D + 1.5 * 2^23), tab_d = table + 2 (2 dk) - 2 * 0x4B400000, mod 2^32), and
// |D| = s I + dk sums to the energy.  Returns the new spins as bits 0..15.
template <bool DECIDE>
__device__ __forceinline__ uint32_t diag_chunk16(const uint32_t (&v)[16], const uint32_t (&rw)[8],
                                                 uint32_t tab_d, float& esum) {
  uint32_t neg_hi = 0, neg_lo = 0;
  float e_a = 0.0f, e_b = 0.0f;
  uint32_t vpair = 0;
#pragma unroll
  for (int e = 15; e >= 0; --e) {
    const float fd = __uint_as_float(v[e]);
    if constexpr (DECIDE) {
      uint32_t vb;
      if (e & 1)
        magic_add2(v[e - 1], v[e], vpair, vb);
      else
        vb = vpair;
      uint32_t m;
      asm volatile("ld.shared.u16 %0, [%1];" : "=r"(m) : "r"(vb * 2u + tab_d));
      const uint32_t w = rw[e >> 1];
      const uint32_t d = (e & 1) ? (w >> 16) : (w & 0xFFFFu);
      const uint32_t diff = d + m * 0xFFFFFFF0u;  // d - 16 m
      if (e >= 8)
        neg_hi = __funnelshift_l(diff, neg_hi, 1);
      else
        neg_lo = __funnelshift_l(diff, neg_lo, 1);
    }
    if (e & 1)
      e_a += fabsf(fd);
    else
      e_b += fabsf(fd);
  }
  esum += e_a + e_b;
  return ~((neg_hi << 8) | neg_lo) & 0xFFFFu;
}

// A thread's 32 columns of one chunk (two 16-column halves): the TMEM load of each half runs
// while its two Philox blocks are drawn (DECIDE: every sweep but the final energy pass),
// then diag_chunk16 / bias_chunk16.  Returns the new spins of the 32 columns as bits.
template <bool DECIDE>
__device__ __forceinline__ uint32_t diag_chunk32(uint32_t ta, uint32_t blk0, uint32_t rg, uint32_t t,
                                                 uint32_t q, const uint32_t* rk, uint32_t tab_d,
                                                 float& esum) {
  uint32_t word = 0;
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    uint32_t v[16];
    tmem_ld16(ta + 16 * h2, v);
    PhiloxOut o0{}, o1{};
    if constexpr (DECIDE) {
      o0 = philox4x32_10_rk(blk0 + 2 * h2, rg, t, q, rk);
      o1 = philox4x32_10_rk(blk0 + 2 * h2 + 1, rg, t, q, rk);
    }
    tmem_wait_ld(v);
    const uint32_t rw8[8] = {o0.x0, o0.x1, o0.x2, o0.x3, o1.x0, o1.x1, o1.x2, o1.x3};
    word |= diag_chunk16<DECIDE>(v, rw8, tab_d, esum) << (16 * h2);
  }
  return word;
}

// As diag_chunk32 for the general table without bias (h = 0, plain image); cw32 holds the
// 32 current spins, eacc collects sum_i s_i I_i.
template <bool DECIDE>
__device__ __forceinline__ uint32_t bias_chunk32(uint32_t ta, uint32_t blk0, uint32_t rg, uint32_t t,
                                                 uint32_t q, const uint32_t* rk, uint32_t cw32,
                                                 uint32_t tab_c, int& eacc) {
  uint32_t word = 0;
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    uint32_t v[16];
    tmem_ld16(ta + 16 * h2, v);
    PhiloxOut o0{}, o1{};
    if constexpr (DECIDE) {
      o0 = philox4x32_10_rk(blk0 + 2 * h2, rg, t, q, rk);
      o1 = philox4x32_10_rk(blk0 + 2 * h2 + 1, rg, t, q, rk);
    }
    tmem_wait_ld(v);
    const uint32_t rw8[8] = {o0.x0, o0.x1, o0.x2, o0.x3, o1.x0, o1.x1, o1.x2, o1.x3};
    const uint32_t cw16 = (cw32 >> (16 * h2)) & 0xFFFFu;
    uint32_t sa = 0, su = 0;
    const uint32_t nb = bias_chunk16<DECIDE>(v, rw8, cw16, tab_c, sa, su);
    eacc += static_cast<int>(2u * (su - static_cast<uint32_t>(__popc(cw16)) * kMagicBits) -
                             (sa - 16u * kMagicBits));
    word |= nb << (16 * h2);
  }
  return word;
}

// DIAG = true: every unit has a diagonal-encoded image (P.dk > 0) and decides from its
// 16-bit table; DIAG = false: no unit has one (bias fast path or general path).  Two
// variants keep the register allocation of each to the paths it runs.
template <bool DIAG>
__global__ void __launch_bounds__(kThreads, 1) sweep_mid_kernel(const __grid_constant__ Launch L) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sRing = smem;
  uint32_t* sTab = reinterpret_cast<uint32_t*>(sRing + kStages * kStageBytes);
  int* sRed = reinterpret_cast<int*>(sTab + kTabWords);  // [kGroups][128 rows]
  int* sH = sRed + kGroups * 128;                         // [kMaxNpad]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sH + kMaxNpad);
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + kBarCount);
  volatile int* sUnit = reinterpret_cast<volatile int*>(sTmem + 1);
  volatile int* sAbort = sUnit + 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool epi = warp >= 2;
  const int quad = warp & 3;                    // TMEM lane quadrant of this warp
  const int grp = epi ? (warp - 2) >> 2 : 0;    // group of kCols columns inside a chunk
  const int row = quad * 32 + lane;             // replica row inside the panel
  const uint32_t full0 = smem_u32(&bars[0]);
  const uint32_t empty0 = smem_u32(&bars[kStages]);
  const uint32_t tfull0 = smem_u32(&bars[2 * kStages]);
  const uint32_t tempty0 = smem_u32(&bars[2 * kStages + kBufs]);
  const uint32_t aready = smem_u32(&bars[2 * kStages + 2 * kBufs]);
  const uint32_t drain = aready + 8;

  if (warp == 1) {
    tmem_alloc(smem_u32(sTmem), kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, kEpiWarps);
    }
    mbar_init(aready, 1);
    mbar_init(drain, 1);
    fence_mbar_init();
    *sAbort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t tlane = tmem + (static_cast<uint32_t>(quad * 32) << 16);  // this warp's TMEM lanes

  // Role counters, continued across units so every mbarrier phase is tracked exactly.
  uint32_t loads = 0, mmas = 0, cpass = 0, apass = 0;
  bool first_unit = true;
  const uint32_t idesc = idesc_e4m3(128, kNT);

  for (;;) {
    if (tid == 0) *sUnit = static_cast<int>(atomicAdd(L.next, 1u));
    __syncthreads();
    const int u = *sUnit;
    if (__syncthreads_or(*sAbort != 0) || u >= L.nwork) break;  // also orders the sUnit reads

    const WorkItem wk = L.work[u];
    const Problem& P = L.probs[wk.prob];
    const int n = P.n, npad = P.npad, R = P.R;
    const int nchunks = npad / kNT, kblocks = npad / 128;
    const int t_begin = L.t_begin, t_end = L.t_begin + L.sweeps;

    if (tid == 0) {
      // ---- producer: coupling K-blocks (chunk-major) into the ring ---------------------
      bool ok = true;
      for (int t = t_begin; t <= t_end && ok; ++t) {
        if (L.inject == 1 && first_unit && t == t_begin) continue;  // injected fault
        for (int c = 0; c < nchunks && ok; ++c)
          for (int kb0 = 0; kb0 < kblocks; kb0 += kKPS) {
            const int nk = kblocks - kb0 < kKPS ? kblocks - kb0 : kKPS;
            const uint32_t s = loads % kStages, use = loads / kStages;
            if ((use > 0 && !wait_phase(empty0 + 8 * s, (use - 1) & 1, L.wait_ns)) ||
                *sAbort != 0) {
              ok = false;
              break;
            }
            mbar_expect_tx(full0 + 8 * s, nk * kBlockBytes);
            if (npad > 256) {
              // images of n > 256 (npad >= 512) are chunk-major: the stage's K-blocks of chunk
              // c are contiguous, one copy
              bulk_g2s(smem_u32(sRing + s * kStageBytes),
                       P.jimg + (static_cast<size_t>(c) * kblocks + kb0) * kBlockBytes, nk * kBlockBytes,
                       full0 + 8 * s);
            } else {
              for (int j = 0; j < nk; ++j)
                bulk_g2s(smem_u32(sRing + s * kStageBytes + j * kBlockBytes),
                         P.jimg + static_cast<size_t>(kb0 + j) * npad * 128 + static_cast<size_t>(c) * kNT * 128,
                         kBlockBytes, full0 + 8 * s);
            }
            ++loads;
          }
      }
      if (!ok) {
        atomicOr(L.err, kDevErrTimeout);
        *sAbort = 1;
      }
    } else if (tid == 32) {
      // ---- MMA issuer: per sweep, wait for s(t) in the A image, then every chunk --------
      const uint32_t idesc_u = P.e5m2 ? idesc_e5m2(128, kNT) : idesc;
      bool ok = true;
      for (int t = t_begin; t <= t_end && ok; ++t) {
        if (!wait_phase(aready, apass & 1, L.wait_ns)) {
          ok = false;
          break;
        }
        ++apass;
        tc_fence_after();
        for (int c = 0; c < nchunks && ok; ++c) {
          const uint32_t b = cpass % kBufs, buse = cpass / kBufs;
          if (buse > 0 && !wait_phase(tempty0 + 8 * b, (buse - 1) & 1, L.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int kb0 = 0; kb0 < kblocks; kb0 += kKPS) {
            const int nk = kblocks - kb0 < kKPS ? kblocks - kb0 : kKPS;
            const uint32_t s = mmas % kStages, use = mmas / kStages;
            if (!wait_phase(full0 + 8 * s, use & 1, L.wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            for (int j = 0; j < nk; ++j) {
              const int kb = kb0 + j;
              const uint32_t b0 = smem_u32(sRing + s * kStageBytes + j * kBlockBytes);
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
                mma_f8_ta(tmem + b * kNT, tmem + kTmemA + kb * 32 + ks * 8, sw128_desc(b0 + ks * 32),
                          idesc_u, (kb > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(empty0 + 8 * s);
            ++mmas;
          }
          if (!ok) break;
          mma_commit(tfull0 + 8 * b);
          ++cpass;
        }
      }
      if (!ok) {
        atomicOr(L.err, kDevErrTimeout);
        *sAbort = 1;
      }
    } else if (epi) {
      // ---- epilogue ---------------------------------------------------------------------
      const int etid = tid - 64;
      const int rg = wk.rbase + row;
      const bool row_valid = rg < R;
      const bool warp_active = wk.rbase + quad * 32 < R;
      // Spins of this thread's 32-column word w of chunk c that exist (columns >= n stay -1).
      auto valid_mask = [&](int c, int w) -> uint32_t {
        const int valid = n - (c * kNT + grp * kCols + 32 * w);
        return valid >= 32 ? 0xFFFFFFFFu : (valid > 0 ? (1u << valid) - 1u : 0u);
      };
      // Bit rows of the caller's arrays as 32-bit words: word c*4 + grp*kWordsPT + w of row
      // rg holds this thread's spins 32w .. 32w+31 of chunk c.
      const int words = P.words;
      uint32_t* cur_io = P.cur_bits + static_cast<size_t>(rg) * words;
      uint32_t* best_io = P.best_bits + static_cast<size_t>(rg) * words;
      auto word_of = [&](int c, int w) { return c * (kNT / 32) + grp * kWordsPT + w; };
      const uint32_t neg8 = P.e5m2 ? 0xBCBCBCBCu : 0xB8B8B8B8u;  // -1 in the unit's FP8 format
      uint32_t cur[kMaxChunks][kWordsPT], nxt[kMaxChunks][kWordsPT];
      int best_E = INT_MAX, best_t = -1, first_hit = -1;
#pragma unroll
      for (int c = 0; c < kMaxChunks; ++c)
#pragma unroll
        for (int w = 0; w < kWordsPT; ++w) {
          cur[c][w] = nxt[c][w] = 0;
          if (c < nchunks && row_valid && word_of(c, w) < words)
            cur[c][w] = cur_io[word_of(c, w)] & valid_mask(c, w);
        }
      if (L.cont && row_valid) {
        best_E = static_cast<int>(P.best_E[rg]);
        best_t = P.best_t[rg];
        first_hit = P.first_hit[rg];
      }
      for (int k = etid; k < npad; k += kEpiThreads) sH[k] = (P.h != nullptr && k < n) ? P.h[k] : 0;
#pragma unroll
      for (int c = 0; c < kMaxChunks; ++c)
#pragma unroll
        for (int w = 0; w < kWordsPT; ++w)
          if (c < nchunks) {
            put_spins32_tm(tlane, c * kNT + grp * kCols + 32 * w, cur[c][w], neg8);
          }
      tmem_wait_st();
      tc_fence_before();
      bool stop = bar_sync_or(1, kEpiThreads, false);
      if (etid == 0) mbar_arrive(aready);

      // Problem fields in registers: the loops below store to global memory, which would
      // otherwise make the compiler reload them from the descriptor.
      const uint32_t q = P.q;
      const int dk = DIAG ? P.dk : 0;
      const int imax = P.imax, stride = dk > 0 ? 2 * dk : P.stride_words;  // words per step
      const uint32_t* thr = dk > 0 ? P.thr_diag : P.thr;
      const long long target = P.target;
      const bool tab_smem = stride <= kTabWords;
      const bool has_target = P.has_target != 0;
      const int dg = P.diag_img ? 256 : 0;  // diagonal-encoded image: D = I + 256 s
      const bool fast = !DIAG && P.h == nullptr && !P.diag_img && tab_smem;
      constexpr bool dfast = DIAG;  // diagonal-encoded table in shared memory (2 dk <= kTabWords)
      // byte address of the entry of D: 2 (bits of D + 1.5*2^23) + tab_d (mod 2^32)
      const uint32_t tab_d = smem_u32(sTab) + 4u * static_cast<uint32_t>(dk) - 2u * kMagicBits;
      const int e_off = dfast ? dk * n : 0;  // sum of |D| over the n spins = sum s I + n dk
      const uint32_t tab_c = smem_u32(sTab) + 4u * static_cast<uint32_t>(imax) - 4u * kMagicBits;  // mod 2^32
      for (int t = t_begin; t <= t_end && !stop; ++t) {
        const bool last = t == t_end;
        if (tab_smem && !last) {
          const uint4* src = reinterpret_cast<const uint4*>(thr + static_cast<size_t>(t) * stride);
          for (int k = etid; k < stride / 4; k += kEpiThreads)
            reinterpret_cast<uint4*>(sTab)[k] = __ldg(src + k);
        }
        if (bar_sync_or(1, kEpiThreads, *sAbort != 0)) break;
        const uint32_t* tab =
            tab_smem ? sTab : thr + static_cast<size_t>(last ? t_begin : t) * stride;
        int eacc = 0;
        bool waitfail = false;
#pragma unroll 1
        for (int c = 0; c < nchunks; ++c) {
          const uint32_t b = cpass % kBufs, buse = cpass / kBufs;
          ++cpass;
          if (!wait_phase(tfull0 + 8 * b, buse & 1, L.wait_ns)) waitfail = true;
          tc_fence_after();
          const uint32_t ta = tmem + (static_cast<uint32_t>(quad * 32) << 16) + b * kNT + grp * kCols;
          const uint32_t blk0 = static_cast<uint32_t>((c * kNT + grp * kCols) >> 3);
          if (dfast) {
            // Diagonal-encoded fields, 16 columns at a time (diag_chunk16).
            static_assert(kCols == 32 && kWordsPT == 1, "one 32-bit spin word per thread and chunk");
            // Columns at or past n (the padding of the last chunk) have zero fields and stay
            // -1: a thread whose 32 columns all lie there skips them (nxt stays 0).
            if (warp_active && c * kNT + grp * kCols < n) {
              float esum = 0.0f;
              const uint32_t word =
                  last ? diag_chunk32<false>(ta, blk0, static_cast<uint32_t>(rg), static_cast<uint32_t>(t), q,
                                             L.round_keys, tab_d, esum)
                       : diag_chunk32<true>(ta, blk0, static_cast<uint32_t>(rg), static_cast<uint32_t>(t), q,
                                            L.round_keys, tab_d, esum);
              nxt[c][0] = word & valid_mask(c, 0);
              eacc += static_cast<int>(esum);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * b);
            continue;
          }
          if (fast) {
            // 16 columns at a time: the TMEM load runs while their two Philox blocks are
            // drawn, then the decisions (bias_chunk16); the buffer is released at the end.
            if (warp_active && c * kNT + grp * kCols < n) {
              const uint32_t word =
                  last ? bias_chunk32<false>(ta, blk0, static_cast<uint32_t>(rg), static_cast<uint32_t>(t), q,
                                             L.round_keys, cur[c][0], tab_c, eacc)
                       : bias_chunk32<true>(ta, blk0, static_cast<uint32_t>(rg), static_cast<uint32_t>(t), q,
                                            L.round_keys, cur[c][0], tab_c, eacc);
              nxt[c][0] = word & valid_mask(c, 0);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * b);
            continue;
          }
          // General path (bias, diagonal-encoded image or a table in global memory), 16
          // columns at a time like the fast path.
          if (warp_active) {
#pragma unroll
            for (int h2 = 0; h2 < kCols / 16; ++h2) {
              uint32_t v[16];
              tmem_ld16(ta + 16 * h2, v);
              PhiloxOut o0{}, o1{};
              if (!last) {
                o0 = philox4x32_10_rk(blk0 + 2 * h2, static_cast<uint32_t>(rg),
                                      static_cast<uint32_t>(t), q, L.round_keys);
                o1 = philox4x32_10_rk(blk0 + 2 * h2 + 1, static_cast<uint32_t>(rg),
                                      static_cast<uint32_t>(t), q, L.round_keys);
              }
              tmem_wait_ld(v);
              const uint32_t rw8[8] = {o0.x0, o0.x1, o0.x2, o0.x3, o1.x0, o1.x1, o1.x2, o1.x3};
              const int w = h2 >> 1;
              const uint32_t cw16 = (cur[c][w] >> (16 * (h2 & 1))) & 0xFFFFu;
              uint32_t nb = 0;
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int col = c * kNT + grp * kCols + 16 * h2 + e;
                const uint32_t s = (cw16 >> e) & 1u;
                const int hv = sH[col];
                const int dgc = col < n ? (s ? dg : -dg) : 0;  // image diagonal inside n only
                // exact float -> int of the integer-valued field (|D| < 2^22)
                const int D = static_cast<int>(__float_as_uint(__fadd_rn(__uint_as_float(v[e]), kMagic)) -
                                               kMagicBits);
                const int I = D + hv - dgc;
                const int term = I + hv;
                eacc += s ? term : -term;
                if (!last) {
                  const uint32_t wd = tab[I + imax];
                  const uint32_t th = s ? (wd >> 16) : (wd & 0xFFFFu);
                  const uint32_t word = rw8[e >> 1];
                  const uint32_t key = (e & 1) ? (word >> 20) : ((word >> 4) & 0xFFFu);
                  nb |= (key >= th ? 1u : 0u) << e;
                }
              }
              if (h2 & 1)
                nxt[c][w] = (nxt[c][w] | (nb << 16)) & valid_mask(c, w);
              else
                nxt[c][w] = nb;
            }
          }
          // TMEM buffer b drained by this warp: let the MMA issuer reuse it.
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty0 + 8 * b);
        }
        if (!last && warp_active) {
          // Every MMA of sweep t has completed (the last chunk's commit was awaited): the A
          // image can take s(t+1).
#pragma unroll
          for (int c = 0; c < kMaxChunks; ++c)
#pragma unroll
            for (int w = 0; w < kWordsPT; ++w)
              if (c < nchunks) {
                put_spins32_tm(tlane, c * kNT + grp * kCols + 32 * w, nxt[c][w], neg8);
              }
          tmem_wait_st();
          tc_fence_before();
        }
        sRed[grp * 128 + row] = eacc;
        stop = bar_sync_or(1, kEpiThreads, waitfail || *sAbort != 0);
        if (stop) {
          if (etid == 0) {
            atomicOr(L.err, kDevErrTimeout);
            *sAbort = 1;
          }
          break;
        }
        if (!last && etid == 0) mbar_arrive(aready);
        int tot = 0;
#pragma unroll
        for (int g = 0; g < kGroups; ++g) tot += sRed[g * 128 + row];
        const int E = -((tot - e_off) / 2);
        if (E < best_E) {
          // the best state lives in the output array: written when it improves
          best_E = E;
          best_t = t;
          if (row_valid) {
#pragma unroll
            for (int c = 0; c < kMaxChunks; ++c)
#pragma unroll
              for (int w = 0; w < kWordsPT; ++w)
                if (c < nchunks && word_of(c, w) < words) best_io[word_of(c, w)] = cur[c][w];
          }
        }
        if (has_target && first_hit < 0 && static_cast<long long>(E) <= target) first_hit = t;
        if (last) {
          if (row_valid) {
#pragma unroll
            for (int c = 0; c < kMaxChunks; ++c)
#pragma unroll
              for (int w = 0; w < kWordsPT; ++w)
                if (c < nchunks && word_of(c, w) < words) cur_io[word_of(c, w)] = cur[c][w];
            if (grp == 0) {
              P.best_E[rg] = static_cast<double>(best_E);
              P.best_t[rg] = best_t;
              P.first_hit[rg] = first_hit;
              P.final_E[rg] = static_cast<double>(E);
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < kMaxChunks; ++c)
#pragma unroll
            for (int w = 0; w < kWordsPT; ++w) cur[c][w] = nxt[c][w];
        }
      }
    }
    first_unit = false;
  }

  // ---- teardown: no copy or MMA of this CTA may still be in flight ------------------------
  if (tid == 32) {
    mma_commit(drain);
    wait_phase(drain, 0, L.wait_ns);
  } else if (tid == 0) {
    for (uint32_t k = loads > kStages ? loads - kStages : 0; k < loads; ++k)
      wait_phase(full0 + 8 * (k % kStages), (k / kStages) & 1, L.wait_ns);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int sweep_mid_smem_bytes() {
  return 1024 + kStages * kStageBytes + kTabWords * 4 + kGroups * 128 * 4 + kMaxNpad * 4 +
         kBarCount * 8 + 32;
}

int sweep_mid_max_npad() { return kMaxNpad; }

int sweep_mid_max_blocks() {
  const int smem = sweep_mid_smem_bytes();
  if (cudaFuncSetAttribute(sweep_mid_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_mid_kernel<false>, kThreads, smem) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

cudaError_t launch_sweep_mid(const Launch& L, int blocks, cudaStream_t st, bool diag) {
  const int smem = sweep_mid_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(diag ? sweep_mid_kernel<true> : sweep_mid_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(L.next, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  if (diag)
    sweep_mid_kernel<true><<<blocks, kThreads, smem, st>>>(L);
  else
    sweep_mid_kernel<false><<<blocks, kThreads, smem, st>>>(L);
  return cudaGetLastError();
}

}  // namespace pim
