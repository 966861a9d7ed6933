// Large-N PIMI sweep kernel (N > 256): persistent, cooperative, one CTA per (128-replica
// tile, NT-spin column block), all sweeps in one launch.  Three operand variants:
//   FP8   integer couplings: FP8 E4M3 spin and coupling images (tcgen05 kind::f8f6f4), both
//         streamed every sweep; exact integer fields and the exact threshold-table decision;
//   BF16  real couplings: BF16 images (kind::f16), FP32 fields, Eq. 4 evaluated in FP32;
//   FP4   integer couplings in {0, +-1, +-2, +-3, +-4, +-6}, NT = 64: the CTA's coupling rows
//         stay in shared memory as packed E2M1 for the whole launch and only the E2M1 spin
//         tile streams (block-scaled kind::mxf4 with unit scale factors, so the products and
//         the FP32 sums stay exact integers); same decision as FP8.
// NT (64 or 128 spins) and the variant are chosen per instance by the host.
//
// Per sweep t (Box 1, PIMI loop; Eq. 2 then Eq. 4):
//   fields   D[r, i] = sum_j S[r, j] J[i, j] for the CTA's 128 replicas and NT spins: the
//            K dimension (all N spins) streams through a shared-memory ring filled by
//            cp.async.bulk (spins of the tile from the global spin image, two K-blocks per
//            copy, rows of J from the coupling image unless they are resident), consumed by
//            tcgen05.mma into TMEM.
//   decision 16 epilogue warps (4 TMEM lane quadrants x 4 column groups); each thread owns
//            one replica and NT/4 spins for the whole anneal, keeps their old / new / best
//            bits in registers, draws the Philox blocks and decides: integer couplings by
//            the step's threshold table at field I = D + h (staged into shared memory while
//            the MMAs run, or read through L1 when it does not fit), real couplings by
//            tanh(b_t I) + xi s + eta_t z >= 0.  It writes the new spins into the other spin
//            image and adds its share of sum_i s_i (I_i + h_i) to the replica's energy
//            accumulator (global atomics, three rotating buffers; int32 for integer
//            couplings, so the energy stays exact).
//   exchange a bounded grid barrier (one arrival atomic on a monotone counter); during the
//            next sweep's K-loop every CTA reads the replica energies of s(t), updates best /
//            first hit (redundantly, identically in all CTAs) and keeps its own spins of s(t)
//            as the best state when the energy improved.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <type_traits>

#include "kernels.h"
#include "philox.cuh"
#include "sm100_ptx.cuh"

namespace pim {
namespace {


constexpr int kTabWords = 8192;     // threshold table of one step staged in shared memory
constexpr int kEpiWarps = 16;
constexpr int kThreads = (2 + kEpiWarps) * 32;
constexpr int kSmemBudget = 227 * 1024;

// K-blocks per ring stage.  A bulk copy costs about 0.16 us of the producer's time whatever
// its size (up to 16 KB measured), so a stage moves two K-blocks of the tile's spins in one
// copy (the spin image is tile-major for that) instead of one copy per K-block.
constexpr int KPS = 2;
// Odd sweeps walk the K-blocks from the last to the first, so a sweep starts on the coupling
// blocks the previous one read last, which are still in L2 (BF16 Max-Cut N = 8192, whose
// 134 MB image just exceeds L2: DRAM reads 136 -> 75 MB per sweep, 43.9 -> 41.7 us).  The
// order depends on the absolute sweep index, so split runs and resumes sum in the same order.
constexpr bool kRev = true;
constexpr int kMaxStagesFp4 = 4;  // ring depth cap of the coupling-resident variant

// Shared-memory plan of one kernel variant: NT output spins per CTA, operand variant OP.
// The streamed variants fix the ring at compile time; the coupling-resident one sizes it at
// run time around its resident coupling block (sweep_big_smem).
template <int NT, int OP>
struct BigCfg {
  static constexpr bool kReal = OP == kBigBf16, kFp4 = OP == kBigFp4;
  static constexpr int kSpinsPerKB = kFp4 ? 256 : (kReal ? 64 : 128);  // per 128-byte row
  static constexpr int kSPT = NT / 4;            // spins per epilogue thread
  static constexpr int kChunks = kSPT / 16;      // 16-spin chunks per thread
  static constexpr int kABytes = 128 * 128;      // one K-block of the spin tile (128 rows x 128 B)
  static constexpr int kBBytes = kFp4 ? 0 : NT * 128;  // streamed coupling rows per K-block
  // K-blocks per ring stage: the coupling-resident variant streams only spins and copies
  // three K-blocks (48 KB) at a time (SK N = 4096, two stages: 8.84 -> 8.45 us per sweep
  // against two K-blocks through three stages; N = 2048: -2 %; N = 1024, 3072: equal).
  static constexpr int kKPS = kFp4 ? 3 : KPS;
  static constexpr int kAux = kReal ? 4096 * 4 : kTabWords * 4;  // noise levels | step table
  static constexpr int kMisc = 4 * 128 * 4 + NT * 4 + 256;      // sRed, sH, barriers, flags
  static constexpr int kFixed = 1024 + kAux + kMisc;
  static constexpr int kFit = (kSmemBudget - kFixed) / (kKPS * (kABytes + kBBytes));
  static constexpr int kStages = kFp4 ? kMaxStagesFp4 : (kFit < 8 ? kFit : 8);  // ring depth (max)
  static constexpr int kSmem = kFixed + kStages * kKPS * (kABytes + kBBytes);
  static constexpr int kTmemCols = kFp4 ? 2 * NT : NT;  // accumulator (+ unit scale factors)
  static_assert(kFp4 || kFit >= 2, "ring too shallow");
  static_assert(!kFp4 || NT == 64, "the coupling-resident variant has 64-spin column blocks");
};

// Shared-memory plan of the coupling-resident variant for npad spins: [pad][ring][resident
// couplings NT x npad / 2][table?][misc].  The 1024-byte alignment pad is reserved only when
// it costs no ring stage; otherwise the kernel checks the base alignment itself.
BigSmem fp4_plan(int npad, int stride_words) {
  using C = BigCfg<64, kBigFp4>;
  BigSmem out;
  if (npad % 256 != 0 || npad > 4096) return out;
  const int stage = C::kKPS * C::kABytes;
  const int jres = 64 * npad / 2;
  const int avail = kSmemBudget - jres - C::kMisc;
  auto fit = [&](int extra) { return (avail - extra) / stage; };
  const int base = std::min(kMaxStagesFp4, fit(0));
  const int pad = std::min(kMaxStagesFp4, fit(1024)) == base ? 1024 : 0;
  // the step table goes to shared memory when the ring keeps at least 96 KB in flight beside it
  const bool tab = stride_words <= kTabWords &&
                   std::min(kMaxStagesFp4, fit(pad + kTabWords * 4)) * stage >= 3 * 32768;
  out.stages = std::min(kMaxStagesFp4, fit(pad + (tab ? kTabWords * 4 : 0)));
  out.tab_smem = tab ? 1 : 0;
  out.bytes = pad + out.stages * stage + jres + (tab ? kTabWords * 4 : 0) + C::kMisc;
  out.ok = out.stages >= 2 && out.bytes <= kSmemBudget;
  return out;
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Grid-wide barrier with a time bound over a monotone 64-bit arrival counter (bar[0..1],
// zeroed before the launch): a CTA's k-th barrier completes once the counter reaches
// k * nblocks, so no reset or generation word is needed and an arrival is one acq_rel
// atomic.  Aborting sets a high bit of the counter, which releases every present and later
// wait at once; all of them then return false (on all threads of the CTA).
constexpr unsigned long long kBarAbort = 1ull << 62;

__device__ __forceinline__ void grid_abort(unsigned int* bar) {
  atomicOr(reinterpret_cast<unsigned long long*>(bar), kBarAbort);
}

__device__ bool grid_barrier(unsigned int* bar, unsigned long long target, int* err, int* sflag,
                             uint64_t limit_ns) {
  const uint64_t limit = limit_ns ? limit_ns : 2000000000ull;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(bar);
    unsigned long long v;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], 1;" : "=l"(v) : "l"(cnt) : "memory");
    v += 1;
    if (v < target) {
      const uint64_t t0 = global_ns();
      uint32_t polls = 0;
      do {
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(cnt) : "memory");
        if ((++polls & 31) == 0 && v < target && global_ns() - t0 > limit) {
          atomicOr(err, kDevErrTimeout);
          grid_abort(bar);
          v |= kBarAbort;
        }
      } while (v < target);
    }
    *sflag = (v & kBarAbort) ? 0 : 1;
  }
  __syncthreads();
  return *sflag != 0;
}

template <int NT, int OP>
__global__ void __launch_bounds__(kThreads, 1) sweep_big_kernel(const __grid_constant__ BigLaunch L) {
  using C = BigCfg<NT, OP>;
  constexpr bool REAL = C::kReal, FP4 = C::kFp4;
  using EAcc = std::conditional_t<REAL, float, int>;  // energy partial sums
  constexpr int kABytes = C::kABytes, kBBytes = C::kBBytes;
  constexpr int kSPT = C::kSPT, kChunks = C::kChunks;
  constexpr int kKPS = C::kKPS;
  constexpr int kMaxStages = C::kStages;
  const int kStages = FP4 ? L.stages : C::kStages;  // ring depth of this launch
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;                               // kStages x kKPS x kABytes
  uint8_t* sB = sA + kStages * kKPS * kABytes;      // kStages x kKPS x kBBytes (streamed)
  uint8_t* sJ = sB + kStages * kKPS * kBBytes;      // resident couplings (FP4): NT x npad / 2
  const int jres_bytes = FP4 ? NT * L.P.npad / 2 : 0;
  const bool tab_smem = L.tab_smem != 0;
  uint32_t* sTab = reinterpret_cast<uint32_t*>(sJ + jres_bytes);  // [kTabWords]
  float* sZ = reinterpret_cast<float*>(sTab);       // [4096] noise levels (real)
  const int aux_bytes = REAL ? C::kAux : (FP4 && !tab_smem ? 0 : C::kAux);
  EAcc* sRed = reinterpret_cast<EAcc*>(sJ + jres_bytes + aux_bytes);  // [4][128 rows]
  uint32_t* sH = reinterpret_cast<uint32_t*>(sRed + 4 * 128);  // [NT] bias: int32 or float bits
  uint64_t* bars = reinterpret_cast<uint64_t*>(sH + NT);       // full[S], empty[S], done, jres
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + 2 * kMaxStages + 2);
  int* sFlag = reinterpret_cast<int*>(sTmem + 1);
  if constexpr (FP4) {
    // The plan may leave no room for the alignment pad: check that the layout fits what the
    // launch provided (uniform over the grid, so every CTA returns before any barrier).
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint32_t end = static_cast<uint32_t>(reinterpret_cast<uint8_t*>(sFlag + 1) - smem_raw);
    if (end > dyn) {
      if (threadIdx.x == 0) atomicOr(L.err, kDevErrLayout);
      return;
    }
  }

  const Problem& P = L.P;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncb = L.ncb;
  const int cb = blockIdx.x % ncb, rt = blockIdx.x / ncb;
  const unsigned int nblocks = gridDim.x;
  const int n = P.n, npad = P.npad, R = P.R, rpad = L.rpad;
  const int kblocks = npad / C::kSpinsPerKB;
  const int t_begin = L.t_begin, t_end = L.t_begin + L.sweeps;
  const bool epi = warp >= 2;
  const int ew = warp - 2;             // epilogue warp 0..15
  const int quad = warp & 3;           // TMEM lane quadrant of this warp
  const int grp = epi ? ew >> 2 : 0;   // column group 0..3 (kSPT spins each)
  const int row = quad * 32 + lane;    // replica row inside the tile
  const int rl = rt * 128 + row;       // replica row inside this launch's images
  const int r = L.rbase + rl;          // replica index
  const int col0 = cb * NT + grp * kSPT;  // first spin of this thread's kSPT
  const bool row_valid = epi && r < R;
  const bool warp_active = epi && (L.rbase + rt * 128 + quad * 32) < R && col0 < n;
  const int valid = n - col0;            // spins of the kSPT that exist
  const uint32_t full_mask = kSPT == 32 ? 0xFFFFFFFFu : ((1u << (kSPT & 31)) - 1u);
  const uint32_t vmask = valid >= kSPT ? full_mask : (valid > 0 ? (1u << valid) - 1u : 0u);

  const uint32_t bar_full0 = smem_u32(&bars[0]);
  const uint32_t bar_empty0 = smem_u32(&bars[kMaxStages]);
  const uint32_t bar_done = smem_u32(&bars[2 * kMaxStages]);
  const uint32_t bar_jres = smem_u32(&bars[2 * kMaxStages + 1]);

  if (warp == 1) {
    tmem_alloc(smem_u32(sTmem), C::kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar_full0 + 8 * s, 1);
      mbar_init(bar_empty0 + 8 * s, 1);
    }
    mbar_init(bar_done, 1);
    mbar_init(bar_jres, 1);
    fence_mbar_init();
  }
  for (int k = tid; k < NT; k += kThreads) {
    const int i = cb * NT + k;
    if constexpr (REAL)
      sH[k] = __float_as_uint((P.hf != nullptr && i < n) ? P.hf[i] : 0.0f);
    else
      sH[k] = static_cast<uint32_t>((P.h != nullptr && i < n) ? P.h[i] : 0);
  }
  if constexpr (REAL)
    for (int k = tid; k < 4096; k += kThreads) sZ[k] = P.zlev[k];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  if constexpr (FP4) {
    // Resident couplings: the CTA's column block (NT rows x all K-blocks, contiguous in the
    // E2M1 image) arrives once, in copies of up to 32 KB on one barrier.
    if (tid == 0) {
      const uint8_t* src = L.j4 + static_cast<size_t>(cb) * jres_bytes;
      mbar_expect_tx(bar_jres, jres_bytes);
      for (int o = 0; o < jres_bytes; o += 32768)
        bulk_g2s(smem_u32(sJ + o), src + o, jres_bytes - o < 32768 ? jres_bytes - o : 32768, bar_jres);
    }
    // Unit scale factors (UE8M0 127 = 2^0) in every TMEM column after the accumulator, so
    // whatever layout the block-scaled MMA reads them in, each scale is 1.
    if (epi && grp == 0) {
#pragma unroll
      for (int c = 0; c < NT; c += 32)
        tmem_fill32(tmem + (static_cast<uint32_t>(quad * 32) << 16) + NT + c, 0x7F7F7F7Fu);
      tmem_wait_st();
    }
    tc_fence_before();
  }

  // ---- per-thread state: this replica's kSPT spins ------------------------------------
  uint32_t cur = 0, best = 0;
  EAcc best_E;
  if constexpr (REAL)
    best_E = FLT_MAX;
  else
    best_E = INT_MAX;
  int best_t = -1, first_hit = -1;
  const int half_words = P.words * 2;  // 16-bit chunks per row in the caller's bit arrays
  const int chunk = col0 >> 4;
  const uint16_t* cur_in = reinterpret_cast<const uint16_t*>(P.cur_bits);
  const uint16_t* best_in = reinterpret_cast<const uint16_t*>(P.best_bits);
  if (row_valid) {
#pragma unroll
    for (int c = 0; c < kChunks; ++c)
      if (chunk + c < half_words) {
        const size_t o = static_cast<size_t>(r) * half_words + chunk + c;
        cur |= static_cast<uint32_t>(cur_in[o]) << (16 * c);
        if (L.cont) best |= static_cast<uint32_t>(best_in[o]) << (16 * c);
      }
    if (L.cont) {
      best_E = static_cast<EAcc>(P.best_E[r]);
      best_t = P.best_t[r];
      first_hit = P.first_hit[r];
    }
  }
  if (!L.cont) best = cur;
  const bool has_target = P.has_target != 0;

  // Spin image s(t) for this CTA's block (rows of the tile, its NT spins): FP8, BF16 or E2M1
  // +-1.  The image is tile-major, [replica tile][K-block][128 rows x 128 B with the 128-byte
  // swizzle], so consecutive K-blocks of one tile are contiguous (one copy per ring stage).
  const size_t tile_bytes = static_cast<size_t>(kblocks) * kABytes;
  auto write_image = [&](uint8_t* img, uint32_t bits) {
    if (!epi || col0 >= npad) return;
    uint8_t* base = img + static_cast<size_t>(rt) * tile_bytes;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const uint32_t b16 = (bits >> (16 * c)) & 0xFFFFu;
      const int k = col0 + 16 * c;
      if constexpr (REAL) {
        *reinterpret_cast<uint4*>(base + sw128_offset(row, 2 * k, 128)) = bf16x8_from_bits(b16 & 0xFFu);
        *reinterpret_cast<uint4*>(base + sw128_offset(row, 2 * k + 16, 128)) = bf16x8_from_bits(b16 >> 8);
      } else if constexpr (FP4) {
        // 16 spins = 8 bytes at byte k / 2 of the row (k is a multiple of 16).
        *reinterpret_cast<uint2*>(base + sw128_offset(row, k >> 1, 128)) =
            make_uint2(e2m1x8_from_bits(b16 & 0xFFu), e2m1x8_from_bits(b16 >> 8));
      } else {
        *reinterpret_cast<uint4*>(base + sw128_offset(row, k, 128)) = fp8x16_from_bits(b16);
      }
    }
  };
  unsigned long long bar_target = nblocks;  // counter value that completes the next barrier
  write_image(L.s_img[0], cur & vmask);
  fence_proxy_async_global();
  if (!grid_barrier(L.bar, bar_target, L.err, sFlag, L.wait_ns)) goto teardown;

  {
    uint32_t loads = 0, mmas = 0, done_phase = 0;
    const uint32_t idesc = REAL ? idesc_bf16(128, NT) : (FP4 ? idesc_mxf4(128, NT) : idesc_e4m3(128, NT));
    bool jres_ready = !FP4;
    // Producer (thread 0): stream the K blocks of image `img` (spins of the tile) and, unless
    // they are resident, of the coupling rows of the column block into the ring.  A stage
    // is refilled once the MMAs that read it have completed (its empty barrier).
    // A stage holds kKPS consecutive K-blocks: the tile's spins of all of them in one copy
    // (the image is tile-major), streamed coupling rows in one copy per K-block.
    auto produce = [&](const uint8_t* img, bool rev) -> bool {
      const uint8_t* a_src = img + static_cast<size_t>(rt) * tile_bytes;
      // Coupling images of n > 256 are chunk-major: 16 KB blocks of 128 rows x one K-block,
      // ordered [row block][K-block], so the stage's K-blocks of a 128-row column block are
      // one copy; a 64-row column block is half of each 16 KB block (one copy per K-block).
      const uint8_t* b_src = P.jimg + static_cast<size_t>(NT == 128 ? cb : cb >> 1) * kblocks * 16384 +
                             (NT == 128 ? 0 : (cb & 1) * 8192);
      const int nst = (kblocks + kKPS - 1) / kKPS;
      for (int si = 0; si < nst; ++si) {
        const int kb0 = (rev ? nst - 1 - si : si) * kKPS;
        const int nk = kblocks - kb0 < kKPS ? kblocks - kb0 : kKPS;
        const uint32_t s = loads % kStages, use = loads / kStages;
        if (use > 0 && !mbar_wait_fast(bar_empty0 + 8 * s, (use - 1) & 1, L.wait_ns)) return false;
        mbar_expect_tx(bar_full0 + 8 * s, nk * (kABytes + kBBytes));
        bulk_g2s(smem_u32(sA + s * kKPS * kABytes), a_src + static_cast<size_t>(kb0) * kABytes,
                 nk * kABytes, bar_full0 + 8 * s);
        if constexpr (kBBytes > 0) {
          if constexpr (NT == 128) {
            bulk_g2s(smem_u32(sB + s * kKPS * kBBytes), b_src + static_cast<size_t>(kb0) * 16384,
                     nk * kBBytes, bar_full0 + 8 * s);
          } else {
            for (int j = 0; j < nk; ++j)
              bulk_g2s(smem_u32(sB + (s * kKPS + j) * kBBytes), b_src + static_cast<size_t>(kb0 + j) * 16384,
                       kBBytes, bar_full0 + 8 * s);
          }
        }
        ++loads;
      }
      return true;
    };
    // MMA issuer (thread 32): D = S_tile x J_block^T, K block by K block as stages land; it
    // never waits for an MMA to finish, only for data.  Each MMA consumes 32 bytes of K
    // (32 FP8, 16 BF16 or 64 E2M1 values).
    auto multiply = [&](bool rev) -> bool {
      if (!jres_ready) {
        if (!mbar_wait_fast(bar_jres, 0, L.wait_ns)) return false;
        jres_ready = true;
      }
      const int nst = (kblocks + kKPS - 1) / kKPS;
      for (int si = 0; si < nst; ++si) {
        const int kb0 = (rev ? nst - 1 - si : si) * kKPS;
        const int nk = kblocks - kb0 < kKPS ? kblocks - kb0 : kKPS;
        const uint32_t s = mmas % kStages, use = mmas / kStages;
        if (!mbar_wait_fast(bar_full0 + 8 * s, use & 1, L.wait_ns)) return false;
        tc_fence_after();
        for (int j = 0; j < nk; ++j) {
          const uint32_t a0 = smem_u32(sA + (s * kKPS + j) * kABytes);
          const uint32_t b0 = FP4 ? smem_u32(sJ + (kb0 + j) * NT * 128)
                                  : smem_u32(sB + (s * kKPS + j) * kBBytes);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t acc = (si > 0 || j > 0 || ks > 0) ? 1u : 0u;
            if constexpr (REAL)
              mma_bf16(tmem, sw128_desc(a0 + ks * 32), sw128_desc(b0 + ks * 32), idesc, acc);
            else if constexpr (FP4)
              mma_mxf4(tmem, sw128_desc(a0 + ks * 32), sw128_desc(b0 + ks * 32), idesc, tmem + NT,
                       tmem + NT, acc);
            else
              mma_e4m3(tmem, sw128_desc(a0 + ks * 32), sw128_desc(b0 + ks * 32), idesc, acc);
          }
        }
        mma_commit(bar_empty0 + 8 * s);
        ++mmas;
      }
      mma_commit(bar_done);
      return true;
    };

    // Best / first-hit bookkeeping of state `state` = s(tt) from its replica energy, complete
    // since the barrier that ended sweep tt.  Returns that energy.
    EAcc* energy = reinterpret_cast<EAcc*>(L.energy);
    auto track = [&](int tt, uint32_t state) -> EAcc {
      // L2 read: the accumulator was written by other SMs during sweep tt.
      const EAcc etot = __ldcg(&energy[((tt - t_begin) % 3) * rpad + rl]);
      EAcc E;
      bool hit;
      if constexpr (REAL) {
        E = -0.5f * etot;
        hit = static_cast<double>(E) <= P.target_f;
      } else {
        E = -(etot / 2);  // s^T J s is even for symmetric integer J with zero diagonal
        hit = static_cast<long long>(E) <= P.target;
      }
      if (E < best_E) {
        best_E = E;
        best_t = tt;
        best = state;
      }
      if (has_target && first_hit < 0 && hit) first_hit = tt;
      return E;
    };

    int cur_img = 0;
    uint32_t prev = 0;  // s(t-1) of this thread's spins, until its energy has been tracked
    for (int t = t_begin; t <= t_end; ++t) {
      const bool last = t == t_end;
      if (tid == 0) {
        fence_proxy_async_global();
        // Injected fault: nothing is loaded in the first sweep, so the MMA thread's first
        // wait cannot complete.
        if (!(L.inject == 1 && t == t_begin) && !produce(L.s_img[cur_img], kRev && (t & 1))) {
          atomicOr(L.err, kDevErrTimeout);
          grid_abort(L.bar);
        }
      } else if (tid == 32) {
        if (!multiply(kRev && (t & 1))) {
          atomicOr(L.err, kDevErrTimeout);
          grid_abort(L.bar);
        }
      }
      // Zero the energy buffer that sweep t+1 will accumulate into (see header).
      if (cb == 0 && epi && grp == 0) __stcg(&energy[((t - t_begin + 1) % 3) * rpad + rl], EAcc(0));
      EAcc eacc = 0;
      uint32_t nxt = 0;
      const bool tab_in_smem = !REAL && tab_smem;
      if (epi) {
        // While the MMAs run: the bookkeeping of s(t-1), whose energy the last barrier
        // completed, and this step's thresholds staged (the previous step's reads ended
        // before that barrier); then sync the 16 epilogue warps.
        if (t > t_begin) track(t - 1, prev);
        if (tab_in_smem && !last) {
          const uint4* src =
              reinterpret_cast<const uint4*>(P.thr + static_cast<size_t>(t) * P.stride_words);
          for (int k = tid - 64; k < P.stride_words / 4; k += kEpiWarps * 32)
            reinterpret_cast<uint4*>(sTab)[k] = __ldg(src + k);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory");
        const bool ok = mbar_wait_fast(bar_done, done_phase, L.wait_ns);
        if (!ok) {
          atomicOr(L.err, kDevErrTimeout);
          grid_abort(L.bar);
        }
        tc_fence_after();
        if (warp_active) {
          const uint32_t* tab = nullptr;
          float b = 0.0f, eta = 0.0f;
          float* dump = nullptr;  // diagnostics: fields of the first sweep (real couplings)
          if (REAL && P.fields_out != nullptr && t == t_begin && !last && row_valid)
            dump = P.fields_out + static_cast<size_t>(r) * n + col0;
          if constexpr (REAL) {
            if (!last) {
              b = P.sched_b[t];
              eta = P.sched_eta[t];
            }
          } else {
            tab = tab_in_smem ? sTab : P.thr + static_cast<size_t>(last ? t_begin : t) * P.stride_words;
          }
#pragma unroll
          for (int c = 0; c < kChunks; ++c) {
            uint32_t v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(quad * 32) << 16) + grp * kSPT + 16 * c, v);
            PhiloxOut o0{}, o1{};
            if (!last) {
              const uint32_t ctr = static_cast<uint32_t>((col0 + 16 * c) >> 3);
              o0 = philox4x32_10_rk(ctr, static_cast<uint32_t>(r), static_cast<uint32_t>(t), P.q,
                                    L.round_keys);
              o1 = philox4x32_10_rk(ctr + 1u, static_cast<uint32_t>(r), static_cast<uint32_t>(t),
                                    P.q, L.round_keys);
            }
            tmem_wait_ld(v);
            const uint32_t rw[8] = {o0.x0, o0.x1, o0.x2, o0.x3, o1.x0, o1.x1, o1.x2, o1.x3};
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int bit = 16 * c + e;
              const uint32_t s = (cur >> bit) & 1u;
              const uint32_t word = rw[e >> 1];
              const uint32_t key = (e & 1) ? (word >> 20) : ((word >> 4) & 0xFFFu);
              if constexpr (REAL) {
                const float hv = __uint_as_float(sH[grp * kSPT + bit]);
                const float I = __fadd_rn(__uint_as_float(v[e]), hv);
                if (dump != nullptr && col0 + bit < n) dump[bit] = I;
                const float term = __fadd_rn(I, hv);
                eacc += s ? term : -term;
                if (!last) {
                  const float x = __fmul_rn(b, I);
                  const float tau = P.act == 0 ? tanhf(x) : staircase(x, P.lut_levels);
                  const float a = __fadd_rn(tau, s ? P.xi : -P.xi);
                  const float delta = __fadd_rn(a, __fmul_rn(eta, sZ[key]));
                  nxt |= (delta >= 0.0f ? 1u : 0u) << bit;
                }
              } else {
                const int hv = static_cast<int>(sH[grp * kSPT + bit]);
                const int I = __float2int_rn(__uint_as_float(v[e])) + hv;
                const int term = I + hv;
                eacc += s ? term : -term;
                if (!last) {
                  const uint32_t w = tab[I + P.imax];
                  const uint32_t th = s ? (w >> 16) : (w & 0xFFFFu);
                  nxt |= (key >= th ? 1u : 0u) << bit;
                }
              }
            }
          }
          nxt &= vmask;
        }
        sRed[grp * 128 + row] = eacc;
      }
      done_phase ^= 1;
      if (!last) write_image(L.s_img[cur_img ^ 1], nxt);
      tc_fence_before();
      __syncthreads();
      if (epi && grp == 0) {
        const EAcc tot = sRed[row] + sRed[128 + row] + sRed[256 + row] + sRed[384 + row];
        atomicAdd(&energy[((t - t_begin) % 3) * rpad + rl], tot);
      }
      fence_proxy_async_global();
      bar_target += nblocks;
      if (!grid_barrier(L.bar, bar_target, L.err, sFlag, L.wait_ns)) goto teardown;
      if (epi) {
        if (last) {
          const EAcc E = track(t, cur);
          if (row_valid) {
#pragma unroll
            for (int c = 0; c < kChunks; ++c)
              if (chunk + c < half_words) {
                const size_t o = static_cast<size_t>(r) * half_words + chunk + c;
                reinterpret_cast<uint16_t*>(P.cur_bits)[o] = static_cast<uint16_t>(cur >> (16 * c));
                reinterpret_cast<uint16_t*>(P.best_bits)[o] = static_cast<uint16_t>(best >> (16 * c));
              }
            if (cb == 0 && grp == 0) {
              P.best_E[r] = static_cast<double>(best_E);
              P.best_t[r] = best_t;
              P.first_hit[r] = first_hit;
              P.final_E[r] = static_cast<double>(E);
            }
          }
        } else {
          prev = cur;
          cur = nxt;
        }
      }
      cur_img ^= 1;
    }
  }

teardown:
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, C::kTmemCols);
}

// Kernel and co-resident CTAs of the (NT, OP) variant at `smem` bytes of dynamic shared
// memory (the attribute is set to the whole budget, so any plan of the variant launches).
template <int NT, int OP>
cudaError_t variant_setup(int smem, const void** fn, int* max_blocks) {
  *fn = reinterpret_cast<const void*>(sweep_big_kernel<NT, OP>);
  const int attr = OP == kBigFp4 ? kSmemBudget : BigCfg<NT, OP>::kSmem;
  cudaError_t e = cudaFuncSetAttribute(sweep_big_kernel<NT, OP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, attr);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_big_kernel<NT, OP>, kThreads,
                                                    smem);
  if (e != cudaSuccess) return e;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *max_blocks = per_sm * sms;
  return cudaSuccess;
}

cudaError_t variant(int nt, int op, int smem, const void** fn, int* max_blocks) {
  if (op == kBigFp4) return nt == 64 ? variant_setup<64, kBigFp4>(smem, fn, max_blocks)
                                     : cudaErrorInvalidValue;
  const bool real = op == kBigBf16;
  if (op != kBigFp8 && op != kBigBf16) return cudaErrorInvalidValue;
  if (nt == 64) return real ? variant_setup<64, kBigBf16>(smem, fn, max_blocks)
                            : variant_setup<64, kBigFp8>(smem, fn, max_blocks);
  if (nt == 128) return real ? variant_setup<128, kBigBf16>(smem, fn, max_blocks)
                             : variant_setup<128, kBigFp8>(smem, fn, max_blocks);
  return cudaErrorInvalidValue;
}

template <int NT, int OP>
BigSmem streamed_plan(int stride_words) {
  BigSmem out;
  out.ok = true;
  out.stages = BigCfg<NT, OP>::kStages;
  out.tab_smem = OP == kBigFp8 && stride_words <= kTabWords ? 1 : 0;
  out.bytes = BigCfg<NT, OP>::kSmem;
  return out;
}

}  // namespace

BigSmem sweep_big_smem(int nt, int op, int npad, int stride_words) {
  if (op == kBigFp4) return nt == 64 ? fp4_plan(npad, stride_words) : BigSmem{};
  if (op == kBigFp8) {
    if (nt == 64) return streamed_plan<64, kBigFp8>(stride_words);
    if (nt == 128) return streamed_plan<128, kBigFp8>(stride_words);
  } else if (op == kBigBf16) {
    if (nt == 64) return streamed_plan<64, kBigBf16>(stride_words);
    if (nt == 128) return streamed_plan<128, kBigBf16>(stride_words);
  }
  return BigSmem{};
}

int sweep_big_max_blocks(int nt, int op, int npad, int stride_words) {
  const BigSmem plan = sweep_big_smem(nt, op, npad, stride_words);
  if (!plan.ok) return 0;
  const void* fn = nullptr;
  int blocks = 0;
  return variant(nt, op, plan.bytes, &fn, &blocks) == cudaSuccess ? blocks : 0;
}

cudaError_t launch_sweep_big(const BigLaunch& L, int nt, int op, int blocks, cudaStream_t st) {
  const BigSmem plan = sweep_big_smem(nt, op, L.P.npad, L.P.stride_words);
  if (!plan.ok || L.stages != plan.stages || L.tab_smem != plan.tab_smem) return cudaErrorInvalidValue;
  if (op == kBigFp4 && L.j4 == nullptr) return cudaErrorInvalidValue;
  const void* fn = nullptr;
  int cap = 0;
  cudaError_t e = variant(nt, op, plan.bytes, &fn, &cap);
  if (e != cudaSuccess) return e;
  if (blocks > cap) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {const_cast<BigLaunch*>(&L)};
  e = cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kThreads), args, plan.bytes, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace pim
