// Large-N PIMI sweep kernel (N > 256): persistent, cooperative, one CTA per (128-replica
// tile, 64-spin column block), all sweeps in one launch.
//
// Per sweep t (Box 1, PIMI loop; Eq. 2 then Eq. 4):
//   fields   D[r, i] = sum_j S[r, j] J[i, j] for the CTA's 128 replicas and 64 spins: the
//            K dimension (all N spins) streams through a 7-stage shared-memory ring filled
//            by cp.async.bulk (spins of the tile from the global spin image, rows of J from
//            the FP8 coupling image), consumed by tcgen05.mma kind::f8f6f4 into TMEM.
//   decision 16 epilogue warps (4 TMEM lane quadrants x 4 column groups); each thread owns
//            one replica and 16 spins for the whole anneal, keeps their old / new / best
//            bits in registers, draws the Philox block, looks the threshold up by field
//            I = D + h in the step's threshold table (staged into shared memory while the
//            MMAs run, or read through L1 when it is larger), writes the new spins as FP8
//            bytes into the other spin image, and adds its share of sum_i s_i (I_i + h_i)
//            to the replica's energy accumulator (global atomics, three rotating buffers).
//   exchange a bounded grid barrier; every CTA then reads the replica energies of s(t),
//            updates best / first hit (redundantly, identically in all CTAs) and copies its
//            own 16 old spins into the best state when the energy improved.
#include <climits>

#include "kernels.h"
#include "philox.cuh"
#include "sm100_ptx.cuh"

namespace pim {
namespace {

constexpr int kNT = 64;           // spins (output columns) per CTA
constexpr int kStages = 7;        // K-block ring depth
constexpr int kTabWords = 8192;   // threshold table of one step staged in shared memory
constexpr int kABytes = 128 * 128;  // one K-block of the spin tile (128 rows x 128 B)
constexpr int kBBytes = kNT * 128;  // one K-block of the coupling rows (64 rows x 128 B)
constexpr int kEpiWarps = 16;
constexpr int kThreads = (2 + kEpiWarps) * 32;

__device__ __forceinline__ uint32_t ld_acquire(const unsigned int* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned int* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Grid-wide barrier with a time bound.  bar[0] = arrivals, bar[1] = generation,
// bar[2] = abort flag.  Returns false (on all threads of the CTA) when the barrier gave up
// or another CTA aborted.
__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, int* err, int* sflag,
                             uint64_t limit_ns) {
  const uint64_t limit = limit_ns ? limit_ns : 2000000000ull;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const uint32_t g = ld_acquire(&bar[1]);
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == nblocks - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      st_release(&bar[1], g + 1);
    } else {
      const uint64_t t0 = global_ns();
      while (ld_acquire(&bar[1]) == g) {
        if (ld_acquire(&bar[2]) != 0) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > limit) {
          atomicOr(err, kDevErrTimeout);
          atomicExch(&bar[2], 1u);
          ok = 0;
          break;
        }
      }
    }
    if (ld_acquire(&bar[2]) != 0) ok = 0;  // another CTA gave up: everyone stops
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

__global__ void __launch_bounds__(kThreads, 1) sweep_big_kernel(const __grid_constant__ BigLaunch L) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;                           // kStages x kABytes
  uint8_t* sB = sA + kStages * kABytes;         // kStages x kBBytes
  uint32_t* sTab = reinterpret_cast<uint32_t*>(sB + kStages * kBBytes);  // [kTabWords]
  float* sRed = reinterpret_cast<float*>(sTab + kTabWords);  // [4 groups][128 rows]
  int* sH = reinterpret_cast<int*>(sRed + 4 * 128);                // [kNT]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sH + kNT);          // full[S], empty[S], done
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
  int* sFlag = reinterpret_cast<int*>(sTmem + 1);

  const Problem& P = L.P;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncb = L.ncb;
  const int cb = blockIdx.x % ncb, rt = blockIdx.x / ncb;
  const unsigned int nblocks = gridDim.x;
  const int n = P.n, npad = P.npad, R = P.R, rpad = L.rpad;
  const int kblocks = npad / 128;
  const int t_begin = L.t_begin, t_end = L.t_begin + L.sweeps;
  const bool epi = warp >= 2;
  const int ew = warp - 2;             // epilogue warp 0..15
  const int quad = warp & 3;           // TMEM lane quadrant of this warp
  const int grp = epi ? ew >> 2 : 0;   // column group 0..3 (16 spins each)
  const int row = quad * 32 + lane;    // replica row inside the tile
  const int rl = rt * 128 + row;       // replica row inside this launch's images
  const int r = L.rbase + rl;          // replica index
  const int col0 = cb * kNT + grp * 16;  // first spin of this thread's 16
  const bool row_valid = epi && r < R;
  const bool warp_active = epi && (L.rbase + rt * 128 + quad * 32) < R && col0 < n;
  const int valid = n - col0;            // spins of the 16 that exist
  const uint32_t vmask = valid >= 16 ? 0xFFFFu : (valid > 0 ? (1u << valid) - 1u : 0u);

  const uint32_t bar_full0 = smem_u32(&bars[0]);
  const uint32_t bar_empty0 = smem_u32(&bars[kStages]);
  const uint32_t bar_done = smem_u32(&bars[2 * kStages]);

  if (warp == 1) {
    tmem_alloc(smem_u32(sTmem), kNT);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar_full0 + 8 * s, 1);
      mbar_init(bar_empty0 + 8 * s, 1);
    }
    mbar_init(bar_done, 1);
    fence_mbar_init();
  }
  for (int k = tid; k < kNT; k += kThreads) {
    const int i = cb * kNT + k;
    sH[k] = (P.h != nullptr && i < n) ? P.h[i] : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;

  // ---- per-thread state: this replica's 16 spins ------------------------------------
  uint32_t cur = 0, best = 0;
  int best_E = INT_MAX, best_t = -1, first_hit = -1;
  const int half_words = P.words * 2;  // 16-bit chunks per row in the caller's bit arrays
  const int chunk = col0 >> 4;
  if (row_valid && chunk < half_words) {
    cur = reinterpret_cast<const uint16_t*>(P.cur_bits)[static_cast<size_t>(r) * half_words + chunk];
    if (L.cont) {
      best = reinterpret_cast<const uint16_t*>(P.best_bits)[static_cast<size_t>(r) * half_words + chunk];
      best_E = static_cast<int>(P.best_E[r]);
      best_t = P.best_t[r];
      first_hit = P.first_hit[r];
    }
  }
  if (!L.cont) best = cur;
  const bool has_target = P.has_target != 0;
  const long long target = P.target;

  // Initial spin image s(t_begin) for this CTA's block (rows of the tile, its 64 spins).
  auto write_image = [&](uint8_t* img, uint32_t bits) {
    if (!epi || col0 >= npad) return;
    const uint4 bytes = make_uint4(
        ((((bits >> 0) & 0xFu) * 0x10204080u) & 0x80808080u) ^ 0xB8B8B8B8u,
        ((((bits >> 4) & 0xFu) * 0x10204080u) & 0x80808080u) ^ 0xB8B8B8B8u,
        ((((bits >> 8) & 0xFu) * 0x10204080u) & 0x80808080u) ^ 0xB8B8B8B8u,
        ((((bits >> 12) & 0xFu) * 0x10204080u) & 0x80808080u) ^ 0xB8B8B8B8u);
    *reinterpret_cast<uint4*>(img + sw128_offset(rl, col0, rpad)) = bytes;
  };
  write_image(L.s_img[0], cur & vmask);
  fence_proxy_async_global();
  if (!grid_barrier(L.bar, nblocks, L.err, sFlag, L.wait_ns)) goto teardown;

  {
    uint32_t loads = 0, mmas = 0, done_phase = 0;
    const uint32_t idesc = (1u << 4) | (static_cast<uint32_t>(kNT >> 3) << 17) |
                           (static_cast<uint32_t>(128 >> 4) << 24);
    // Producer (thread 0): stream the K blocks of image `img` (spins of the tile) and of the
    // coupling rows of the column block into the ring.  A stage is refilled once the MMAs
    // that read it have completed (its empty barrier).
    auto produce = [&](const uint8_t* img) -> bool {
      const uint8_t* a_src = img + static_cast<size_t>(rt) * 128 * 128;
      const uint8_t* b_src = P.jimg + static_cast<size_t>(cb) * kNT * 128;
      for (int kb = 0; kb < kblocks; ++kb) {
        const uint32_t s = loads % kStages, use = loads / kStages;
        if (use > 0 && !mbar_wait_bounded(bar_empty0 + 8 * s, (use - 1) & 1, L.wait_ns)) return false;
        mbar_expect_tx(bar_full0 + 8 * s, kABytes + kBBytes);
        bulk_g2s(smem_u32(sA + s * kABytes), a_src + static_cast<size_t>(kb) * rpad * 128, kABytes,
                 bar_full0 + 8 * s);
        bulk_g2s(smem_u32(sB + s * kBBytes), b_src + static_cast<size_t>(kb) * npad * 128, kBBytes,
                 bar_full0 + 8 * s);
        ++loads;
      }
      return true;
    };
    // MMA issuer (thread 32): D = S_tile x J_block^T, K block by K block as stages land; it
    // never waits for an MMA to finish, only for data.
    auto multiply = [&]() -> bool {
      for (int kb = 0; kb < kblocks; ++kb) {
        const uint32_t s = mmas % kStages, use = mmas / kStages;
        if (!mbar_wait_bounded(bar_full0 + 8 * s, use & 1, L.wait_ns)) return false;
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          mma_e4m3(tmem, sw128_desc(a0 + ks * 32), sw128_desc(b0 + ks * 32), idesc,
                   (kb > 0 || ks > 0) ? 1u : 0u);
        mma_commit(bar_empty0 + 8 * s);
        ++mmas;
      }
      mma_commit(bar_done);
      return true;
    };

    int cur_img = 0;
    for (int t = t_begin; t <= t_end; ++t) {
      const bool last = t == t_end;
      if (tid == 0) {
        fence_proxy_async_global();
        // Injected fault: nothing is loaded in the first sweep, so the MMA thread's first
        // wait cannot complete.
        if (!(L.inject == 1 && t == t_begin) && !produce(L.s_img[cur_img])) {
          atomicOr(L.err, kDevErrTimeout);
          atomicExch(&L.bar[2], 1u);
        }
      } else if (tid == 32) {
        if (!multiply()) {
          atomicOr(L.err, kDevErrTimeout);
          atomicExch(&L.bar[2], 1u);
        }
      }
      // Zero the energy buffer that sweep t+1 will accumulate into (see header).
      if (cb == 0 && epi && grp == 0) __stcg(&L.energy[((t - t_begin + 1) % 3) * rpad + rl], 0.0f);
      float eacc = 0.0f;
      uint32_t nxt = 0;
      const bool tab_in_smem = P.stride_words <= kTabWords;
      if (epi) {
        // Stage this step's thresholds while the MMAs run (the previous step's reads ended
        // before the last grid barrier), then sync the 16 epilogue warps.
        if (tab_in_smem && !last) {
          const uint4* src =
              reinterpret_cast<const uint4*>(P.thr + static_cast<size_t>(t) * P.stride_words);
          for (int k = tid - 64; k < P.stride_words / 4; k += kEpiWarps * 32)
            reinterpret_cast<uint4*>(sTab)[k] = __ldg(src + k);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory");
        const bool ok = mbar_wait_bounded(bar_done, done_phase, L.wait_ns);
        if (!ok) {
          atomicOr(L.err, kDevErrTimeout);
          atomicExch(&L.bar[2], 1u);
        }
        tc_fence_after();
        if (warp_active) {
          uint32_t v[16];
          tmem_ld16(tmem + (static_cast<uint32_t>(quad * 32) << 16) + grp * 16, v);
          PhiloxOut o0{}, o1{};
          if (!last) {
            o0 = philox4x32_10_rk(static_cast<uint32_t>(col0 >> 3), static_cast<uint32_t>(r),
                                  static_cast<uint32_t>(t), P.q, L.round_keys);
            o1 = philox4x32_10_rk(static_cast<uint32_t>((col0 >> 3) + 1), static_cast<uint32_t>(r),
                                  static_cast<uint32_t>(t), P.q, L.round_keys);
          }
          tmem_wait_ld(v);
          const uint32_t rw[8] = {o0.x0, o0.x1, o0.x2, o0.x3, o1.x0, o1.x1, o1.x2, o1.x3};
          const uint32_t* tab =
              tab_in_smem ? sTab : P.thr + static_cast<size_t>(last ? t_begin : t) * P.stride_words;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int hv = sH[grp * 16 + e];
            const int I = __float2int_rn(__uint_as_float(v[e])) + hv;
            const uint32_t s = (cur >> e) & 1u;
            const int term = I + hv;
            eacc += static_cast<float>(s ? term : -term);
            if (!last) {
              const uint32_t w = tab[I + P.imax];
              const uint32_t th = s ? (w >> 16) : (w & 0xFFFFu);
              const uint32_t word = rw[e >> 1];
              const uint32_t key = (e & 1) ? (word >> 20) : ((word >> 4) & 0xFFFu);
              nxt |= (key >= th ? 1u : 0u) << e;
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
        const float tot = sRed[row] + sRed[128 + row] + sRed[256 + row] + sRed[384 + row];
        atomicAdd(&L.energy[((t - t_begin) % 3) * rpad + rl], tot);
      }
      fence_proxy_async_global();
      if (!grid_barrier(L.bar, nblocks, L.err, sFlag, L.wait_ns)) goto teardown;
      if (epi) {
        // L2 read: the accumulator was written by other SMs during this sweep.
        const float etot = __ldcg(&L.energy[((t - t_begin) % 3) * rpad + rl]);
        const int E = -(static_cast<int>(etot) / 2);
        if (E < best_E) {
          best_E = E;
          best_t = t;
          best = cur;
        }
        if (has_target && first_hit < 0 && E <= target) first_hit = t;
        if (last) {
          if (row_valid && chunk < half_words) {
            reinterpret_cast<uint16_t*>(P.cur_bits)[static_cast<size_t>(r) * half_words + chunk] =
                static_cast<uint16_t>(cur);
            reinterpret_cast<uint16_t*>(P.best_bits)[static_cast<size_t>(r) * half_words + chunk] =
                static_cast<uint16_t>(best);
            if (cb == 0 && grp == 0) {
              P.best_E[r] = static_cast<double>(best_E);
              P.best_t[r] = best_t;
              P.first_hit[r] = first_hit;
              P.final_E[r] = static_cast<double>(E);
            }
          }
        } else {
          cur = nxt;
        }
      }
      cur_img ^= 1;
    }
  }

teardown:
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, kNT);
}

}  // namespace

int sweep_big_smem_bytes() {
  return 1024 + kStages * (kABytes + kBBytes) + kTabWords * 4 + 4 * 128 * 4 + kNT * 4 +
         (2 * kStages + 1) * 8 + 16;
}

int sweep_big_tile_n() { return kNT; }

int sweep_big_max_blocks() {
  const int smem = sweep_big_smem_bytes();
  if (cudaFuncSetAttribute(sweep_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_big_kernel, kThreads, smem) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

cudaError_t launch_sweep_big(const BigLaunch& L, int blocks, cudaStream_t st) {
  const int smem = sweep_big_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(sweep_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_big_kernel, kThreads, smem);
  if (e != cudaSuccess) return e;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (blocks > per_sm * sms) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {const_cast<BigLaunch*>(&L)};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(sweep_big_kernel), dim3(blocks),
                                  dim3(kThreads), args, smem, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace pim
