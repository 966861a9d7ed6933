// Conventional PIM with sequential updates (Eq. 3; Box 1, orange path), the baseline the
// fully parallel loop is compared with.  One warp per replica; sweep k updates spins
// i = 0 .. n-1 one after another, each from the field of the current state:
//   the replica's fields I_i = sum_j J_ij s_j + h_i and its spins live in shared memory;
//   step (k, i): every lane reads I_i and s_i (broadcast), takes the 12-bit key of draw
//   (i>>3, r, k, q) -- one Philox block per 8 consecutive spins -- and decides with the
//   threshold table of schedule entry k (the same exact decisions as the parallel path);
//   on a flip the warp adds 2 s_i' J_i (row i of J = column i, coalesced int8 loads) to I.
// Energies E = -1/2 sum_i s_i (I_i + h_i) are evaluated on the state at the start of every
// sweep and on the final state, with the best-state / first-hit bookkeeping of the
// parallel kernels.  No waits between warps: every warp runs on its own.
#include <climits>

#include "kernels.h"
#include "philox.cuh"

namespace pim {
namespace {

constexpr int kWarps = 4;  // replicas per block

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__global__ void __launch_bounds__(kWarps * 32) sequential_kernel(const __grid_constant__ SeqLaunch L) {
  extern __shared__ int smem_seq[];
  const Problem& P = L.P;
  const int n = P.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * kWarps + warp;
  if (r >= P.R) return;  // a whole warp; the kernel has no block-level synchronisation
  int* I = smem_seq + static_cast<size_t>(warp) * n;                                   // [n]
  int8_t* s = reinterpret_cast<int8_t*>(smem_seq + static_cast<size_t>(kWarps) * n) +
              static_cast<size_t>(warp) * n;                                           // [n]
  const int words = P.words;
  uint32_t* cur_io = P.cur_bits + static_cast<size_t>(r) * words;
  uint32_t* best_io = P.best_bits + static_cast<size_t>(r) * words;
  const int8_t* J = P.j8;
  const int32_t* h = P.h;
  const int imax = P.imax, stride = P.stride_words;

  for (int j = lane; j < n; j += 32) s[j] = ((cur_io[j >> 5] >> (j & 31)) & 1u) ? 1 : -1;
  __syncwarp();
  // fields of the starting state, one row of J per iteration, lanes across the row
  for (int i = 0; i < n; ++i) {
    const int8_t* Ji = J + static_cast<size_t>(i) * n;
    int acc = 0;
    for (int j = lane; j < n; j += 32) acc += Ji[j] * s[j];
    acc = static_cast<int>(warp_sum(acc));
    if (lane == 0) I[i] = acc + (h ? h[i] : 0);
  }
  __syncwarp();

  long long best_E = LLONG_MAX;
  int best_t = -1, first_hit = -1;
  if (L.cont) {
    best_E = static_cast<long long>(P.best_E[r]);
    best_t = P.best_t[r];
    first_hit = P.first_hit[r];
  }
  // E(s) on the current state, bookkeeping at schedule index t; returns E.
  auto evaluate = [&](int t) -> long long {
    long long acc = 0;
    for (int j = lane; j < n; j += 32) acc += static_cast<long long>(s[j]) * (I[j] + (h ? h[j] : 0));
    const long long E = -(warp_sum(acc) / 2);
    if (E < best_E) {
      best_E = E;
      best_t = t;
      for (int w = lane; w < words; w += 32) {
        uint32_t b = 0;
        for (int e = 0; e < 32; ++e) {
          const int j = 32 * w + e;
          if (j < n && s[j] > 0) b |= 1u << e;
        }
        best_io[w] = b;
      }
    }
    if (P.has_target && first_hit < 0 && E <= P.target) first_hit = t;
    return E;
  };

  const int t_end = L.t_begin + L.sweeps;
  for (int k = L.t_begin; k < t_end; ++k) {
    evaluate(k);
    const uint32_t* tab = P.thr + static_cast<size_t>(k) * stride;
    uint32_t rw[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
      if ((i & 7) == 0) {
        const PhiloxOut o = philox4x32_10_rk(static_cast<uint32_t>(i >> 3), static_cast<uint32_t>(r),
                                             static_cast<uint32_t>(k), P.q, L.round_keys);
        rw[0] = o.x0;
        rw[1] = o.x1;
        rw[2] = o.x2;
        rw[3] = o.x3;
      }
      const int si = s[i];
      const int Ii = I[i];
      const uint32_t word = rw[(i & 7) >> 1];
      const uint32_t key = (i & 1) ? (word >> 20) : ((word >> 4) & 0xFFFu);
      const uint32_t w = tab[Ii + imax];
      const uint32_t th = si > 0 ? (w >> 16) : (w & 0xFFFFu);
      const int snew = key >= th ? 1 : -1;
      if (snew != si) {  // the same on every lane
        const int d = snew - si;
        const int8_t* Ji = J + static_cast<size_t>(i) * n;
        for (int j = lane; j < n; j += 32) I[j] += Ji[j] * d;
        __syncwarp();
        if (lane == 0) s[i] = static_cast<int8_t>(snew);
      }
      __syncwarp();
    }
  }
  const long long E = evaluate(t_end);
  for (int w = lane; w < words; w += 32) {
    uint32_t b = 0;
    for (int e = 0; e < 32; ++e) {
      const int j = 32 * w + e;
      if (j < n && s[j] > 0) b |= 1u << e;
    }
    cur_io[w] = b;
  }
  if (lane == 0) {
    P.best_E[r] = static_cast<double>(best_E);
    P.best_t[r] = best_t;
    P.first_hit[r] = first_hit;
    P.final_E[r] = static_cast<double>(E);
  }
}

}  // namespace

int sequential_smem_bytes(int n) { return kWarps * n * 5; }

cudaError_t launch_sequential(const SeqLaunch& L, cudaStream_t st) {
  const int smem = sequential_smem_bytes(L.P.n);
  cudaError_t e = cudaFuncSetAttribute(sequential_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int blocks = (L.P.R + kWarps - 1) / kWarps;
  sequential_kernel<<<blocks, kWarps * 32, smem, st>>>(L);
  return cudaGetLastError();
}

}  // namespace pim
