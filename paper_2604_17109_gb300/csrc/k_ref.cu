// Plain FP32 comparator path: one instance at a time, per sweep one float32 field GEMM
// kernel and one update kernel.  It makes the same decisions as the fused kernel (same
// threshold tables, same noise stream) and is the baseline the fused kernel is measured
// against.
#include "kernels.h"
#include "philox.cuh"

namespace pim {

// I[r][i] = sum_j S[r][j] * J[i][j]  (R x n times n x n^T), 64x64 tiles, 4x4 per thread.
__global__ void __launch_bounds__(256) ref_field_kernel(const float* __restrict__ S,
                                                        const float* __restrict__ Jf, int R,
                                                        int n, float* __restrict__ I) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * 64, i0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int row = e >> 4, kk = e & 15;
      const int r = r0 + row, i = i0 + row, k = k0 + kk;
      As[kk][row] = (r < R && k < n) ? S[static_cast<size_t>(r) * n + k] : 0.0f;
      Bs[kk][row] = (i < n && k < n) ? Jf[static_cast<size_t>(i) * n + k] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty * 4 + u];
        b[u] = Bs[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = r0 + ty * 4 + u, i = i0 + tx * 4 + v;
      if (r < R && i < n) I[static_cast<size_t>(r) * n + i] = acc[u][v];
    }
}

// One block per replica.  Mode 0: decide s(t+1) and book-keep E(s(t)); mode 1 (after the
// last sweep): only book-keep E(s(T)).  S holds s(t) as +-1 floats and is overwritten with
// s(t+1); best / current spins are kept as bits.
__global__ void __launch_bounds__(256) ref_update_kernel(Problem P, int t, int final_pass,
                                                         uint32_t key_lo, uint32_t key_hi,
                                                         int first_pass_fresh,
                                                         float* __restrict__ S,
                                                         const float* __restrict__ I) {
  extern __shared__ uint32_t sh[];  // [words] old bits, [words] new bits
  __shared__ long long red[8];
  __shared__ int better_flag;
  uint32_t* old_bits = sh;
  uint32_t* new_bits = sh + P.words;
  const int r = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long esum = 0;
  for (int base = 0; base < P.words * 32; base += 256) {
    const int i = base + threadIdx.x;
    const bool valid = i < P.n;
    float s = 0.f, acc = 0.f;
    if (valid) {
      s = S[static_cast<size_t>(r) * P.n + i];
      acc = I[static_cast<size_t>(r) * P.n + i];
    }
    const int hi = (valid && P.h) ? P.h[i] : 0;
    const int field = static_cast<int>(acc) + hi;
    const bool up_old = s > 0.f;
    if (valid) esum += up_old ? (field + hi) : -(field + hi);
    bool up_new = false;
    if (valid && !final_pass) {
      const uint32_t w = P.thr[static_cast<size_t>(t) * P.stride_words + (field + P.imax)];
      const uint32_t thr = up_old ? (w >> 16) : (w & 0xFFFFu);
      const PhiloxOut o = philox4x32_10(static_cast<uint32_t>(i >> 3), static_cast<uint32_t>(r),
                                        static_cast<uint32_t>(t), P.q, key_lo, key_hi);
      const uint32_t key = philox_half(o, i & 7) >> 4;
      up_new = key >= thr;
      S[static_cast<size_t>(r) * P.n + i] = up_new ? 1.0f : -1.0f;
    }
    const uint32_t bo = __ballot_sync(0xFFFFFFFFu, valid && up_old);
    const uint32_t bn = __ballot_sync(0xFFFFFFFFu, valid && up_new);
    const int wi = (base >> 5) + warp;
    if (lane == 0 && wi < P.words) {
      old_bits[wi] = bo;
      new_bits[wi] = bn;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) esum += __shfl_xor_sync(0xFFFFFFFFu, esum, off);
  if (lane == 0) red[warp] = esum;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int k = 0; k < 8; ++k) tot += red[k];
    const long long E = -(tot / 2);
    const bool fresh = first_pass_fresh != 0;
    const double bestE = fresh ? 0.0 : P.best_E[r];
    const bool better = fresh || static_cast<double>(E) < bestE;
    if (better) {
      P.best_E[r] = static_cast<double>(E);
      P.best_t[r] = t;
    }
    if (fresh) P.first_hit[r] = -1;
    if (P.has_target && (fresh || P.first_hit[r] < 0) && E <= P.target) P.first_hit[r] = t;
    if (final_pass) P.final_E[r] = static_cast<double>(E);
    better_flag = better;
  }
  __syncthreads();
  for (int w = threadIdx.x; w < P.words; w += 256) {
    if (better_flag) P.best_bits[static_cast<size_t>(r) * P.words + w] = old_bits[w];
    P.cur_bits[static_cast<size_t>(r) * P.words + w] = final_pass ? old_bits[w] : new_bits[w];
  }
}

__global__ void ref_expand_kernel(Problem P, float* __restrict__ S) {
  const int r = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const uint32_t w = P.cur_bits[static_cast<size_t>(r) * P.words + (i >> 5)];
  S[static_cast<size_t>(r) * P.n + i] = ((w >> (i & 31)) & 1u) ? 1.0f : -1.0f;
}

cudaError_t launch_ref_anneal(const Problem* h_probs, const Problem* d_probs, int nprob,
                              int t_begin, int sweeps, uint32_t key_lo, uint32_t key_hi,
                              int cont, float* d_S, float* d_I, int* d_err, cudaStream_t st) {
  (void)d_probs;
  (void)d_err;
  for (int p = 0; p < nprob; ++p) {
    const Problem& P = h_probs[p];
    ref_expand_kernel<<<dim3((P.n + 255) / 256, P.R), 256, 0, st>>>(P, d_S);
    const dim3 ggrid((P.n + 63) / 64, (P.R + 63) / 64);
    const size_t shm = 2 * P.words * sizeof(uint32_t);
    for (int s = 0; s <= sweeps; ++s) {
      const int t = t_begin + s;
      ref_field_kernel<<<ggrid, 256, 0, st>>>(d_S, P.jf, P.R, P.n, d_I);
      const int fresh = (s == 0 && !cont) ? 1 : 0;
      ref_update_kernel<<<P.R, 256, shm, st>>>(P, t, s == sweeps ? 1 : 0, key_lo, key_hi, fresh,
                                               d_S, d_I);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pim
