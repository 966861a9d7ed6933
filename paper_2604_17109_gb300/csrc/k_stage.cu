// Staging kernels: coupling images, decision thresholds and initial spins.
#include <cuda_fp8.h>

#include "kernels.h"
#include "philox.cuh"

namespace pim {

// ---------------------------------------------------------------------------------------
// J (int8, row-major n x n) -> FP8 E4M3 operand image of the fused kernel.  The image is
// the K-major layout in which the MMA reads the B operand: row i (output spin), K = j,
// value J_ij; zero outside n x n.  One thread per image byte.
// ---------------------------------------------------------------------------------------
__global__ void stage_fp8_image_kernel(const int8_t* __restrict__ J, int n, int npad, int diag,
                                       int e5m2, int chunk_major, uint8_t* __restrict__ img) {
  const uint32_t dst = blockIdx.x * blockDim.x + threadIdx.x;
  if (dst >= static_cast<uint32_t>(npad) * npad) return;
  const uint32_t block_bytes = static_cast<uint32_t>(npad) * 128u;
  uint32_t off = dst;  // position in the K-block-major layout
  if (chunk_major) {
    // 16 KB block q = (row block c) * kblocks + kb holds K-block kb of rows 128 c .. 128 c + 127
    const uint32_t kblocks = static_cast<uint32_t>(npad) >> 7, q = dst >> 14;
    off = (q % kblocks) * block_bytes + (q / kblocks) * 16384u + (dst & 16383u);
  }
  const int kb = off / block_bytes;
  const uint32_t rem = off % block_bytes;
  const int i = (rem >> 10) * 8 + ((rem & 1023) >> 7);
  const int within = rem & 127;
  const int chunk = (within >> 4) ^ (i & 7);
  const int j = kb * 128 + chunk * 16 + (within & 15);
  uint8_t v = 0;
  if (i < n && j < n) {
    const int val = i == j ? diag : J[static_cast<size_t>(i) * n + j];
    const __nv_fp8_storage_t e = __nv_cvt_float_to_fp8(static_cast<float>(val), __NV_SATFINITE,
                                                       e5m2 ? __NV_E5M2 : __NV_E4M3);
    v = static_cast<uint8_t>(e);
  }
  img[dst] = v;
}

cudaError_t launch_stage_fp8_image(const int8_t* d_J, int n, int npad, int diag, uint8_t* d_img,
                                   cudaStream_t st, bool e5m2, bool chunk_major) {
  if (chunk_major && npad % 128 != 0) return cudaErrorInvalidValue;
  const uint32_t total = static_cast<uint32_t>(npad) * npad;
  stage_fp8_image_kernel<<<(total + 255) / 256, 256, 0, st>>>(d_J, n, npad, diag, e5m2 ? 1 : 0,
                                                              chunk_major ? 1 : 0, d_img);
  return cudaGetLastError();
}

// E2M1 coupling image of the coupling-resident large-N variant (column block width 64):
// [npad/64 column blocks][npad/256 K-blocks][64 rows x 128 B], each row holding 256 packed
// E2M1 values (element j in nibble j % 2 of byte j / 2, low nibble first) with the 128-byte
// swizzle, so one column block's couplings are contiguous.  Couplings are integers in
// {0, +-1, +-2, +-3, +-4, +-6} (checked by the host), all exact in E2M1 (sign, 2-bit
// exponent, 1-bit mantissa).  One thread per 16-byte chunk (32 couplings).
__device__ __forceinline__ uint32_t e2m1_code(int v) {
  const int a = v < 0 ? -v : v;
  const uint32_t mag = a == 1 ? 2u : a == 2 ? 4u : a == 3 ? 5u : a == 4 ? 6u : a == 6 ? 7u : 0u;
  return mag | (v < 0 && mag ? 8u : 0u);
}

__global__ void stage_fp4_image_kernel(const int8_t* __restrict__ J, int n, int npad,
                                       uint8_t* __restrict__ img) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t chunks = static_cast<uint32_t>(npad) * npad / 32u;
  if (q >= chunks) return;
  const int kb4 = npad / 256;
  const uint32_t block = q / 512u, within = q % 512u;
  const int cb = block / kb4, kb = block % kb4;
  const int r = within / 8, pc = within % 8;
  const int i = cb * 64 + r;
  const int j0 = kb * 256 + ((pc ^ (r & 7)) * 32);
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  if (i < n) {
    const int8_t* row = J + static_cast<size_t>(i) * n;
    for (int e = 0; e < 32; ++e) {
      const int j = j0 + e;
      const uint32_t code = j < n ? e2m1_code(row[j]) : 0u;
      w[e >> 3] |= code << (4 * (e & 7));
    }
  }
  reinterpret_cast<uint4*>(img)[q] = make_uint4(w[0], w[1], w[2], w[3]);
}

cudaError_t launch_stage_fp4_image(const int8_t* d_J, int n, int npad, uint8_t* d_img,
                                   cudaStream_t st) {
  if (npad % 256) return cudaErrorInvalidValue;
  const uint32_t chunks = static_cast<uint32_t>(npad) * npad / 32u;
  stage_fp4_image_kernel<<<(chunks + 255) / 256, 256, 0, st>>>(d_J, n, npad, d_img);
  return cudaGetLastError();
}

__global__ void stage_f32_kernel(const int8_t* __restrict__ J, int n, float* __restrict__ jf) {
  const size_t k = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < static_cast<size_t>(n) * n) jf[k] = static_cast<float>(J[k]);
}

cudaError_t launch_stage_f32(const int8_t* d_J, int n, float* d_jf, cudaStream_t st) {
  const size_t total = static_cast<size_t>(n) * n;
  stage_f32_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(d_J, n, d_jf);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Decision thresholds.  For step t, field I and current spin s the float32 rule
//   a = tau_t(I) + (s>0 ? xi : -xi);   delta(m) = a + eta_t * z(m);   s' = +1 iff delta >= 0
// is non-decreasing in the key m (z is increasing, both roundings are monotone), so it is
// exactly "m >= M" with M the least key giving delta >= 0 (4096 = never).  Each thread
// finds M for one (t, I) and both s by bisection, with explicitly rounded float32
// operations (no contraction into FMA).  Word = M(s=-1) | M(s=+1) << 16.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t least_up_key(float a, float eta, const float* z) {
  int lo = 0, hi = 4096;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const float delta = __fadd_rn(a, __fmul_rn(eta, z[mid]));
    if (delta >= 0.0f)
      hi = mid;
    else
      lo = mid + 1;
  }
  return static_cast<uint32_t>(lo);
}

__global__ void thresholds_kernel(const float* __restrict__ tau, const float* __restrict__ eta,
                                  const float* __restrict__ z, float xi, int imax,
                                  int stride_words, uint32_t* __restrict__ thr) {
  __shared__ float zs[4096];
  for (int k = threadIdx.x; k < 4096; k += blockDim.x) zs[k] = z[k];
  __syncthreads();
  const int t = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int width = 2 * imax + 1;
  if (idx >= stride_words) return;
  uint32_t word = 0;
  if (idx < width) {
    const float tv = tau[static_cast<size_t>(t) * width + idx];
    const float e = eta[t];
    const uint32_t m_down = least_up_key(__fadd_rn(tv, -xi), e, zs);
    const uint32_t m_up = least_up_key(__fadd_rn(tv, xi), e, zs);
    word = m_down | (m_up << 16);
  }
  thr[static_cast<size_t>(t) * stride_words + idx] = word;
}

cudaError_t launch_thresholds(const float* d_tau, const float* d_eta, const float* d_z,
                              float xi, int steps, int imax, int stride_words,
                              uint32_t* d_thr, cudaStream_t st) {
  dim3 grid((stride_words + 127) / 128, steps);
  thresholds_kernel<<<grid, 128, 0, st>>>(d_tau, d_eta, d_z, xi, imax, stride_words, d_thr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Thresholds re-indexed by D = I + 256 s: entry D + 512 holds M(s = sign D, I = D - 256 s).
// With |I| <= imax <= 255 the two ranges D < 0 (s = -1) and D > 0 (s = +1) are disjoint;
// unreachable entries are zero.
// ---------------------------------------------------------------------------------------
__global__ void diag_thresholds_kernel(const uint32_t* __restrict__ thr, int imax, int stride_words,
                                       int K, uint16_t* __restrict__ out) {
  const int t = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;  // 0 .. 4K-1
  if (k >= 4 * K) return;
  const int D = k - 2 * K;
  uint16_t v = 0;
  if (D != 0) {
    const bool up = D > 0;
    const int I = D - (up ? K : -K);
    if (I >= -imax && I <= imax) {
      const uint32_t w = thr[static_cast<size_t>(t) * stride_words + (I + imax)];
      v = static_cast<uint16_t>(up ? (w >> 16) : (w & 0xFFFFu));
    }
  }
  out[static_cast<size_t>(t) * 4 * K + k] = v;
}

cudaError_t launch_diag_thresholds(const uint32_t* d_thr, int steps, int imax, int stride_words,
                                   int K, uint32_t* d_thr_diag, cudaStream_t st) {
  dim3 grid(4 * K / 256, steps);
  diag_thresholds_kernel<<<grid, 256, 0, st>>>(d_thr, imax, stride_words, K,
                                               reinterpret_cast<uint16_t*>(d_thr_diag));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Initial spin bits.  Philox mode: spin i of replica r is +1 iff bit 15 of its draw at
// step field 0xFFFFFFFF is set.  Host mode: pack int8 +-1 (d_init[R][n], instance 0 only).
// Grid: x = word, y = replica, z = problem.
// ---------------------------------------------------------------------------------------
__global__ void init_bits_kernel(const Problem* __restrict__ probs, const int8_t* __restrict__ init,
                                 uint32_t key_lo, uint32_t key_hi) {
  const Problem& P = probs[blockIdx.z];
  const int r = blockIdx.y * blockDim.y + threadIdx.y;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.R || w >= P.words) return;
  uint32_t bits = 0;
  if (init != nullptr) {
    for (int b = 0; b < 32; ++b) {
      const int i = w * 32 + b;
      if (i < P.n && init[static_cast<size_t>(r) * P.n + i] > 0) bits |= 1u << b;
    }
  } else {
    for (int g = 0; g < 4; ++g) {
      const int i0 = w * 32 + g * 8;
      if (i0 >= P.n) break;
      const PhiloxOut o = philox4x32_10(static_cast<uint32_t>(i0 >> 3), static_cast<uint32_t>(r),
                                        0xFFFFFFFFu, P.q, key_lo, key_hi);
      for (int k = 0; k < 8; ++k) {
        const int i = i0 + k;
        if (i < P.n && ((philox_half(o, k) >> 15) & 1u)) bits |= 1u << (g * 8 + k);
      }
    }
  }
  P.cur_bits[static_cast<size_t>(r) * P.words + w] = bits;
}

cudaError_t launch_init_bits(const Problem* d_probs, int nprob, int maxR, int max_words,
                             const int8_t* d_init, uint32_t key_lo, uint32_t key_hi,
                             cudaStream_t st) {
  dim3 block(8, 32);
  dim3 grid((max_words + 7) / 8, (maxR + 31) / 32, nprob);
  init_bits_kernel<<<grid, block, 0, st>>>(d_probs, d_init, key_lo, key_hi);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Gather copy: every job's block, 16 bytes per thread and step; one CTA per job in turn.
// Results of many instances reach pinned host memory in one launch instead of one copy
// command per instance.
// ---------------------------------------------------------------------------------------
__global__ void gather_copy_kernel(const CopyJob* __restrict__ jobs, int count) {
  for (int j = blockIdx.x; j < count; j += gridDim.x) {
    const uint4* src = static_cast<const uint4*>(jobs[j].src);
    uint4* dst = static_cast<uint4*>(jobs[j].dst);
    const unsigned long long n16 = jobs[j].bytes / 16;
    for (unsigned long long i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
  }
}

cudaError_t launch_gather_copy(const CopyJob* d_jobs, int count, cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  const int blocks = count < 1024 ? count : 1024;
  gather_copy_kernel<<<blocks, 256, 0, st>>>(d_jobs, count);
  return cudaGetLastError();
}

// One word from device memory into mapped pinned host memory (the error-word mirror).
__global__ void mirror_word_kernel(const int* __restrict__ d, int* h) {
  *reinterpret_cast<volatile int*>(h) = *reinterpret_cast<const volatile int*>(d);
}

cudaError_t launch_mirror_word(const int* d, int* h_dev, cudaStream_t st) {
  mirror_word_kernel<<<1, 1, 0, st>>>(d, h_dev);
  return cudaGetLastError();
}

}  // namespace pim
