// Launch functions of the device kernels (host side, internal to the library).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pim_device.cuh"

struct pim_instance;

namespace pim {

// Byte offset of element (row, k) inside a K-major, 128-byte-swizzled operand image with
// `rows` rows: K-blocks of 128 bytes, each block rows x 128 bytes, 8-row atoms of 1024
// bytes, 16-byte chunk index XOR-ed with (row % 8).
__host__ __device__ inline uint32_t sw128_offset(int row, int k, int rows) {
  const int kb = k >> 7;
  const int chunk = (k & 127) >> 4;
  return static_cast<uint32_t>(kb) * rows * 128u + (row >> 3) * 1024u + (row & 7) * 128u +
         ((chunk ^ (row & 7)) << 4) + (k & 15);
}

// Staging (once per instance).
// diag != 0 puts that value on the diagonal of the image (inside n x n); e5m2 selects the
// E5M2 element format (default E4M3).  The image is a sequence of 16 KB blocks of 128 rows x
// one 128-byte K-block: K-block-major ([kb][npad / 128 row blocks]) by default, chunk-major
// ([npad / 128 row blocks][kb]: the K-blocks of 128 output rows contiguous) when
// chunk_major is set (npad a multiple of 128).
cudaError_t launch_stage_fp8_image(const int8_t* d_J, int n, int npad, int diag, uint8_t* d_img,
                                   cudaStream_t st, bool e5m2 = false, bool chunk_major = false);
cudaError_t launch_stage_f32(const int8_t* d_J, int n, float* d_jf, cudaStream_t st);
// E2M1 image of the coupling-resident large-N variant, npad x npad / 2 bytes (npad a
// multiple of 256; couplings in {0, +-1, +-2, +-3, +-4, +-6}).
cudaError_t launch_stage_fp4_image(const int8_t* d_J, int n, int npad, uint8_t* d_img,
                                   cudaStream_t st);

// Decision thresholds for all steps: tau [steps][2*imax+1], eta [steps], z [4096].
cudaError_t launch_thresholds(const float* d_tau, const float* d_eta, const float* d_z,
                              float xi, int steps, int imax, int stride_words,
                              uint32_t* d_thr, cudaStream_t st);

// Re-index the thresholds by D = I + K s (D = -2K..2K-1, 16-bit entries, [steps][4K]); needs
// imax < K, K a power of two >= 64.
cudaError_t launch_diag_thresholds(const uint32_t* d_thr, int steps, int imax, int stride_words,
                                   int K, uint32_t* d_thr_diag, cudaStream_t st);

// Copies one int from device memory to mapped pinned host memory (h_dev: its device address).
cudaError_t launch_mirror_word(const int* d, int* h_dev, cudaStream_t st);

// Copies every job's block (jobs in device memory).
cudaError_t launch_gather_copy(const CopyJob* d_jobs, int count, cudaStream_t st);

// Initial spin bits: from Philox (d_init == nullptr) or from int8 +-1 spins [R][n].
cudaError_t launch_init_bits(const Problem* d_probs, int nprob, int maxR, int max_words,
                             const int8_t* d_init, uint32_t key_lo, uint32_t key_hi,
                             cudaStream_t st);

// Fused tensor-core sweep kernel (n <= 256): `blocks` CTAs, one per work item, or, when
// L.chunks > 0, persistent CTAs that take (chunk, item) segments from a queue.
cudaError_t launch_sweep_tc(const Launch& L, int npad_max, int blocks, cudaStream_t st,
                            bool diag);
int sweep_tc_smem_bytes(int npad, int stride_words_max);

// Real-valued couplings (BF16 operands, FP32 decision), n <= 256.
cudaError_t launch_sweep_float(const Launch& L, int npad, int blocks, cudaStream_t st);
int sweep_float_smem_bytes(int npad);
// BF16 image: the same block structure as the FP8 image (16 KB blocks of 128 rows x one
// 128-byte K-block of 64 values), K-block-major or chunk-major.
cudaError_t launch_stage_bf16_image(const uint16_t* d_J, int n, int npad, uint8_t* d_img,
                                    cudaStream_t st, bool chunk_major = false);
// Persistent serving variant of the real-valued kernel: `blocks` CTAs take requests from Q
// until it stays empty for Q.idle_ns or Q.stop is set (L: sweeps, round keys, waits).
cudaError_t launch_serve_float(const Launch& L, const ServeQueue& Q, int npad, int blocks,
                               cudaStream_t st);

// Large-N kernel (n > 256): cooperative launch of `blocks` = (rpad/128) * ncb CTAs, each
// computing nt (64 or 128) output spins.  Operand variants (op):
//   kBigFp8   FP8 E4M3 spins and couplings, both streamed every sweep (integer couplings);
//   kBigBf16  BF16 spins and couplings, FP32 decision (real couplings);
//   kBigFp4   coupling-resident: the CTA's 64 coupling rows stay in shared memory as packed
//             E2M1 for the whole launch and only E2M1 spins stream (integer couplings in
//             {0, +-1, +-2, +-3, +-4, +-6}, npad <= 4096, nt = 64).
enum BigOp : int { kBigFp8 = 0, kBigBf16 = 1, kBigFp4 = 2 };
// Shared-memory plan of a variant: ring depth, whether the step's threshold table is staged
// in shared memory, dynamic shared-memory bytes.  ok = false when the variant does not fit.
struct BigSmem {
  bool ok = false;
  int stages = 0;
  int tab_smem = 0;
  int bytes = 0;
};
BigSmem sweep_big_smem(int nt, int op, int npad, int stride_words);
// L.stages / L.tab_smem must hold sweep_big_smem's plan for (nt, op, P.npad, P.stride_words).
cudaError_t launch_sweep_big(const BigLaunch& L, int nt, int op, int blocks, cudaStream_t st);
// Co-resident CTAs on the current device for that plan (0 on error or when it does not fit).
int sweep_big_max_blocks(int nt, int op, int npad, int stride_words);

// Persistent mid-N kernel (integer couplings, npad <= 1024): `blocks` CTAs take the units
// of L.work from the counter L.next (zeroed by the launch).
// diag: every unit has P.dk > 0 (diagonal-encoded variant), else none has.
cudaError_t launch_sweep_mid(const Launch& L, int blocks, cudaStream_t st, bool diag);
int sweep_mid_max_blocks();
int sweep_mid_max_npad();

// Sequential (conventional PIM) kernel: one warp per replica, integer couplings.
cudaError_t launch_sequential(const SeqLaunch& L, cudaStream_t st);
int sequential_smem_bytes(int n);

// Plain FP32 comparator path: per sweep one field GEMM and one update kernel.
cudaError_t launch_ref_anneal(const Problem* h_probs, const Problem* d_probs, int nprob,
                              int t_begin, int sweeps, uint32_t key_lo, uint32_t key_hi,
                              int cont, float* d_S, float* d_I, int* d_err, cudaStream_t st);

// Sets the thread-local message returned by pim_last_error.
void set_last_error(const char* msg);

// Device arrays of a real-coupling instance's schedule (b_t = fl32(beta_t c), eta_t, the
// 4096 noise levels) with its xi and activation, for the serving kernel; PIM_ERR_STATE
// without a real-valued schedule.
int schedule_device_arrays(const pim_instance* inst, const float** b_t, const float** eta,
                           const float** zlev, float* xi, int* act, int* lut_levels);

}  // namespace pim
