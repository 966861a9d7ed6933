// Device-visible launch descriptors shared by the runtime and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pim {

// Device error bits, OR-ed into the launch's error word.
enum : int {
  kDevErrTimeout = 1,      // a bounded mbarrier wait gave up
  kDevErrFieldRange = 2,   // a field fell outside the threshold table (cannot happen for
                           // a valid instance; checked so a bad table never reads out of range)
  kDevErrLayout = 4,       // dynamic shared memory not 1024-byte aligned where the kernel's
                           // layout has no room for the alignment pad (the kernel did nothing)
};

// Per-instance parameters of one launch.  All pointers are device pointers.
struct Problem {
  const uint8_t* jimg;     // FP8 E4M3 couplings, npad x npad, 128B-swizzled K-major image
  const uint8_t* jimg4;    // E2M1 image of the coupling-resident large-N variant, or null
  const float* jf;         // float32 row-major n x n (plain path)
  const int8_t* j8;        // int8 row-major n x n (sequential path)
  const int32_t* h;        // int32 bias or nullptr
  const uint32_t* thr;     // decision thresholds [steps][stride_words], entry I + imax
  const uint32_t* thr_diag;  // 16-bit thresholds by D = I + 256 s, [steps][1024], entry D+512
  double* best_E;          // [R]
  double* final_E;         // [R]
  int32_t* best_t;         // [R]
  int32_t* first_hit;      // [R]
  uint32_t* best_bits;     // [R][words]   bit i of word i/32 set <=> spin i = +1
  uint32_t* cur_bits;      // [R][words]   state in / state out
  int n, npad, words;
  int imax, stride_words;
  int R;
  uint32_t q;              // instance counter word of the noise stream
  int has_target;
  long long target;        // first-hit when energy <= target (integer couplings)
  // Real-valued couplings (BF16 operand image in jimg):
  const float* hf;         // float bias or nullptr
  const float* sched_b;    // b_t = fl32(beta_t c), [steps]
  const float* sched_eta;  // eta_t, [steps]
  const float* zlev;       // 4096 noise levels
  float xi;
  int act;                 // 0 tanh, 1 L-level staircase
  int lut_levels;
  double target_f;         // first-hit when energy <= target_f (real couplings)
  int diag_img;            // 1: the FP8 image carries 256 on the diagonal (D = I + 256 s)
  // Mid-N kernel, diagonal-encoded decisions: jimg carries dk on the diagonal (dk = 256:
  // E4M3 image; dk > 256: E5M2 image, e5m2 = 1) and thr_diag holds 16-bit thresholds by
  // D = I + dk s, [steps][4 dk].  dk = 0: general table.
  int dk;
  int e5m2;
  // Diagnostics (real couplings): when set, the kernel writes the FP32 fields
  // I = sum_j J_ij s_j + h_i of the run's first sweep, [R][n] row-major, as its decision
  // uses them.
  float* fields_out;
  // Real couplings in the fixed-point datapath (fix_w > 0; ap_fixed<fix_w, fix_w - fix_f>,
  // values held as integers in units of 2^-fix_f): jimg and jimg_lo are the BF16 images of
  // the high and low parts of Q(c J) (their sum is exact), hf = Q(c h), sched_b = fl32(beta_t)
  // (c is folded into the couplings), and the decision runs on the integer tables below.
  const uint8_t* jimg_lo;
  int fix_w, fix_f;
  const int32_t* fix_tau;  // [2^fix_w]: Q(act(x)) for x = (m - 2^(fix_w-1)) 2^-fix_f
  const int32_t* fix_eta;  // [steps]: Q(eta_t)
  const int32_t* fix_z;    // [4096]: Q(z(key))
  int fix_xi;              // Q(xi)
};

// One block copy of a gather launch: `bytes` (a multiple of 16) from src to dst, both
// 16-byte aligned device-visible addresses (dst may be mapped pinned host memory).
struct CopyJob {
  const void* src;
  void* dst;
  unsigned long long bytes;
};

// One unit of work of the fused sweep kernel: (problem index, first replica).
struct WorkItem {
  int prob;
  int rbase;
};

// Philox4x32-10 round keys for a 64-bit seed: rk[2r] = lo + r * 0x9E3779B9 and
// rk[2r+1] = hi + r * 0xBB67AE85 (mod 2^32), r = 0..9 (the Weyl key schedule).
inline void philox_round_keys(uint64_t seed, uint32_t* rk) {
  uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0;
    rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

struct Launch {
  const Problem* probs;
  const WorkItem* work;
  int nwork;
  int t_begin;
  int sweeps;
  uint32_t key_lo, key_hi;
  uint32_t round_keys[20];  // Philox round keys of (key_lo, key_hi)
  int cont;                // 1: keep previous best / first-hit records
  int stride_words_max;    // largest table stride among the problems (smem sizing)
  int* err;                // device error word
  uint64_t wait_ns;        // limit of every device-side wait (0 = 2 s)
  int inject;              // fault injection for tests: 1 = skip the first field MMA
  unsigned int* next;      // persistent kernels: global unit counter (zeroed per launch)
  // Fused kernel, chunked queue (chunks > 0): every work item's sweeps are cut into
  // `chunks` consecutive shares; persistent CTAs take (chunk, item) segments in the order
  // q = chunk * nwork + item from ready[nwork] and hand an item's state on through
  // ready[item] = chunks done.  ready holds nwork + 1 words, zeroed per launch.
  int chunks;
  unsigned int* ready;
};

// Device-side request queue of the persistent serving kernel (real couplings, n <= 256,
// R <= 128 replicas per request).  The host writes request k into slot k % nslots (its
// descriptor, with the couplings as a BF16 operand image and the bias, and room for the
// results, all in mapped pinned host memory) and then publishes it with a release store of
// tail = k + 1.  Persistent CTAs claim requests in order from the device counter head,
// run them and release-store done[slot] = k + 1 after the results.  A CTA that finds no
// request for idle_ns (a bounded wait), or finds stop set, ends; exit_status records why.
struct ServeQueue {
  const unsigned int* tail;  // mapped host memory: requests published
  const unsigned int* stop;  // mapped host memory: non-zero = end when no request is waiting
  unsigned int* done;        // mapped host memory: [nslots]
  const char* slots;         // mapped host memory: [nslots] slots of slot_bytes, each
                             // beginning with its request's Problem descriptor
  unsigned int* head;        // device memory: requests claimed
  int* exit_status;          // device memory: 0 running, 1 idle limit reached, 2 stopped
  const float* zlev;         // device memory: the 4096 noise levels of every request
  int nslots;
  unsigned long long slot_bytes;
  uint64_t idle_ns;
};

// Launch of the large-N kernel: one instance, all sweeps, cooperative grid of
// (replica tiles) x (nt-spin column blocks).
struct BigLaunch {
  Problem P;
  uint8_t* s_img[2];       // spin images (A operand), ping-pong: tile-major,
                           // [rpad/128][K-blocks][128 rows x 128 B, 128-byte swizzle];
                           // a 128-byte row holds 128 FP8, 64 BF16 or 256 E2M1 spins
  const uint8_t* j4;       // E2M1 coupling image of the coupling-resident variant (else null)
  int stages;              // K-block ring depth and threshold-table placement of the
  int tab_smem;            //   variant's shared-memory plan
  float* energy;           // [3][rpad] rotating per-replica energy accumulators (zeroed);
                           // int32 for integer couplings, float for real couplings
  int nt;                  // output spins per CTA (64 or 128)
  unsigned int* bar;       // grid barrier: 64-bit monotone arrival counter with an abort
                           // bit (zeroed, 8-byte aligned)
  int rbase;               // first replica of this launch
  int rpad;                // replica rows of this launch (multiple of 128)
  int ncb;                 // column blocks = npad / nt
  int t_begin;
  int sweeps;
  int cont;
  uint32_t round_keys[20];
  int* err;
  uint64_t wait_ns;        // limit of every device-side wait (0 = 2 s)
  int inject;              // fault injection for tests: 1 = load nothing in the first sweep
};

// Launch of the sequential (conventional PIM) kernel: one instance, sweeps t_begin ..
// t_begin+sweeps-1 of n single-spin updates each.
struct SeqLaunch {
  Problem P;
  int t_begin;
  int sweeps;
  int cont;
  uint32_t round_keys[20];
};

}  // namespace pim
