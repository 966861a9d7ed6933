/*
 * pim.h -- C ABI of the GB300 PIMI sweep library.
 *
 * The library runs the probabilistic Ising machine with inertia (PIMI) of
 * arXiv 2604.17109: fully parallel, synchronous spin updates
 *
 *     I_i(t)   = sum_j J_ij s_j(t) + h_i                                  (Eq. 2)
 *     s_i(t+1) = sign[ tanh(beta(t) I_i(t)) + xi s_i(t) + eta(t) N(0,1) ]  (Eq. 4)
 *
 * over many replicas ("trials", Box 1) and many instances at once, tracking for every
 * replica the Ising energy H(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i (Eq. 1) of
 * every visited state, the best state, and the first step whose energy reaches a target
 * (success criterion of the supplementary CCTS section).
 *
 * Conventions shared by every entry point
 *  - Every call returns a status (pim_status); nothing throws across the ABI.  On error
 *    pim_last_error() returns a thread-local message describing the last failure.
 *  - Host buffers passed in are only read during the call; the library deep-copies what
 *    it keeps.  The caller owns every buffer it passes and every output buffer.
 *  - Device state (staged couplings, schedules, spins, results) is owned by the
 *    pim_instance and freed by pim_destroy.
 *  - Spin arrays on the host are int8 values -1/+1, row-major (replica, spin).
 *  - Annealing calls are asynchronous on the CUDA stream passed as `cuda_stream`
 *    (a cudaStream_t; NULL = the legacy default stream).  Result getters synchronise on
 *    the instance's last run before copying (an instance annealed in a batch completes
 *    with the whole batch: one completion event per run).
 *  - pim_create uploads and stages its inputs asynchronously on library-owned streams;
 *    the first anneal of the instance waits for them on the device (the host does not).
 *  - One GPU: all device memory lives on the device that is current when pim_create
 *    runs; later calls must run with that device current.
 */
#ifndef PIM_H
#define PIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum pim_status {
  PIM_OK = 0,
  PIM_PENDING = 1,          /* pim_poll: the submitted work has not finished yet */
  PIM_ERR_INVALID = -1,     /* bad argument: sizes, asymmetric J, non-zero diagonal, ... */
  PIM_ERR_NOMEM = -2,       /* device or host allocation refused */
  PIM_ERR_CUDA = -3,        /* a CUDA runtime call failed (message has the CUDA error) */
  PIM_ERR_STATE = -4,       /* call out of order (no schedule, no previous state, ...) */
  PIM_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  PIM_ERR_UNSUPPORTED = -6  /* valid request that this build does not implement */
} pim_status;

/* Element type of the host coupling matrix passed to pim_create. */
typedef enum pim_j_type {
  PIM_J_INT8 = 0,  /* int8, integer couplings |J_ij| <= 16 (held exactly as FP8 E4M3) */
  PIM_J_FP32 = 1,  /* float32 real couplings, rounded to BF16 for the tensor cores */
  PIM_J_FP64 = 2   /* float64 real couplings, rounded to BF16 for the tensor cores */
} pim_j_type;

/* Noise term of the update rule. */
typedef enum pim_noise {
  PIM_NOISE_GAUSS = 0,   /* eta(t) N(0,1), Eq. 4 */
  PIM_NOISE_UNIFORM = 1  /* eta(t) U(-1,1), Eq. 3 */
} pim_noise;

/* Activation applied to beta(t) I_i(t). */
typedef enum pim_act {
  PIM_ACT_TANH = 0,  /* tanh, Eq. 4 */
  PIM_ACT_LUT = 1    /* L-level staircase of Algorithm "LUT-based tanh approximation" */
} pim_act;

/* Flags of pim_anneal / pim_anneal_batch. */
typedef enum pim_flags {
  PIM_CONTINUE = 1,     /* start from the instance's current state and keep its best /
                           first-hit records (resume); replicas must equal the last run's */
  PIM_PATH_FP32REF = 2, /* run the plain FP32 two-kernels-per-sweep comparator path instead
                           of the fused tensor-core sweep kernel (same decisions) */
  PIM_PATH_MID = 4,     /* put every integer instance with n <= 1024 on the persistent mid-N
                           kernel (same decisions; for tests and tuning) */
  PIM_PATH_BIG = 8,     /* put every instance with n > 256 on the large-N cooperative kernel
                           (same decisions; for tests and tuning).  Without either flag the
                           library picks the kernel of each instance from its cost model. */
  PIM_RESULTS_TO_HOST = 16, /* after the run, copy every instance's results (all of what
                           pim_energies, pim_best_state and pim_final_state return) into
                           library-owned pinned host memory on the same stream, so those
                           getters wait for the run and read host memory instead of issuing
                           a synchronous copy each.  Costs R * (24 + 8 * words) bytes of
                           device-to-host traffic per instance and run. */
  PIM_PATH_FP8 = 32     /* FP8 E4M3 operands only: no E2M1 coupling-resident variant of the
                           large-N kernel, which applies to integer couplings in {0, +-1, +-2,
                           +-3, +-4, +-6} with 256 < n <= 4096; same decisions, for tests and
                           tuning.  Without it the library picks the variant from its cost
                           model or measured times. */
} pim_flags;

typedef struct pim_instance pim_instance;

/*
 * pim_create -- stage one Ising instance (J, h) on the device.
 * Defines the problem of Eq. 1 / Eq. 2 (Ising Hamiltonian and local field).
 *   out      receives the new handle (set to NULL on failure).
 *   n        number of spins, 1 <= n <= 8192; the fused kernels serve n <= 256, the
 *            large-N kernel n > 256 (integer and real couplings alike).  For integer J with
 *            256 < n <= 4096 and every entry in {0, +-1, +-2, +-3, +-4, +-6} the instance
 *            also keeps an E2M1 (FP4) copy of J, n_pad^2 / 2 bytes, for the large-N
 *            kernel's coupling-resident variant (exact: those integers are E2M1 values).
 *   j_type   element type of J (pim_j_type).
 *   J        host, row-major n x n; must be symmetric with a zero diagonal.
 *   h        host bias, n entries: int32 when j_type == PIM_J_INT8, else the float type
 *            of J (kept as float32); NULL means h = 0.
 *            Real couplings are rounded to the nearest BF16 value (ties to even); fields
 *            accumulate in FP32 and the decision of Eq. 4 is evaluated in FP32 on the device
 *            (tanhf), so results agree with a float64 evaluation within FP32 error rather
 *            than bit for bit.
 *   scale_c  coupling scale c > 0 applied after the multiply-accumulate (the paper's
 *            2/sqrt(N) for Max-Cut, 1/sqrt(N) for SK-1): the activation sees beta_t*c*I.
 *            Energies are reported in unscaled units of J and h.
 * Errors: PIM_ERR_INVALID (n out of range, J asymmetric, diagonal non-zero, |J| > 16 for
 *         integer J, non-finite values or |J| > 1e30, scale_c <= 0 or not finite; the first
 *         offending entry in row-major order is named), PIM_ERR_NOMEM, PIM_ERR_CUDA.
 */
int pim_create(pim_instance** out, int n, int j_type, const void* J, const void* h,
               double scale_c);

/*
 * pim_set_schedule -- annealing schedule of Eq. 4 (beta(t), eta(t), xi).
 * Schedule section of the supplementary PIMI implementation (inverse-temperature,
 * noise and self-alignment paragraphs); the schedule values are inputs here.
 *   steps      number of schedule entries T >= 1; anneals use steps [t_begin, t_end).
 *   beta, eta  host float arrays of `steps` entries; beta >= 0, eta >= 0, finite.
 *   xi         inertia (self-alignment) strength, finite, >= 0.
 *   noise_kind pim_noise;  act_kind pim_act;  lut_levels L >= 2 (used by PIM_ACT_LUT).
 * Builds, for every step t, the exact decision thresholds of the float32 rule
 *   delta = (tau_t(I) + xi s) + eta_t z(m),  s' = +1 iff delta >= 0,
 * with tau_t(I) = fl32(tanh(fl32(beta_t c) * I)) and z(m) one of 4096 noise levels
 * selected by a 12-bit key m from the Philox stream.  Threshold tables are shared
 * between instances with the same (schedule, c, field range).
 * Errors: PIM_ERR_INVALID, PIM_ERR_NOMEM, PIM_ERR_CUDA.
 */
int pim_set_schedule(pim_instance* inst, int steps, const float* beta, const float* eta,
                     float xi, int noise_kind, int act_kind, int lut_levels);

/*
 * pim_set_schedule_fixed -- as pim_set_schedule, with the decision of Eq. 4 evaluated in
 * the fixed-point datapath of the supplementary quantization section:
 * ap_fixed<total_bits, int_bits, AP_TRN_ZERO, AP_SAT> (int_bits include the sign; each
 * value truncated toward zero to a multiple of 2^-(total_bits - int_bits), then saturated).
 * Order of the datapath (every intermediate quantized, Q = that format):
 *   u = Q(c I)  (normalisation after the multiply-accumulate),  x = Q(beta_t u),
 *   tau = Q(tanh(x)) or Q(L-level staircase(x)),  a = Q(tau + s Q(xi)),
 *   n = Q(Q(eta_t) Q(z)),  s' = +1 iff Q(a + n) >= 0.
 * The paper uses <4,2> for Max-Cut / SK and <16,4> for MIMO.
 * Integer couplings: the decision stays monotone in the noise key, so the same kernels run
 * it from exact key thresholds, built on the host.
 * Real couplings (n <= 128, total_bits <= 16; the MIMO pipeline of the paper): the couplings
 * and bias are stored in the format too, with the scale folded in: J_q = Q(c J), h_q = Q(c h)
 * (values of order one, as the FPGA holds them); the field I = J_q s + h_q is accumulated
 * exactly and u = Q(I).  The device holds J_q as two BF16 images whose sum is exact and
 * evaluates the datapath above on integers in units of 2^-(total_bits - int_bits), with
 * tau read from a table of Q(tanh(x)) (or the staircase) over every representable x.
 * Energies and targets of such a run are those of the quantized, scaled problem
 * -1/2 s^T J_q s - h_q^T s (exact).
 *   total_bits in [2, 32], int_bits in [1, total_bits].
 * Errors: PIM_ERR_INVALID, PIM_ERR_UNSUPPORTED (real couplings with n > 128 or
 *         total_bits > 16, or a row of J_q whose exact sum needs more than 2^24 units),
 *         PIM_ERR_NOMEM, PIM_ERR_CUDA.
 */
int pim_set_schedule_fixed(pim_instance* inst, int steps, const float* beta, const float* eta,
                           float xi, int noise_kind, int act_kind, int lut_levels, int total_bits,
                           int int_bits);

/*
 * pim_anneal -- run sweeps t_begin .. t_begin+sweeps-1 of Eq. 4 on `replicas` replicas.
 * Box 1 (PIMI loop) and the supplementary algorithm "Fully unrolled PIMI update".
 *   replicas      R >= 1 independent trials.
 *   t_begin       first schedule step (0 for a fresh run); t_begin + sweeps <= steps.
 *   sweeps        number of synchronous sweeps (>= 0).
 *   seed          64-bit Philox key; draws use counter (i>>3, r, t, instance_id).
 *   instance_id   counter word that separates instances sharing a seed.
 *   init_spins    host int8 R x n of -1/+1, or NULL: Philox initial spins (bit 15 of the
 *                 draw at step field 0xFFFFFFFF).  Ignored with PIM_CONTINUE.
 *   target_energy first-hit threshold: records the first t with H(s(t)) <= target;
 *                 NaN disables it.
 *   flags         pim_flags.
 *   cuda_stream   cudaStream_t to enqueue on (NULL = legacy default stream).
 * Records for every replica the minimum of H over s(t_begin) .. s(t_begin+sweeps)
 * (earliest wins ties), its step and state, the first-hit step and the final state.
 * Errors: PIM_ERR_INVALID, PIM_ERR_STATE (no schedule; CONTINUE without a previous run
 *         of the same R), PIM_ERR_UNSUPPORTED, PIM_ERR_NOMEM, PIM_ERR_CUDA.
 */
int pim_anneal(pim_instance* inst, int replicas, int t_begin, int sweeps, uint64_t seed,
               uint32_t instance_id, const int8_t* init_spins, double target_energy,
               int flags, void* cuda_stream);

/*
 * pim_anneal_batch -- one launch over many instances (the kernels of the paper process
 * instances back to back; here all of them share one grid).
 *   insts         `count` handles, each with a schedule set.
 *   replicas      count entries, R_q >= 1.
 *   t_begin, sweeps, seed, flags, cuda_stream  as pim_anneal, common to all instances.
 *   instance_ids  count counter words, or NULL for 0 .. count-1.
 *   targets       count first-hit targets, or NULL for none.
 * Initial spins come from Philox (or the previous state with PIM_CONTINUE).
 * Errors: as pim_anneal.
 */
int pim_anneal_batch(pim_instance* const* insts, int count, const int* replicas, int t_begin,
                     int sweeps, uint64_t seed, const uint32_t* instance_ids,
                     const double* targets, int flags, void* cuda_stream);

/*
 * Batch plans -- many instances of uneven n and replica count in one persistent,
 * CUDA-graph-replayed launch sequence.  This is the device-side counterpart of the
 * supplementary "Kernel execution" and "Host-side task scheduling" subsections (one kernel
 * processes instance after instance without idling, fed by a scheduler): here the
 * instances' (instance, replica panel) units are taken by persistent CTAs from a device
 * counter, with no host work between instances.
 *
 * pim_batch_create builds, once, everything a run of the batch needs: the kernel of each
 * instance (fused n <= 256, persistent mid-N n <= 1024 integer, large-N cooperative; chosen
 * by the library's time model unless PIM_PATH_MID / PIM_PATH_BIG force it), the problem
 * descriptors and unit lists on the device, the result buffers of every instance and the
 * large-N scratch.
 *   out           receives the handle (NULL on failure).
 *   insts, count  instances with schedules; they must outlive the batch and keep their
 *                 schedule and replica counts while it exists (pim_batch_run checks).
 *   replicas      count entries >= 1; instance_ids (NULL = 0..count-1) and targets (NULL
 *                 or NaN = none) as in pim_anneal_batch.
 *   flags         0, PIM_PATH_MID or PIM_PATH_BIG, each optionally with PIM_PATH_FP8.
 * pim_batch_run runs sweeps t_begin .. t_begin+sweeps-1 of every instance, asynchronously on
 * `cuda_stream`: the first run with given (t_begin, sweeps, seed, run_flags) captures the
 * batch's launches into a CUDA graph (later changes update the instantiated graph in
 * place) and every run replays it with one cudaGraphLaunch.  run_flags: PIM_CONTINUE and / or
 * PIM_RESULTS_TO_HOST.
 * Results are read with the per-instance getters.  A batch whose launches cannot be
 * captured runs them directly instead (pim_batch_info reports which).
 * pim_batch_info: kernel launches per run and whether runs replay a graph (1) or not (0).
 * pim_batch_route: the kernel instance `index` runs on -- *kernel 0 fused (n <= 256), 1
 * persistent mid-N, 2 large-N -- and, for the large-N kernel, its tile width (64 or 128
 * output spins per CTA) and operand variant (0 FP8 E4M3 streamed, 1 BF16 streamed, 2 E2M1
 * with the couplings resident in shared memory); both 0 / -1 otherwise.  Any output pointer
 * may be NULL.
 * Errors: PIM_ERR_INVALID, PIM_ERR_STATE (instance changed since creation, CONTINUE without
 *         a previous run), PIM_ERR_UNSUPPORTED, PIM_ERR_NOMEM, PIM_ERR_CUDA.
 *
 * Autotuning (pim_autotune mode 1, the default): pim_batch_create first times, on the
 * batch's own staged instances and with result buffers of its own, every shape class it has
 * not met before on this device -- the fused kernel per (npad, decision path) unit, the
 * persistent mid-N kernel per unit, and the large-N kernel per (operand variant, npad,
 * replica tiles) instance sweep at both tile widths (64 and 128 spins; the E2M1
 * coupling-resident variant at 64) -- a few sweeps each, and keeps the
 * times in a process-wide cache keyed by device name and class.  The router and the
 * large-N tile plan of every later run (pim_anneal, pim_anneal_batch, batch plans) use the
 * measured times where the cache has them and the analytic model elsewhere.  All candidate
 * kernels give identical results, so tuning changes speed only.
 */
typedef struct pim_batch pim_batch;
int pim_batch_create(pim_batch** out, pim_instance* const* insts, int count, const int* replicas,
                     const uint32_t* instance_ids, const double* targets, int flags);
int pim_batch_run(pim_batch* batch, int t_begin, int sweeps, uint64_t seed, int run_flags,
                  void* cuda_stream);
int pim_batch_info(const pim_batch* batch, int* kernel_launches, int* uses_graph);
int pim_batch_route(const pim_batch* batch, int index, int* kernel, int* tile_width, int* operand);
void pim_batch_destroy(pim_batch* batch);

/*
 * pim_autotune -- how kernels and large-N tile widths are chosen (process-wide; the paper's
 * counterpart is the host-side task scheduling it replaces).  mode 0: the analytic cost model
 * only; mode 1 (default): pim_batch_create measures new shape classes first (see above).
 * When the environment variable PIM_TUNE_CACHE names a file, measured times are appended
 * to it and read back by later processes.
 * Errors: PIM_ERR_INVALID (mode not 0 or 1).
 *
 * pim_tune_report -- the measured times, one line per shape class:
 * "<device>|<kernel>|<a>|<b>|<c>|<d> <microseconds>" with kernel fused (a = npad,
 * b = 1 diagonal-encoded; us per unit sweep, two CTAs per SM), mid (a = npad, b = decision
 * path; us per unit sweep, one CTA per SM) or big (a = operand variant 0 FP8, 1 BF16, 2
 * E2M1, b = npad, c = replica tiles, d = tile width; us per instance sweep).  Writes at most cap bytes (NUL-terminated) to
 * out (may be NULL) and the size needed to *needed (may be NULL).
 */
int pim_autotune(int mode);
int pim_tune_report(char* out, size_t cap, size_t* needed);

/*
 * Measurement probes (no anneal; they synchronise the device): the rates of the units the
 * sweep kernels are bound by on the current GPU, for the roofline fractions the benchmark
 * reports beside the prescribed peaks.
 * pim_probe_tensor -- one CTA per SM issues `iters` tcgen05.mma of M = 128, N = 256 back to
 *   back on shared-memory operands into one TMEM accumulator; *tflops = dense rate over all
 *   SMs.  kind 0: FP8 E4M3 (kind::f8f6f4, K = 32), 1: BF16 (kind::f16, K = 16), 2: E2M1
 *   block-scaled with unit scale factors (kind::mxf4, K = 64) -- the operand kinds of the
 *   sweep kernels.  Keep iters x 1 MFLOP within a second of work (e.g. 20000).
 * pim_probe_ingest -- one CTA per SM streams `iters` cp.async.bulk copies of `bytes` (a
 *   multiple of 16, at most 32768) from an L2-resident source through a 4-stage ring, no
 *   compute; *gbs_per_sm = bytes per nanosecond of the slowest SM.  shared 0: each SM reads
 *   its own 256 KB; shared 1: all SMs read the same 256 KB.
 * Errors: PIM_ERR_INVALID (arguments), PIM_ERR_NOMEM, PIM_ERR_CUDA, PIM_ERR_TIMEOUT (a
 *   bounded wait of the probe gave up).
 */
int pim_probe_tensor(int kind, int iters, double* tflops);
int pim_probe_ingest(int bytes, int iters, int shared, double* gbs_per_sm);

/*
 * pim_anneal_sequential -- conventional PIM with sequential updates (Eq. 3; Box 1, orange
 * path), the baseline of the fully parallel loop, on integer couplings.
 *   Sweep k (schedule entry k) updates spins i = 0 .. n-1 one after another, each from the
 *   field of the current state, with beta_k, eta_k, the instance's xi (xi = 0 gives Eq. 3;
 *   xi > 0 adds the inertia term of Eq. 4), noise kind and activation, and the draw of
 *   counter (i>>3, r, k, instance_id): the same numbers the parallel loop draws in sweep k.
 *   Energies are evaluated on the state at the start of every sweep and on the final
 *   state; best / first-hit / final records are read with the usual getters.
 *   replicas, t_begin, sweeps, seed, instance_id, init_spins, target_energy, cuda_stream
 *   as pim_anneal; flags: PIM_CONTINUE and / or PIM_RESULTS_TO_HOST.  One warp per replica.
 * Errors: PIM_ERR_INVALID, PIM_ERR_STATE, PIM_ERR_UNSUPPORTED (real couplings, n too large
 *         for shared memory), PIM_ERR_NOMEM, PIM_ERR_CUDA.
 */
int pim_anneal_sequential(pim_instance* inst, int replicas, int t_begin, int sweeps,
                          uint64_t seed, uint32_t instance_id, const int8_t* init_spins,
                          double target_energy, int flags, void* cuda_stream);

/*
 * MIMO detection (supplementary sections on MIMO detection and on the Delta-Ising MIMO
 * formulation).  Complex arrays are interleaved (re, im) doubles; H is row-major nr x nt.
 *
 * pim_mimo_formulate -- FP64 host formulation of one uplink detection problem
 * y = H x + n as the Ising instance of the residual around the hard-sliced MMSE estimate:
 *   x_mmse = slice((H^H H + mmse_reg I)^-1 H^H y)              (MMSE baseline section)
 *   real equivalent Hr = [[Re H, -Im H], [Im H, Re H]], yr = [Re y; Im y]
 *   d = u - x_mmse = T s with T = [I, I] for 4-/16-QAM (corrections {-2, 0, 2}) and
 *   T = [2I, I, I] for 64-QAM; n = (2 or 3) * 2 nt spins, spin k = block b, component m
 *   J = -2 zeroDiag(T^T Hr^T Hr T),  h = 2 T^T Hr^T (yr - Hr x_mmse)
 * so that the library energy -1/2 s^T J s - h^T s equals ||y - H(x_mmse + T s)||^2 up to a
 * constant (the paper's form -h^T s - s^T J_p s with J = 2 J_p).
 *   J: caller-allocated n x n, h: n, x_mmse: nt complex (slicing onto the square-QAM
 *   levels -L+1, .., L-1).  qam in {4, 16, 64}; mmse_reg > 0 (the paper prints
 *   1 / (Es/N0)).
 * pim_mimo_reconstruct -- x_hat = slice(x_mmse + T s) for spins s (n int8 +-1), nt complex
 *   out (reconstruction section).
 * pim_mimo_formulate_depth / pim_mimo_reconstruct_depth -- the same with the correction
 *   set chosen by `depth` (spins per real symbol component): 2 = T = [I, I] (corrections
 *   {-2, 0, 2}), 3 = T = [2I, I, I] (corrections {-4, .., 4}), 0 = the constellation's
 *   default above; n = depth * 2 nt.  The paper prints both sets and leaves the choice per
 *   constellation open ("higher-order constellations require larger sets").
 * Errors: PIM_ERR_INVALID (sizes, constellation, depth, non-positive-definite MMSE system).
 */
int pim_mimo_formulate(int nt, int nr, int qam, const double* H, const double* y,
                       double mmse_reg, double* J, double* h, double* x_mmse);
int pim_mimo_reconstruct(int nt, int qam, const double* x_mmse, const int8_t* spins,
                         double* x_hat);
int pim_mimo_formulate_depth(int nt, int nr, int qam, int depth, const double* H,
                             const double* y, double mmse_reg, double* J, double* h,
                             double* x_mmse);
int pim_mimo_reconstruct_depth(int nt, int qam, int depth, const double* x_mmse,
                               const int8_t* spins, double* x_hat);

/*
 * MIMO-detection server -- the real-time request loop of the supplementary "Kernel
 * execution" and "Host-side task scheduling" subsections on one GPU: continuous batching
 * with memory admission.  A dispatcher thread admits queued requests while one of
 * `max_inflight` stream slots is free and the device bytes of the admitted requests stay
 * within `mem_budget`, formulates each (pim_mimo_formulate), stages it as a BF16 instance,
 * and launches every request admitted at that moment as one batch (at most `max_batch`),
 * so requests that arrive while others run are admitted as slots and memory free up and
 * their work overlaps on the device.  A completion thread selects each request's replica
 * of lowest reported best energy (ties: lowest index), evaluates that state's FP64 energy,
 * reconstructs x_hat and records the latency (submit -> result available).
 * Device-side request queue (device_queue = 1; n <= 256 spins, replicas <= 128): instead of
 * batched launches, one persistent kernel (min(SMs, max_batch x max_inflight) CTAs) takes
 * the requests from a queue in mapped pinned host memory.  The dispatcher formulates a
 * request, writes its BF16 coupling image, bias and descriptor into the next free slot
 * (2 x CTAs slots) and publishes it with a release store of the queue's tail; a CTA claims
 * it from a device counter, runs the whole anneal (all replicas in one CTA) and writes the
 * results into the slot before a done flag, which the completion thread polls.  The
 * kernel's wait for requests is bounded: after idle_s without one it ends (no GPU time
 * spent idling), and the server launches it again for the next request.
 * Every request uses the server's schedule (beta, eta, xi,
 * scale_c, Gaussian noise, tanh), `replicas`, `sweeps`, `seed`, and its request_id as the
 * instance counter word, so its result does not depend on what it was batched with.
 */
typedef struct pim_mimo_server_config {
  int nt, nr, qam;        /* system size and constellation (4, 16, 64) */
  int replicas, sweeps;   /* trials and PIMI steps per request */
  const float* beta;      /* [sweeps], copied at creation */
  const float* eta;       /* [sweeps], copied at creation */
  float xi;               /* inertia */
  double scale_c;         /* coupling scale applied to the accumulated field */
  uint64_t seed;          /* Philox key of every request */
  int max_batch;          /* requests per launch, >= 1 */
  int max_inflight;       /* launches in flight (streams), >= 1 */
  size_t mem_budget;      /* device bytes admitted requests may hold (raised to one request) */
  int device_queue;       /* 0: host batching as above; 1: device-side request queue (below) */
  double idle_s;          /* device queue: the serving kernel ends after this long without a
                             request (> 0; it is relaunched when requests come again) */
} pim_mimo_server_config;
typedef struct pim_mimo_server pim_mimo_server;
int pim_mimo_server_create(pim_mimo_server** out, const pim_mimo_server_config* cfg);
/* Copies H (nr x nt complex) and y (nr complex); returns a ticket immediately. */
int pim_mimo_server_submit(pim_mimo_server* server, const double* H, const double* y,
                           double mmse_reg, uint32_t request_id, uint64_t* ticket);
/* PIM_PENDING, PIM_OK or the request's error. */
int pim_mimo_server_poll(pim_mimo_server* server, uint64_t ticket);
/* Waits up to timeout_s; on PIM_OK writes x_hat (nt complex), the FP64 energy of the chosen
   replica and the latency in microseconds, and forgets the ticket; PIM_PENDING on timeout. */
int pim_mimo_server_result(pim_mimo_server* server, uint64_t ticket, double timeout_s,
                           double* x_hat, double* best_energy, double* latency_us);
/* Completed requests, latency percentiles (us), mean requests per launch, peak admitted
   bytes; returns the first error a batch met (PIM_OK if none). */
int pim_mimo_server_stats(pim_mimo_server* server, uint64_t* completed, double* p50_us,
                          double* p99_us, double* mean_batch, size_t* peak_bytes);
/* Native load driver: submits request k (H_all + k nr nt, y_all + k nr complex) at
   arrival_us[k] microseconds after the call starts, waits for all, and writes each
   request's x_hat (nt complex), energy and latency (each output may be NULL). */
int pim_mimo_server_replay(pim_mimo_server* server, int count, const double* H_all,
                           const double* y_all, const double* reg_all,
                           const double* arrival_us, double* x_hat_all,
                           double* best_energy_all, double* latency_us_all);
/* Device queue only: waits up to timeout_s for the serving kernel to end with no request
   left in flight.  PIM_ERR_TIMEOUT: it ended because its bounded wait for requests ran out
   (idle_s); PIM_OK: it ended on a stop; PIM_PENDING: still running at timeout;
   PIM_ERR_UNSUPPORTED: the server batches on the host (device_queue = 0). */
int pim_mimo_server_idle_wait(pim_mimo_server* server, double timeout_s);
/* Stops admitting, finishes the batches in flight, drops requests still queued and frees
   the server; no other call on the server may run concurrently with it. */
void pim_mimo_server_destroy(pim_mimo_server* server);

/*
 * pim_results_dev -- the last anneal's records copied device to device, stream-ordered
 * after it on `cuda_stream` (the host does not wait): for callers that keep results on
 * the GPU (a serving loop, a framework's tensors).  Device pointers, each may be NULL:
 *   best_E, final_E       R doubles;  best_t, first_hit_t  R int32;
 *   best_bits, final_bits R x pim_state_words(inst) uint32 words, bit i of word i/32 set
 *                         <=> spin i = +1 (bits past n are 0).
 * pim_state_words -- words per replica of the bit arrays (0 for NULL).
 * Errors: PIM_ERR_INVALID, PIM_ERR_STATE (no anneal has run), PIM_ERR_CUDA.
 */
int pim_results_dev(pim_instance* inst, double* best_E, int32_t* best_t, int32_t* first_hit_t,
                    double* final_E, uint32_t* best_bits, uint32_t* final_bits, void* cuda_stream);
int pim_state_words(const pim_instance* inst);

/*
 * pim_fields -- diagnostic read-out of the local fields of Eq. 2, I_i = sum_j J_ij s_j + h_i,
 * exactly as the sweep kernel of a real-coupling instance forms them (J rounded to BF16,
 * FP32 accumulation in tensor memory, + h in FP32) and feeds them to its Eq. 4 decision.
 * It runs sweep 0 of the instance's schedule from the given states on the kernel the instance
 * is routed to (the fused real-valued kernel for n <= 256, the large-N kernel otherwise) with
 * the kernel's field capture switched on, then returns the captured fields.  This is how the
 * BF16 field error against a float64 evaluation is measured.
 *   inst        real-coupling instance (PIM_J_FP32 / PIM_J_FP64) with a schedule.
 *   replicas    R >= 1 states.
 *   spins       host int8 R x n of -1/+1: s for each replica.
 *   fields      host float32 R x n output, row-major (replica, spin).
 *   flags       0 or PIM_PATH_BIG (no effect for n <= 256).
 *   cuda_stream cudaStream_t; the call returns when the fields are in `fields`.
 * The instance's records (pim_energies, ...) afterwards are those of this one-sweep run.
 * Errors: PIM_ERR_INVALID, PIM_ERR_STATE (no schedule), PIM_ERR_UNSUPPORTED (integer couplings:
 *         their fields are exact integers), PIM_ERR_NOMEM, PIM_ERR_CUDA.
 */
int pim_fields(pim_instance* inst, int replicas, const int8_t* spins, float* fields, int flags,
               void* cuda_stream);

/* pim_sync -- block until the instance's last anneal has finished.
 * Errors: PIM_ERR_CUDA, PIM_ERR_TIMEOUT (a device-side bounded wait gave up).
 * Device-side error bits are kept per device and cleared when reported.  Every run copies
 * them into host memory at its end, before it is marked finished; a synchronising call
 * reports the bits of the latest such copy.  With concurrent launches on one device, a
 * PIM_ERR_TIMEOUT is thus reported by the first synchronising call on a run that ended
 * after it was raised, which may belong to another instance of that device. */
int pim_sync(pim_instance* inst);

/*
 * pim_energies -- per-replica results of the last anneal (host outputs, R entries each;
 * any pointer may be NULL).  Synchronises first.
 *   best_E       minimum energy H over the visited states (Eq. 1, unscaled units).
 *   best_t       step t of the state that reached best_E.
 *   first_hit_t  first step with H <= target, or -1.
 *   final_E      H of the final state s(t_begin + sweeps).
 * Errors: PIM_ERR_STATE (no anneal yet), PIM_ERR_CUDA, PIM_ERR_TIMEOUT.
 */
int pim_energies(pim_instance* inst, double* best_E, int32_t* best_t, int32_t* first_hit_t,
                 double* final_E);

/* pim_best_state / pim_final_state -- host int8 R x n of -1/+1.  Synchronises first.
 * Errors: PIM_ERR_STATE, PIM_ERR_CUDA, PIM_ERR_TIMEOUT. */
int pim_best_state(pim_instance* inst, int8_t* out);
int pim_final_state(pim_instance* inst, int8_t* out);

/* pim_replicas -- R of the last anneal (0 before the first). */
int pim_replicas(const pim_instance* inst);

/*
 * pim_kernel_ms -- device time, in milliseconds, of the sweep kernel launch(es) of the
 * instance's last anneal (all sweeps plus the final energy evaluation; staging and initial
 * spins excluded), measured with CUDA events recorded on the launching stream around the
 * launch.  Synchronises first.  With PIM_PATH_FP32REF it covers all the per-sweep kernels.
 * Errors: PIM_ERR_STATE (no anneal yet), PIM_ERR_CUDA.
 */
int pim_kernel_ms(pim_instance* inst, float* ms);

/*
 * pim_submit / pim_poll -- asynchronous anneal on the library's own stream.
 * pim_submit enqueues pim_anneal(inst, replicas, 0, sweeps, seed, 0, NULL, NaN, 0) and
 * returns a ticket; pim_poll returns PIM_PENDING while it runs, PIM_OK when done, or an
 * error.  A ticket is valid until the instance is destroyed or re-submitted.
 * Errors: as pim_anneal; pim_poll: PIM_ERR_INVALID for an unknown ticket.
 */
int pim_submit(pim_instance* inst, int replicas, int sweeps, uint64_t seed, uint64_t* ticket);
int pim_poll(uint64_t ticket);

/* pim_destroy -- free the instance and its device memory (NULL is a no-op).  Waits for
 * its pending work first. */
void pim_destroy(pim_instance* inst);

/* pim_last_error -- thread-local description of the last failure ("" if none). */
const char* pim_last_error(void);

/*
 * pim_set_fault_injection -- testing hook for the failure handling of the fused kernels
 * (no counterpart in the paper).  Applies to launches made after the call, process-wide.
 *   mode           0 = off; 1 = the sweep kernels skip their first field computation (no MMA
 *                  issued, no operand loaded), so their first bounded wait cannot complete.
 *   wait_limit_ns  limit of every device-side wait of later launches (0 = 2 s).
 * With mode 1 the kernel gives up after the limit, stops every thread at the next barrier,
 * releases its tensor memory and returns; the next synchronising call on the instance
 * reports PIM_ERR_TIMEOUT and the CUDA context stays usable.
 * Errors: PIM_ERR_INVALID (unknown mode).
 */
int pim_set_fault_injection(int mode, uint64_t wait_limit_ns);

/*
 * Inspection entry points (host only; no GPU needed).
 * pim_noise_levels -- the 4096 float32 noise levels z(m) the decision tables use:
 *   Gaussian: z(m) = fl32(Phi^-1((m+0.5)/4096)) for m < 2048 and z(4095-m) = -z(m);
 *   uniform:  z(m) = (2m - 4095)/4096.
 * pim_activation_levels -- tau_t(I) for I = -imax .. imax (2*imax+1 floats) for one b_t:
 *   tanh: fl32(tanh(b_t * I)) evaluated in float64; LUT: Algorithm "LUT-based tanh
 *   approximation" with L = lut_levels.
 * Errors: PIM_ERR_INVALID.
 */
int pim_noise_levels(int noise_kind, float* out4096);
int pim_activation_levels(float b_t, int imax, int act_kind, int lut_levels, float* out);

/*
 * pim_thresholds -- copy the device decision table of the instance's schedule to the
 * host: for every step t and field I = -imax..imax a uint32 word whose low half is the
 * least key m with a +1 decision when s_i(t) = -1 and whose high half is the same for
 * s_i(t) = +1 (4096 = never).  Layout [steps][stride_words]; entry I is at index
 * I + imax.  `*steps`, `*imax` and `*stride_words` are returned when non-NULL; `out` may
 * be NULL to query the sizes only.
 * Errors: PIM_ERR_STATE (no schedule), PIM_ERR_INVALID (cap too small), PIM_ERR_CUDA.
 */
int pim_thresholds(pim_instance* inst, uint32_t* out, size_t cap_words, int* steps, int* imax,
                   int* stride_words);

/*
 * pim_anneal_noalloc -- the fused sweep path for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a deployment entry point of the library.
 *
 * Who needs it: code that must not call cudaMalloc while it runs -- a real-time detection
 * loop where an allocation can synchronise the device and stall every other stream, a host
 * framework that owns all device memory through its own pool or a fixed arena and hands
 * out only buffers it allocated, or a process whose memory budget was fixed at start-up.
 * Such a caller passes its own inputs and outputs; every other buffer the path needs
 * (staged couplings, activation and decision tables, launch descriptors, the device error
 * word) lives in one file-scope device array of 16 MiB that every GPU which loads this
 * library holds until the process exits.  The call makes no cudaMalloc, cudaFree or other
 * allocating call.
 *
 * Runs sweeps 0 .. steps-1 of Eq. 4 with Gaussian noise and the tanh activation, h = 0,
 * Philox initial spins, exactly as pim_create + pim_set_schedule(noise GAUSS, act TANH) +
 * pim_anneal(t_begin 0, sweeps = steps, init NULL, flags 0) would, with the same results.
 *   n, J, scale_c    host int8 row-major n x n couplings (symmetric, zero diagonal) with
 *                    max_i sum_j |J_ij| <= 255; n <= PIM_NOALLOC_MAX_N; c > 0 as pim_create.
 *   steps, beta, eta host float schedules of `steps` <= PIM_NOALLOC_MAX_STEPS entries; xi >= 0.
 *   replicas         1 .. PIM_NOALLOC_MAX_REPLICAS; seed, instance_id, target_energy as
 *                    pim_anneal (NaN disables the first hit).
 *   best_E, best_t, first_hit_t, final_E   device arrays of `replicas` entries (outputs).
 *   best_bits, final_bits   device uint32 arrays [replicas][words], words = 2*ceil(n/64);
 *                    bit i of word i/32 of row r is set when spin i of replica r is +1.
 *   cuda_stream      cudaStream_t (NULL = legacy default stream); the call returns after the
 *                    anneal has finished on it.
 * Set-up: the first call on a device looks up that device's address of the array
 * (cudaGetSymbolAddress, with the device current).  Under CUDA's default lazy module
 * loading that lookup is also what loads the library's device code on that device, and the
 * load is where the 16 MiB array is reserved (it may synchronise the device).  So the first
 * call on each device does allocate: make one warm-up call at start-up, before the
 * real-time part and before any stream capture; later calls allocate nothing.
 * Sharing: every call uses the same array and leaves the last call's contents in it (the
 * error word is cleared at the start of each call).  Calls whose work overlaps on the GPU
 * would race on the array; this entry point serialises its own calls with a host lock and
 * waits for its work, so it never overlaps itself.
 * Errors: PIM_ERR_INVALID (sizes beyond the maxima, bad J, NULL pointers, bad schedule),
 *         PIM_ERR_TIMEOUT, PIM_ERR_CUDA, PIM_ERR_UNSUPPORTED (device index >= 64).
 */
#define PIM_NOALLOC_MAX_N 256
#define PIM_NOALLOC_MAX_STEPS 2048
#define PIM_NOALLOC_MAX_REPLICAS 4096
int pim_anneal_noalloc(int n, const int8_t* J, double scale_c, int steps, const float* beta,
                       const float* eta, float xi, int replicas, uint64_t seed,
                       uint32_t instance_id, double target_energy, double* best_E,
                       int32_t* best_t, int32_t* first_hit_t, double* final_E,
                       uint32_t* best_bits, uint32_t* final_bits, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PIM_H */
