// Host runtime of the C ABI declared in include/pim.h: argument checking, device memory,
// schedule tables, launch assembly and result copies.  Every sweep of the method runs in
// the device kernels; this file only stages inputs and moves results.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "host_tables.h"
#include "kernels.h"
#include "pim.h"

#define PIM_API extern "C" __attribute__((visibility("default")))

extern "C" void pim_destroy(pim_instance* inst);

using namespace pim;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? PIM_ERR_NOMEM : PIM_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(call, what)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
  } while (0)

constexpr int kMaxN = 8192;        // plain path limit
constexpr int kMaxNTensor = 256;   // fused kernel limit
constexpr int kMaxNpadFp4 = 4096;  // coupling-resident large-N variant: 64 x npad / 2 bytes
                                   // of E2M1 couplings per CTA fit in shared memory
constexpr int kMaxNFixedReal = 128;  // fixed-point real couplings: two coupling images fit in
                                     // the fused real-valued kernel's shared memory
constexpr int kMaxImaxTensor = 511;
constexpr int kMaxImaxDiag = 255;  // |I| < 256: D = I + 256 s keeps the sign of s
constexpr int kMaxDiagK = 2048;    // widest diagonal of the E5M2 images (table of 4K entries)

// Diagonal K = 2^k > imax of the wide diagonal-encoded mode (E5M2 images, 256 < K <= 2048),
// or 0 when the field range needs none or is too wide.
int wide_diag_k(int imax) {
  if (imax <= kMaxImaxDiag || imax >= kMaxDiagK) return 0;
  int K = 512;
  while (K <= imax) K <<= 1;
  return K;
}

// Decision thresholds of one (schedule, c, field range), shared between instances.
struct Schedule {
  int steps = 0;
  int imax = 0;          // table covers I = -imax .. imax
  int stride_words = 0;  // per-step stride, multiple of 4 words (16 bytes)
  uint32_t* d_thr = nullptr;
  uint32_t* d_thr_diag = nullptr;  // by D = I + 256 s (only when imax <= 255)
  uint32_t* d_thr_dk = nullptr;    // by D = I + dk s, 16-bit entries [steps][4 dk] (wide mode)
  int dk = 0;
  // Real-valued couplings: the decision is evaluated on the device from these.
  float* d_bt = nullptr;   // b_t = fl32(beta_t c)
  float* d_eta = nullptr;  // eta_t
  float* d_z = nullptr;    // 4096 noise levels
  float xi = 0.0f;
  int act = 0, lut = 0;
  int device = 0;
  // Real couplings in the fixed-point datapath (fix_w > 0): d_bt holds fl32(beta_t) (the
  // scale c is folded into the quantized couplings) and the decision uses these integer
  // tables, in units of 2^-(fix_w - fix_i).
  int fix_w = 0, fix_i = 0;
  int32_t* d_fix_tau = nullptr;  // [2^fix_w] Q(act(x))
  int32_t* d_fix_eta = nullptr;  // [steps] Q(eta_t)
  int32_t* d_fix_z = nullptr;    // [4096] Q(z)
  int32_t fix_xi = 0;            // Q(xi)
  ~Schedule() {
    if (d_thr || d_thr_diag || d_thr_dk || d_bt || d_fix_tau) {
      int prev = 0;
      cudaGetDevice(&prev);
      cudaSetDevice(device);
      cudaFree(d_thr);
      cudaFree(d_thr_diag);
      cudaFree(d_thr_dk);
      cudaFree(d_bt);
      cudaFree(d_eta);
      cudaFree(d_z);
      cudaFree(d_fix_tau);
      cudaFree(d_fix_eta);
      cudaFree(d_fix_z);
      cudaSetDevice(prev);
    }
  }
};

// Fault injection for tests (pim_set_fault_injection).
std::atomic<int> g_inject{0};
std::atomic<uint64_t> g_wait_ns{0};

std::mutex g_sched_mu;
std::map<std::string, std::weak_ptr<Schedule>> g_sched_cache;

// Per-device error word written by the kernels, and a mapped pinned host mirror that a
// one-thread kernel refreshes at the end of every run, before its completion event, so
// result getters read host memory instead of issuing a synchronous copy.  (A copy command
// would queue on the copy engine behind copies of other streams that wait for their own
// kernels, delaying this run's completion; a kernel does not.)
struct ErrWord {
  int* d = nullptr;
  int* h = nullptr;
  int* h_dev = nullptr;  // device address of h; null: read d synchronously instead
};
std::mutex g_err_mu;
std::map<int, ErrWord> g_err_word;

ErrWord* error_word(int dev) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  auto it = g_err_word.find(dev);
  if (it != g_err_word.end()) return &it->second;
  ErrWord w;
  if (cudaMalloc(&w.d, sizeof(int)) != cudaSuccess) return nullptr;
  if (cudaHostAlloc(&w.h, sizeof(int), cudaHostAllocPortable | cudaHostAllocMapped) != cudaSuccess) {
    cudaFree(w.d);
    return nullptr;
  }
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&w.h_dev), w.h, 0) != cudaSuccess) {
    cudaGetLastError();
    w.h_dev = nullptr;
  }
  cudaMemset(w.d, 0, sizeof(int));
  *w.h = 0;
  return &(g_err_word[dev] = w);
}

int* device_error_word(int dev) {
  ErrWord* w = error_word(dev);
  return w ? w->d : nullptr;
}

// CUDA events without timing, reused across instances (creating and destroying two per
// instance is a visible share of staging small instances).
std::mutex g_ev_mu;
std::map<int, std::vector<cudaEvent_t>> g_free_events;

cudaError_t take_event(int dev, cudaEvent_t* ev) {
  {
    std::lock_guard<std::mutex> lk(g_ev_mu);
    auto& v = g_free_events[dev];
    if (!v.empty()) {
      *ev = v.back();
      v.pop_back();
      return cudaSuccess;
    }
  }
  return cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
}

void give_event(int dev, cudaEvent_t ev) {
  if (!ev) return;
  std::lock_guard<std::mutex> lk(g_ev_mu);
  g_free_events[dev].push_back(ev);
}

// Host-to-device uploads of run descriptors through pinned staging buffers: a copy from
// pageable memory may make the driver synchronise with the stream first, which would stall
// the host behind the previous run.  A buffer is reused once the event recorded after its
// copy has completed.
struct UploadBuf {
  void* h = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
  bool busy = false;
};
std::mutex g_up_mu;
std::map<int, std::vector<std::unique_ptr<UploadBuf>>> g_up;

cudaError_t upload_async(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  UploadBuf* u = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_up_mu);
    for (auto& b : g_up[dev])
      if (!b->busy && b->cap >= bytes && cudaEventQuery(b->ev) == cudaSuccess) {
        u = b.get();
        break;
      }
    if (!u) {
      auto b = std::make_unique<UploadBuf>();
      size_t cap = 4096;
      while (cap < bytes) cap <<= 1;
      cudaError_t e = cudaHostAlloc(&b->h, cap, cudaHostAllocPortable);
      if (e != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming)) != cudaSuccess) {
        cudaFreeHost(b->h);
        return e;
      }
      b->cap = cap;
      u = b.get();
      g_up[dev].push_back(std::move(b));
    }
    u->busy = true;
  }
  std::memcpy(u->h, src, bytes);
  cudaError_t e = cudaMemcpyAsync(dst, u->h, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(u->ev, st);
  std::lock_guard<std::mutex> lk(g_up_mu);
  u->busy = false;
  return e;
}

// Completion event of one run, shared by every instance of the run (one record per run,
// however many instances it holds); back to the free list with its last holder.
struct RunEvent {
  cudaEvent_t ev = nullptr;
  int device = 0;
  ~RunEvent() { give_event(device, ev); }
};

// Pinned host blocks for results copied back with the run, kept in power-of-two size
// classes and reused (page-locking memory costs far more than a small copy).
std::mutex g_pin_mu;
std::multimap<size_t, void*> g_free_pinned;

size_t pinned_class(size_t bytes) {
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  return c;
}

void* take_pinned(size_t cls) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    auto it = g_free_pinned.find(cls);
    if (it != g_free_pinned.end()) {
      void* p = it->second;
      g_free_pinned.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaHostAlloc(&p, cls, cudaHostAllocPortable | cudaHostAllocMapped) != cudaSuccess) return nullptr;
  return p;
}

void give_pinned(void* p, size_t cls) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_free_pinned.emplace(cls, p);
}

// Per device: non-blocking streams for input uploads, staging kernels and frees, and a memory
// pool that keeps freed blocks (instance buffers come and go with every request).
struct DeviceCtx {
  cudaStream_t staging = nullptr;
  // Copy-only stream for the inputs of pim_create: it never waits behind a kernel, so
  // pageable uploads proceed while sweep kernels hold every SM.
  cudaStream_t upload = nullptr;
  // Kernel-free stream on which blocks go back to the pool once their run has finished, so
  // the free executes right then and the next allocations reuse the block (a free queued
  // behind staging kernels would wait for SMs that a running sweep kernel holds, and the
  // pool would grow instead, which stalls the host until the GPU is idle).
  cudaStream_t release = nullptr;
  cudaMemPool_t pool = nullptr;
  // Instances record their `ready` event on `staging` in the order of stage_seq, so a run
  // waits only for the latest of its instances' events.
  std::mutex stage_mu;
  uint64_t stage_seq = 0;
};
std::mutex g_ctx_mu;
std::map<int, DeviceCtx> g_ctx;

DeviceCtx* device_ctx(int dev) {
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  DeviceCtx& c = g_ctx[dev];
  if (!c.staging) {
    if (cudaStreamCreateWithFlags(&c.staging, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaStreamCreateWithFlags(&c.upload, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaStreamCreateWithFlags(&c.release, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&c.pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  return &c;
}

// The staging stream waits for everything queued so far on the upload stream.
cudaError_t staging_after_upload(DeviceCtx* c, int dev) {
  cudaEvent_t up = nullptr;
  cudaError_t e = take_event(dev, &up);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventRecord(up, c->upload)) == cudaSuccess) e = cudaStreamWaitEvent(c->staging, up, 0);
  give_event(dev, up);  // the wait above holds this record
  return e;
}

// Stream-ordered allocation from the library's pool.
cudaError_t pool_alloc(void** p, size_t bytes, int dev, cudaStream_t st) {
  DeviceCtx* c = device_ctx(dev);
  if (!c) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(p, bytes, c->pool, st);
}

// Free `p` on the release stream once `after` (if any) has completed.
void pool_free_after(void* p, int dev, cudaEvent_t after) {
  if (!p) return;
  DeviceCtx* c = device_ctx(dev);
  if (!c) return;
  if (after) cudaStreamWaitEvent(c->release, after, 0);
  cudaFreeAsync(p, c->release);
}

// Stream-ordered scratch for one run on st, from the library's pool of the current device
// (which keeps its memory, unlike the default pool that returns it at every sync).
cudaError_t run_alloc(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  return pool_alloc(p, bytes, dev, st);
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// CUDA events around one sweep-kernel launch, shared by the instances of that launch.
struct LaunchTimer {
  cudaEvent_t start = nullptr, stop = nullptr;
  ~LaunchTimer() {
    if (start) cudaEventDestroy(start);
    if (stop) cudaEventDestroy(stop);
  }
};

}  // namespace

struct pim_instance {
  int device = 0;
  int n = 0, npad = 0, words = 0;
  double c = 1.0;
  int imax = 0;  // exact max_i sum_j |J_ij| + |h_i|
  bool has_h = false;
  bool diag = false;  // image carries 256 on the diagonal (h = 0, imax <= 255)
  // Mid-N range, h = 0, couplings exact in E5M2: a second image in E5M2 with dk5 = 2^k >
  // the table's field bound (at least 256) on the diagonal, for the mid-N kernel's
  // diagonal-encoded path.
  uint8_t* d_img5 = nullptr;
  int dk5 = 0;
  // 256 < n, npad <= 4096, couplings in {0, +-1, +-2, +-3, +-4, +-6}: the E2M1 image of the
  // coupling-resident large-N variant (column-block-major, npad x npad / 2 bytes).
  uint8_t* d_img4 = nullptr;
  bool real = false;  // real-valued couplings: BF16 operand image, float bias
  float* d_hf = nullptr;
  // Fixed-point datapath of real couplings (n <= kMaxNFixedReal): the couplings and bias as
  // given (float64), and the device block built from them for format (fix_w, fix_i):
  // BF16 images of the high and low parts of Q(c J), then Q(c h) as float32.
  std::vector<double> host_J, host_h;
  char* d_fix = nullptr;
  uint8_t* d_fix_hi = nullptr;
  uint8_t* d_fix_lo = nullptr;
  float* d_fix_h = nullptr;
  int fix_w = 0, fix_i = 0;
  char* d_slab = nullptr;   // J8 | image | bias (one pool block)
  char* d_res = nullptr;    // results (one pool block)
  cudaEvent_t ready = nullptr;  // staging of the inputs done
  uint64_t ready_seq = 0;       // order of `ready` on the device's staging stream
  int8_t* d_J8 = nullptr;
  uint8_t* d_img = nullptr;
  float* d_jf = nullptr;
  int32_t* d_h = nullptr;
  std::shared_ptr<Schedule> sched;
  // results of the last anneal
  int R = 0, R_cap = 0;
  double* d_bestE = nullptr;
  double* d_finalE = nullptr;
  int32_t* d_bestT = nullptr;
  int32_t* d_first = nullptr;
  uint32_t* d_best_bits = nullptr;
  uint32_t* d_cur_bits = nullptr;
  bool has_results = false;
  size_t res_bytes = 0;      // size of the d_res block
  char* h_res = nullptr;     // pinned copy of d_res (PIM_RESULTS_TO_HOST)
  void* h_res_dev = nullptr; // its device-side address (mapped pinned memory), or null
  size_t h_res_cap = 0;
  bool h_res_valid = false;  // the last run copied its results into h_res
  std::shared_ptr<RunEvent> done;  // completion of the last run (shared with its batch)
  cudaEvent_t done_ev() const { return done ? done->ev : nullptr; }
  uint64_t ticket = 0;
  std::shared_ptr<LaunchTimer> timer;
};

namespace {

void free_results(pim_instance* p) {
  pool_free_after(p->d_res, p->device, p->done_ev());
  p->d_res = nullptr;
  p->d_bestE = p->d_finalE = nullptr;
  p->d_bestT = p->d_first = nullptr;
  p->d_best_bits = p->d_cur_bits = nullptr;
  p->R_cap = 0;
}

// Results of R replicas in one block, stream-ordered on the anneal's stream:
// best_E | final_E (f64) | best_t | first_hit (i32) | best bits | current bits.
int ensure_results(pim_instance* p, int R, cudaStream_t st) {
  if (R <= p->R_cap) return PIM_OK;
  free_results(p);
  p->h_res_valid = false;
  const size_t bits = static_cast<size_t>(R) * p->words * sizeof(uint32_t);
  const size_t scal = align256(static_cast<size_t>(R) * 24);
  void* d = nullptr;
  CK(pool_alloc(&d, scal + 2 * align256(bits), p->device, st), "allocating results");
  p->d_res = static_cast<char*>(d);
  p->d_bestE = reinterpret_cast<double*>(p->d_res);
  p->d_finalE = p->d_bestE + R;
  p->d_bestT = reinterpret_cast<int32_t*>(p->d_finalE + R);
  p->d_first = p->d_bestT + R;
  p->d_best_bits = reinterpret_cast<uint32_t*>(p->d_res + scal);
  p->d_cur_bits = reinterpret_cast<uint32_t*>(p->d_res + scal + align256(bits));
  p->R_cap = R;
  p->res_bytes = scal + 2 * align256(bits);
  return PIM_OK;
}

// After a run's completion event: the mirror holds the error bits as of that run's end.
int check_device_errors(int dev) {
  ErrWord* w = error_word(dev);
  if (!w) return PIM_OK;
  int h = 0;
  if (w->h_dev)
    h = *static_cast<volatile int*>(w->h);
  else
    CK(cudaMemcpy(&h, w->d, sizeof(int), cudaMemcpyDeviceToHost), "reading device error word");
  if (h != 0) {
    cudaMemset(w->d, 0, sizeof(int));
    *static_cast<volatile int*>(w->h) = 0;
    if (h & kDevErrTimeout) return fail(PIM_ERR_TIMEOUT, "a device-side bounded wait gave up");
    return fail(PIM_ERR_CUDA, "device error bits 0x%x", h);
  }
  return PIM_OK;
}

int sync_instance(pim_instance* p) {
  if (p->done) CK(cudaEventSynchronize(p->done->ev), "cudaEventSynchronize");
  return check_device_errors(p->device);
}

std::string schedule_key(int steps, const float* beta, const float* eta, float xi, int noise,
                         int act, int lut, double c, int imax, int device) {
  std::string k;
  auto put = [&](const void* d, size_t b) { k.append(static_cast<const char*>(d), b); };
  put(&steps, sizeof steps);
  put(&xi, sizeof xi);
  put(&noise, sizeof noise);
  put(&act, sizeof act);
  put(&lut, sizeof lut);
  put(&c, sizeof c);
  put(&imax, sizeof imax);
  put(&device, sizeof device);
  put(beta, steps * sizeof(float));
  put(eta, steps * sizeof(float));
  return k;
}

int build_schedule(std::shared_ptr<Schedule>& out, int steps, const float* beta,
                   const float* eta, float xi, int noise, int act, int lut, double c, int imax,
                   int device) {
  auto s = std::make_shared<Schedule>();
  s->steps = steps;
  s->imax = imax;
  s->device = device;
  const int width = 2 * imax + 1;
  s->stride_words = (width + 3) & ~3;
  std::vector<float> tau(static_cast<size_t>(steps) * width);
  for (int t = 0; t < steps; ++t)
    activation_levels(scaled_beta(beta[t], c), imax, act, lut, &tau[static_cast<size_t>(t) * width]);
  std::vector<float> z(kNoiseLevels);
  noise_levels(noise == PIM_NOISE_GAUSS ? 0 : 1, z.data());
  float *d_tau = nullptr, *d_eta = nullptr, *d_z = nullptr;
  cudaStream_t st = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_tau);
    cudaFree(d_eta);
    cudaFree(d_z);
    if (st) cudaStreamDestroy(st);
  };
  auto ck = [&](cudaError_t e, const char* what) -> int {
    if (e == cudaSuccess) return PIM_OK;
    cleanup();
    return cuda_fail(e, what);
  };
  int rc;
  if ((rc = ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "cudaStreamCreate"))) return rc;
  if ((rc = ck(cudaMalloc(&s->d_thr, static_cast<size_t>(steps) * s->stride_words * 4),
               "cudaMalloc thresholds")))
    return rc;
  if ((rc = ck(cudaMalloc(&d_tau, tau.size() * 4), "cudaMalloc tau"))) return rc;
  if ((rc = ck(cudaMalloc(&d_eta, steps * 4), "cudaMalloc eta"))) return rc;
  if ((rc = ck(cudaMalloc(&d_z, kNoiseLevels * 4), "cudaMalloc z"))) return rc;
  if ((rc = ck(cudaMemcpyAsync(d_tau, tau.data(), tau.size() * 4, cudaMemcpyHostToDevice, st),
               "upload tau")))
    return rc;
  if ((rc = ck(cudaMemcpyAsync(d_eta, eta, steps * 4, cudaMemcpyHostToDevice, st), "upload eta")))
    return rc;
  if ((rc = ck(cudaMemcpyAsync(d_z, z.data(), kNoiseLevels * 4, cudaMemcpyHostToDevice, st),
               "upload z")))
    return rc;
  if ((rc = ck(launch_thresholds(d_tau, d_eta, d_z, xi, steps, imax, s->stride_words, s->d_thr, st),
               "threshold kernel")))
    return rc;
  if (imax <= kMaxImaxDiag) {
    if ((rc = ck(cudaMalloc(&s->d_thr_diag, static_cast<size_t>(steps) * 1024 * 2),
                 "cudaMalloc diagonal thresholds")))
      return rc;
    if ((rc = ck(launch_diag_thresholds(s->d_thr, steps, imax, s->stride_words, 256, s->d_thr_diag, st),
                 "diagonal threshold kernel")))
      return rc;
  }
  if (const int K = wide_diag_k(imax)) {
    if ((rc = ck(cudaMalloc(&s->d_thr_dk, static_cast<size_t>(steps) * 4 * K * 2),
                 "cudaMalloc wide diagonal thresholds")))
      return rc;
    if ((rc = ck(launch_diag_thresholds(s->d_thr, steps, imax, s->stride_words, K, s->d_thr_dk, st),
                 "wide diagonal threshold kernel")))
      return rc;
    s->dk = K;
  }
  if ((rc = ck(cudaStreamSynchronize(st), "threshold build"))) return rc;
  cleanup();
  out = s;
  return PIM_OK;
}

int table_imax(const pim_instance* p) {
  // Round the exact field bound up to 64k-1 so instances of similar size share tables.
  return p->imax | 63;
}

}  // namespace

namespace pim {
void set_last_error(const char* msg) { g_last_error = msg; }

int schedule_device_arrays(const pim_instance* inst, const float** b_t, const float** eta,
                           const float** zlev, float* xi, int* act, int* lut_levels) {
  if (!inst || !inst->real || !inst->sched || !inst->sched->d_bt || inst->sched->fix_w > 0)
    return PIM_ERR_STATE;
  *b_t = inst->sched->d_bt;
  *eta = inst->sched->d_eta;
  *zlev = inst->sched->d_z;
  *xi = inst->sched->xi;
  *act = inst->sched->act;
  *lut_levels = inst->sched->lut;
  return PIM_OK;
}
}  // namespace pim

// ----------------------------------------------------------------------------------------
PIM_API const char* pim_last_error(void) { return g_last_error.c_str(); }

PIM_API int pim_noise_levels(int noise_kind, float* out4096) {
  if (!out4096 || (noise_kind != PIM_NOISE_GAUSS && noise_kind != PIM_NOISE_UNIFORM))
    return fail(PIM_ERR_INVALID, "pim_noise_levels: bad arguments");
  noise_levels(noise_kind == PIM_NOISE_GAUSS ? 0 : 1, out4096);
  return PIM_OK;
}

PIM_API int pim_activation_levels(float b_t, int imax, int act_kind, int lut_levels, float* out) {
  if (!out || imax < 0 || !std::isfinite(b_t) || (act_kind != PIM_ACT_TANH && act_kind != PIM_ACT_LUT) ||
      (act_kind == PIM_ACT_LUT && lut_levels < 2))
    return fail(PIM_ERR_INVALID, "pim_activation_levels: bad arguments");
  activation_levels(b_t, imax, act_kind, lut_levels, out);
  return PIM_OK;
}

namespace {

// Runs fn(begin, end) over [0, count) in contiguous parts on up to 16 host threads, at
// least `grain` items per thread; small jobs (`work` < 2M elements) stay on the calling
// thread, where spawning threads would cost more than it saves.
template <class F>
void parallel_for(int count, F fn, int grain = 64, size_t work = SIZE_MAX) {
  const int hw = static_cast<int>(std::thread::hardware_concurrency());
  const int nth = work < (2u << 20) ? 1 : std::max(1, std::min({hw, 16, count / grain}));
  if (nth == 1) {
    fn(0, count);
    return;
  }
  std::vector<std::thread> th;
  const int per = (count + nth - 1) / nth;
  for (int k = 0; k < nth; ++k) {
    const int b = k * per, e = std::min(count, b + per);
    if (b < e) th.emplace_back(fn, b, e);
  }
  for (auto& t : th) t.join();
}

// First (row-major order) position (i, j), i < j, where a[i*n+j] != a[j*n+i], or (-1, -1).
// Compares 64 x 64 tiles against their transposes so both reads stay cache-friendly.
template <class T>
std::pair<int, int> first_asymmetry(const T* a, int n) {
  constexpr int kB = 64;
  const int nb = (n + kB - 1) / kB;
  std::vector<long long> first(nb, -1);
  std::atomic<int> next{0};  // block rows have triangular work: hand them out one by one
  parallel_for(nb, [&](int, int) {
    for (int bi = next++; bi < nb; bi = next++) {
      long long hit = -1;
      const int i1 = std::min(n, (bi + 1) * kB);
      for (int bj = bi; bj < nb; ++bj) {
        const int j0 = bj * kB, j1 = std::min(n, (bj + 1) * kB);
        for (int i = bi * kB; i < i1; ++i)
          for (int j = std::max(i + 1, j0); j < j1; ++j)
            if (!(a[static_cast<size_t>(i) * n + j] == a[static_cast<size_t>(j) * n + i])) {
              const long long pos = static_cast<long long>(i) * n + j;
              if (hit < 0 || pos < hit) hit = pos;
            }
      }
      first[bi] = hit;
    }
  }, 1, static_cast<size_t>(n) * n);
  for (long long h : first)
    if (h >= 0) return {static_cast<int>(h / n), static_cast<int>(h % n)};
  return {-1, -1};
}

// sum_j |row[j]| into *sum and whether some entry lies outside [-16, 16]; *not_e5m2 is set
// when some |entry| in 9..16 is odd (9, 11, 13, 15 have no exact E5M2 encoding).  Byte
// arithmetic with 16-bit partial sums (|v| <= 128, 256 of them fit) so that the loop
// vectorises.
bool abs_row_sum_i8(const int8_t* row, int n, int* sum, bool* not_e5m2, bool* not_e2m1) {
  int s = 0;
  uint8_t out = 0, odd = 0, nf4 = 0;
  for (int j0 = 0; j0 < n; j0 += 256) {
    const int j1 = std::min(n, j0 + 256);
    uint16_t part = 0;
    for (int j = j0; j < j1; ++j) {
      const uint8_t u = static_cast<uint8_t>(row[j]);
      const uint8_t neg = static_cast<uint8_t>(-(u >> 7));  // 0xFF for negative entries
      const uint8_t a = static_cast<uint8_t>((u ^ neg) - neg);  // |v| (128 for -128)
      part += a;
      out |= static_cast<uint8_t>(static_cast<uint8_t>(u + 16) > 32);
      odd |= static_cast<uint8_t>((a > 8) & a);
      nf4 |= static_cast<uint8_t>((a > 6) | (a == 5));  // E2M1 integers: 0..4 and 6
    }
    s += part;
  }
  *sum = s;
  *not_e5m2 = (odd & 1) != 0;
  *not_e2m1 = nf4 != 0;
  return out != 0;
}

// Transposes an 8 x 8 byte block held as 8 words (word k = row k, byte c = column c,
// little-endian byte order) with three rounds of masked swaps: 4x4, 2x2, then 1x1 blocks.
void transpose_8x8_bytes(uint64_t* w) {
  for (int k = 0; k < 4; ++k) {
    const uint64_t t = ((w[k] >> 32) ^ w[k + 4]) & 0x00000000FFFFFFFFull;
    w[k] ^= t << 32;
    w[k + 4] ^= t;
  }
  for (int k : {0, 1, 4, 5}) {
    const uint64_t t = ((w[k] >> 16) ^ w[k + 2]) & 0x0000FFFF0000FFFFull;
    w[k] ^= t << 16;
    w[k + 2] ^= t;
  }
  for (int k = 0; k < 8; k += 2) {
    const uint64_t t = ((w[k] >> 8) ^ w[k + 1]) & 0x00FF00FF00FF00FFull;
    w[k] ^= t << 8;
    w[k + 1] ^= t;
  }
}

// Whether a byte matrix equals its transpose: 8 x 8 blocks of the upper triangle against the
// transposed mirror block, the ragged edge element by element.  first_asymmetry locates
// the mismatch when there is one.
bool symmetric_i8(const int8_t* a, int n) {
  const int nb = n / 8;
  std::atomic<int> next{0};
  std::atomic<bool> ok{true};
  parallel_for(nb, [&](int, int) {
    uint64_t diff = 0;
    for (int I = next++; I < nb; I = next++)
      for (int K = I; K < nb; ++K) {
        uint64_t A[8], B[8];
        for (int k = 0; k < 8; ++k) {
          std::memcpy(&A[k], a + static_cast<size_t>(8 * I + k) * n + 8 * K, 8);
          std::memcpy(&B[k], a + static_cast<size_t>(8 * K + k) * n + 8 * I, 8);
        }
        transpose_8x8_bytes(A);
        for (int k = 0; k < 8; ++k) diff |= A[k] ^ B[k];
      }
    if (diff) ok = false;
  }, 8, static_cast<size_t>(n) * n);
  for (int i = 0; i < n && ok; ++i)
    for (int j = std::max(8 * nb, i + 1); j < n; ++j)
      if (a[static_cast<size_t>(i) * n + j] != a[static_cast<size_t>(j) * n + i]) return false;
  return ok;
}

// Round a double to the nearest BF16 value (8 significant bits, ties to even) and return
// its bit pattern: round the 52-bit double significand at bit 45 (a carry moves into the
// exponent), then narrow to float, which is exact for finite values in float range.
uint16_t bf16_bits_rne(double v) {
  uint64_t b;
  std::memcpy(&b, &v, sizeof b);
  b += ((1ull << 44) - 1) + ((b >> 45) & 1);
  b &= ~((1ull << 45) - 1);
  double r;
  std::memcpy(&r, &b, sizeof r);
  const float f = static_cast<float>(r);
  uint32_t bits;
  std::memcpy(&bits, &f, sizeof bits);
  return static_cast<uint16_t>(bits >> 16);
}

// Real-valued couplings: J rounded to BF16 for the tensor-core operand, bias as float.
int create_real(pim_instance** out, int n, int j_type, const void* J, const void* h, double c) {
  auto at = [&](const void* a, size_t k) -> double {
    return j_type == PIM_J_FP32 ? static_cast<double>(static_cast<const float*>(a)[k])
                                : static_cast<const double*>(a)[k];
  };
  // One pass over 64 x 64 tile pairs (T, T^transpose), block rows shared out among host
  // threads: finiteness, zero diagonal, symmetry, and both tiles rounded to BF16.  Each
  // input element is read once; the first error in row-major order (of the upper triangle
  // for asymmetry) is reported.
  constexpr int kB = 64;
  const int nb = (n + kB - 1) / kB;
  std::unique_ptr<uint16_t[]> jb(new (std::nothrow) uint16_t[static_cast<size_t>(n) * n]);
  if (!jb) return fail(PIM_ERR_NOMEM, "pim_create: host allocation failed");
  std::vector<long long> err_pos(nb, -1);
  std::vector<int> err_kind(nb, 0);  // 1 not finite, 2 diagonal, 3 asymmetric
  std::atomic<int> next{0};
  parallel_for(nb, [&](int, int) {
    for (int bi = next++; bi < nb; bi = next++) {
      long long pos = -1;
      int kind = 0;
      auto note = [&](int i, int j, int k) {
        const long long q = static_cast<long long>(i) * n + j;
        if (pos < 0 || q < pos || (q == pos && k < kind)) {
          pos = q;
          kind = k;
        }
      };
      const int i0 = bi * kB, i1 = std::min(n, i0 + kB);
      for (int bj = bi; bj < nb; ++bj) {
        const int j0 = bj * kB, j1 = std::min(n, j0 + kB);
        for (int i = i0; i < i1; ++i)
          for (int j = std::max(j0, bi == bj ? i : j0); j < j1; ++j) {
            const double v = at(J, static_cast<size_t>(i) * n + j);
            const double w = at(J, static_cast<size_t>(j) * n + i);
            const bool fv = std::isfinite(v) && std::fabs(v) <= 1e30;
            const bool fw = std::isfinite(w) && std::fabs(w) <= 1e30;
            if (!fv) note(i, j, 1);
            if (!fw) note(j, i, 1);
            if (i == j && fv && v != 0.0) note(i, i, 2);
            if (fv && fw && v != w) note(i, j, 3);
            jb[static_cast<size_t>(i) * n + j] = bf16_bits_rne(fv ? v : 0.0);
            jb[static_cast<size_t>(j) * n + i] = bf16_bits_rne(fw ? w : 0.0);
          }
      }
      err_pos[bi] = pos;
      err_kind[bi] = kind;
    }
  }, 1, static_cast<size_t>(n) * n);
  long long pos = -1;
  int kind = 0;
  for (int b = 0; b < nb; ++b)
    if (err_pos[b] >= 0 && (pos < 0 || err_pos[b] < pos || (err_pos[b] == pos && err_kind[b] < kind))) {
      pos = err_pos[b];
      kind = err_kind[b];
    }
  if (pos >= 0) {
    const int i = static_cast<int>(pos / n), j = static_cast<int>(pos % n);
    if (kind == 1) return fail(PIM_ERR_INVALID, "pim_create: J[%d][%d] not finite", i, j);
    if (kind == 2)
      return fail(PIM_ERR_INVALID, "pim_create: J[%d][%d] != 0 (diagonal must be zero)", i, i);
    return fail(PIM_ERR_INVALID, "pim_create: J is not symmetric at (%d, %d)", i, j);
  }
  std::vector<float> hf(n, 0.0f);
  bool has_h = false;
  if (h)
    for (int i = 0; i < n; ++i) {
      const double v = at(h, i);
      if (!std::isfinite(v)) return fail(PIM_ERR_INVALID, "pim_create: h[%d] not finite", i);
      hf[i] = static_cast<float>(v);
      has_h |= hf[i] != 0.0f;
    }
  auto* p = new (std::nothrow) pim_instance();
  if (!p) return fail(PIM_ERR_NOMEM, "pim_create: host allocation failed");
  cudaGetDevice(&p->device);
  p->real = true;
  if (n <= kMaxNFixedReal) {  // kept for pim_set_schedule_fixed
    p->host_J.resize(static_cast<size_t>(n) * n);
    p->host_h.assign(n, 0.0);
    for (size_t k = 0; k < p->host_J.size(); ++k) p->host_J[k] = at(J, k);
    if (h)
      for (int i = 0; i < n; ++i) p->host_h[i] = at(h, i);
  }
  p->n = n;
  p->npad = n <= 128 ? 128 : (n <= 256 ? 256 : ((n + 127) / 128) * 128);
  p->words = ((n + 63) / 64) * 2;
  p->c = c;
  p->has_h = has_h;
  auto bail = [&](cudaError_t e, const char* what) {
    const int rc = cuda_fail(e, what);
    pim_destroy(p);
    return rc;
  };
  cudaError_t e;
  DeviceCtx* ctx = device_ctx(p->device);
  if (!ctx) return bail(cudaErrorMemoryAllocation, "device context");
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t o_img = align256(nn * 2), o_h = o_img + align256(static_cast<size_t>(p->npad) * p->npad * 2);
  void* slab = nullptr;
  if ((e = pool_alloc(&slab, o_h + align256(n * sizeof(float)), p->device, ctx->upload)) != cudaSuccess)
    return bail(e, "allocating J");
  p->d_slab = static_cast<char*>(slab);
  uint16_t* d_bf = reinterpret_cast<uint16_t*>(p->d_slab);
  p->d_img = reinterpret_cast<uint8_t*>(p->d_slab + o_img);
  if ((e = cudaMemcpyAsync(d_bf, jb.get(), nn * 2, cudaMemcpyHostToDevice, ctx->upload)) != cudaSuccess)
    return bail(e, "upload J");
  if (has_h) {
    p->d_hf = reinterpret_cast<float*>(p->d_slab + o_h);
    if ((e = cudaMemcpyAsync(p->d_hf, hf.data(), n * sizeof(float), cudaMemcpyHostToDevice,
                             ctx->upload)) != cudaSuccess)
      return bail(e, "upload h");
  }
  if ((e = staging_after_upload(ctx, p->device)) != cudaSuccess) return bail(e, "staging order");
  if ((e = launch_stage_bf16_image(d_bf, n, p->npad, p->d_img, ctx->staging, n > kMaxNTensor)) != cudaSuccess)
    return bail(e, "stage BF16 J image");
  if ((e = take_event(p->device, &p->ready)) != cudaSuccess)
    return bail(e, "cudaEventCreate");
  {
    std::lock_guard<std::mutex> lk(ctx->stage_mu);
    if ((e = cudaEventRecord(p->ready, ctx->staging)) != cudaSuccess) return bail(e, "cudaEventRecord");
    p->ready_seq = ++ctx->stage_seq;
  }
  *out = p;
  return PIM_OK;
}

int build_real_schedule(std::shared_ptr<Schedule>& out, int steps, const float* beta,
                        const float* eta, float xi, int noise, int act, int lut, double c,
                        int device) {
  auto s = std::make_shared<Schedule>();
  s->steps = steps;
  s->device = device;
  s->xi = xi;
  s->act = act;
  s->lut = lut;
  std::vector<float> bt(steps);
  for (int t = 0; t < steps; ++t) bt[t] = scaled_beta(beta[t], c);
  std::vector<float> z(kNoiseLevels);
  noise_levels(noise == PIM_NOISE_GAUSS ? 0 : 1, z.data());
  CK(cudaMalloc(&s->d_bt, steps * 4), "cudaMalloc schedule");
  CK(cudaMalloc(&s->d_eta, steps * 4), "cudaMalloc schedule");
  CK(cudaMalloc(&s->d_z, kNoiseLevels * 4), "cudaMalloc schedule");
  CK(cudaMemcpy(s->d_bt, bt.data(), steps * 4, cudaMemcpyHostToDevice), "upload schedule");
  CK(cudaMemcpy(s->d_eta, eta, steps * 4, cudaMemcpyHostToDevice), "upload schedule");
  CK(cudaMemcpy(s->d_z, z.data(), kNoiseLevels * 4, cudaMemcpyHostToDevice), "upload schedule");
  out = s;
  return PIM_OK;
}

}  // namespace

PIM_API int pim_create(pim_instance** out, int n, int j_type, const void* J, const void* h,
                       double scale_c) {
  if (!out) return fail(PIM_ERR_INVALID, "pim_create: out is NULL");
  *out = nullptr;
  if (n < 1 || n > kMaxN) return fail(PIM_ERR_INVALID, "pim_create: n=%d out of [1, %d]", n, kMaxN);
  if (!J) return fail(PIM_ERR_INVALID, "pim_create: J is NULL");
  if (!(scale_c > 0.0) || !std::isfinite(scale_c))
    return fail(PIM_ERR_INVALID, "pim_create: scale_c must be finite and > 0");
  if (j_type == PIM_J_FP32 || j_type == PIM_J_FP64) return create_real(out, n, j_type, J, h, scale_c);
  if (j_type != PIM_J_INT8) return fail(PIM_ERR_INVALID, "pim_create: unknown j_type %d", j_type);
  const int8_t* J8 = static_cast<const int8_t*>(J);
  const int32_t* h32 = static_cast<const int32_t*>(h);
  // Row pass (parallel): zero diagonal, |J_ij| <= 16 (exact in E4M3 with exact products),
  // row sums of |J| + |h| (the field bound); then the symmetry check.
  std::vector<long long> rowsum(n, 0);
  std::vector<int> bad(n, -1);
  std::vector<uint8_t> no_e5m2(n, 0), no_e2m1(n, 0);
  parallel_for(n, [&](int i0, int i1) {
    for (int i = i0; i < i1; ++i) {
      const int8_t* row = J8 + static_cast<size_t>(i) * n;
      long long s = h32 ? std::llabs(static_cast<long long>(h32[i])) : 0;
      int sum = 0;
      bool ne = false, nf4 = false;
      if (abs_row_sum_i8(row, n, &sum, &ne, &nf4) || row[i] != 0) {
        for (int j = 0; j < n; ++j) {  // locate the first offending entry of the row
          const int v = row[j];
          if ((i == j && v != 0) || v < -16 || v > 16) {
            bad[i] = j;
            break;
          }
        }
      }
      rowsum[i] = s + sum;
      no_e5m2[i] = ne ? 1 : 0;
      no_e2m1[i] = nf4 ? 1 : 0;
    }
  }, 64, static_cast<size_t>(n) * n);
  long long imax = 0;
  for (int i = 0; i < n; ++i) {
    if (bad[i] == i)
      return fail(PIM_ERR_INVALID, "pim_create: J[%d][%d] != 0 (diagonal must be zero)", i, i);
    if (bad[i] >= 0) {
      const int v = J8[static_cast<size_t>(i) * n + bad[i]];
      return fail(PIM_ERR_INVALID, "pim_create: |J[%d][%d]| = %d > 16", i, bad[i], v < 0 ? -v : v);
    }
    imax = std::max(imax, rowsum[i]);
  }
  if (!symmetric_i8(J8, n)) {
    const auto asym = first_asymmetry(J8, n);
    return fail(PIM_ERR_INVALID, "pim_create: J is not symmetric at (%d, %d)", asym.first, asym.second);
  }
  if (imax > (1 << 20)) return fail(PIM_ERR_INVALID, "pim_create: field range too large");
  auto* p = new (std::nothrow) pim_instance();
  if (!p) return fail(PIM_ERR_NOMEM, "pim_create: host allocation failed");
  cudaGetDevice(&p->device);
  p->n = n;
  p->npad = n <= 128 ? 128 : ((n + 255) / 256) * 256;
  p->words = (n + 31) / 32;
  if (p->words & 1) p->words += 1;  // even word count: rows of 16-bit chunks stay aligned
  p->c = scale_c;
  p->imax = static_cast<int>(imax);
  p->has_h = false;
  if (h32)
    for (int i = 0; i < n; ++i) p->has_h |= h32[i] != 0;
  auto bail = [&](cudaError_t e, const char* what) {
    const int rc = cuda_fail(e, what);
    pim_destroy(p);
    return rc;
  };
  // One pool block J8 | FP8 image | bias (| E5M2 image), uploaded on the library's upload
  // stream and staged on its staging stream; anneals wait for the `ready` event instead of
  // the host waiting here.
  cudaError_t e;
  DeviceCtx* ctx = device_ctx(p->device);
  if (!ctx) return bail(cudaErrorMemoryAllocation, "device context");
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t img = static_cast<size_t>(p->npad) * p->npad;
  bool e5m2_exact = true, e2m1_exact = true;
  for (int i = 0; i < n; ++i) e5m2_exact &= no_e5m2[i] == 0;
  for (int i = 0; i < n; ++i) e2m1_exact &= no_e2m1[i] == 0;
  if (n > kMaxNTensor && p->npad <= sweep_mid_max_npad() && !p->has_h && e5m2_exact)
    p->dk5 = table_imax(p) <= kMaxImaxDiag ? 256 : wide_diag_k(table_imax(p));
  const bool fp4 = n > kMaxNTensor && p->npad <= kMaxNpadFp4 && e2m1_exact;
  const size_t o_img = align256(nn), o_h = o_img + align256(img);
  const size_t o_img5 = o_h + align256(n * sizeof(int32_t));
  const size_t o_img4 = o_img5 + (p->dk5 ? align256(img) : 0);
  void* slab = nullptr;
  if ((e = pool_alloc(&slab, o_img4 + (fp4 ? align256(img / 2) : 0), p->device, ctx->upload)) != cudaSuccess)
    return bail(e, "allocating J");
  p->d_slab = static_cast<char*>(slab);
  p->d_J8 = reinterpret_cast<int8_t*>(p->d_slab);
  p->d_img = reinterpret_cast<uint8_t*>(p->d_slab + o_img);
  if ((e = cudaMemcpyAsync(p->d_J8, J8, nn, cudaMemcpyHostToDevice, ctx->upload)) != cudaSuccess)
    return bail(e, "upload J");
  if (p->has_h) {
    p->d_h = reinterpret_cast<int32_t*>(p->d_slab + o_h);
    if ((e = cudaMemcpyAsync(p->d_h, h32, n * sizeof(int32_t), cudaMemcpyHostToDevice,
                             ctx->upload)) != cudaSuccess)
      return bail(e, "upload h");
  }
  if ((e = staging_after_upload(ctx, p->device)) != cudaSuccess) return bail(e, "staging order");
  p->diag = n <= kMaxNTensor && !p->has_h && (p->imax | 63) <= kMaxImaxDiag;
  if ((e = launch_stage_fp8_image(p->d_J8, n, p->npad, p->diag ? 256 : 0, p->d_img, ctx->staging, false,
                                   n > kMaxNTensor)) !=
      cudaSuccess)
    return bail(e, "stage J image");
  if (p->dk5) {
    p->d_img5 = reinterpret_cast<uint8_t*>(p->d_slab + o_img5);
    if ((e = launch_stage_fp8_image(p->d_J8, n, p->npad, p->dk5, p->d_img5, ctx->staging, true, true)) !=
        cudaSuccess)
      return bail(e, "stage E5M2 J image");
  }
  if (fp4) {
    p->d_img4 = reinterpret_cast<uint8_t*>(p->d_slab + o_img4);
    if ((e = launch_stage_fp4_image(p->d_J8, n, p->npad, p->d_img4, ctx->staging)) != cudaSuccess)
      return bail(e, "stage E2M1 J image");
  }
  if ((e = take_event(p->device, &p->ready)) != cudaSuccess)
    return bail(e, "cudaEventCreate");
  {
    std::lock_guard<std::mutex> lk(ctx->stage_mu);
    if ((e = cudaEventRecord(p->ready, ctx->staging)) != cudaSuccess) return bail(e, "cudaEventRecord");
    p->ready_seq = ++ctx->stage_seq;
  }
  *out = p;
  return PIM_OK;
}

PIM_API int pim_set_schedule(pim_instance* inst, int steps, const float* beta, const float* eta,
                             float xi, int noise_kind, int act_kind, int lut_levels) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_set_schedule: instance is NULL");
  if (steps < 1 || !beta || !eta) return fail(PIM_ERR_INVALID, "pim_set_schedule: bad steps/arrays");
  if (!std::isfinite(xi) || xi < 0.0f) return fail(PIM_ERR_INVALID, "pim_set_schedule: xi must be finite, >= 0");
  if (noise_kind != PIM_NOISE_GAUSS && noise_kind != PIM_NOISE_UNIFORM)
    return fail(PIM_ERR_INVALID, "pim_set_schedule: unknown noise kind %d", noise_kind);
  if (act_kind != PIM_ACT_TANH && act_kind != PIM_ACT_LUT)
    return fail(PIM_ERR_INVALID, "pim_set_schedule: unknown activation %d", act_kind);
  if (act_kind == PIM_ACT_LUT && lut_levels < 2)
    return fail(PIM_ERR_INVALID, "pim_set_schedule: lut_levels must be >= 2");
  if (act_kind == PIM_ACT_TANH) lut_levels = 0;
  for (int t = 0; t < steps; ++t)
    if (!std::isfinite(beta[t]) || beta[t] < 0.0f || !std::isfinite(eta[t]) || eta[t] < 0.0f)
      return fail(PIM_ERR_INVALID, "pim_set_schedule: beta/eta[%d] must be finite and >= 0", t);
  const int imax = inst->real ? -1 : table_imax(inst);  // -1 marks a real-valued schedule
  const std::string key = schedule_key(steps, beta, eta, xi, noise_kind, act_kind, lut_levels,
                                       inst->c, imax, inst->device);
  std::shared_ptr<Schedule> s;
  {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    auto it = g_sched_cache.find(key);
    if (it != g_sched_cache.end()) s = it->second.lock();
  }
  if (!s) {
    const int rc = inst->real ? build_real_schedule(s, steps, beta, eta, xi, noise_kind, act_kind,
                                                    lut_levels, inst->c, inst->device)
                              : build_schedule(s, steps, beta, eta, xi, noise_kind, act_kind,
                                               lut_levels, inst->c, imax, inst->device);
    if (rc != PIM_OK) return rc;
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched_cache[key] = s;
  }
  if (inst->done) cudaEventSynchronize(inst->done->ev);
  inst->sched = s;
  return PIM_OK;
}

namespace {

// Decision thresholds of the fixed-point datapath, built on the host (fixed_thresholds)
// and uploaded; the diagonal-encoded re-indexing runs on the device as for float32 tables.
int build_fixed_schedule(std::shared_ptr<Schedule>& out, int steps, const float* beta,
                         const float* eta, float xi, int noise, int act, int lut, double c,
                         int imax, int total_bits, int int_bits, int device) {
  auto s = std::make_shared<Schedule>();
  s->steps = steps;
  s->imax = imax;
  s->device = device;
  s->stride_words = (2 * imax + 1 + 3) & ~3;
  std::vector<float> z(kNoiseLevels);
  noise_levels(noise == PIM_NOISE_GAUSS ? 0 : 1, z.data());
  std::vector<uint32_t> words(static_cast<size_t>(steps) * s->stride_words, 0u);
  for (int t = 0; t < steps; ++t)
    fixed_thresholds(c, beta[t], eta[t], xi, act, lut, total_bits, int_bits, z.data(), imax,
                     words.data() + static_cast<size_t>(t) * s->stride_words);
  CK(cudaMalloc(&s->d_thr, words.size() * 4), "cudaMalloc thresholds");
  CK(cudaMemcpy(s->d_thr, words.data(), words.size() * 4, cudaMemcpyHostToDevice), "upload thresholds");
  if (imax <= kMaxImaxDiag) {
    CK(cudaMalloc(&s->d_thr_diag, static_cast<size_t>(steps) * 1024 * 2), "cudaMalloc diagonal thresholds");
    CK(launch_diag_thresholds(s->d_thr, steps, imax, s->stride_words, 256, s->d_thr_diag, nullptr),
       "diagonal threshold kernel");
    CK(cudaDeviceSynchronize(), "diagonal threshold kernel");
  }
  if (const int K = wide_diag_k(imax)) {
    CK(cudaMalloc(&s->d_thr_dk, static_cast<size_t>(steps) * 4 * K * 2),
       "cudaMalloc wide diagonal thresholds");
    CK(launch_diag_thresholds(s->d_thr, steps, imax, s->stride_words, K, s->d_thr_dk, nullptr),
       "wide diagonal threshold kernel");
    CK(cudaDeviceSynchronize(), "wide diagonal threshold kernel");
    s->dk = K;
  }
  out = s;
  return PIM_OK;
}

double bf16_value(uint16_t bits) {
  const uint32_t u = static_cast<uint32_t>(bits) << 16;
  float f;
  std::memcpy(&f, &u, sizeof f);
  return static_cast<double>(f);
}

// Device block of a real instance for the fixed-point datapath ap_fixed<W, I>: the couplings
// Q(c J) (scale folded in, so the stored values are of order one) as two BF16 images whose
// sum is exact -- the high part rounds Q(c J) to 8 significant bits, the low part holds the
// remaining at most 8 bits -- and the bias Q(c h) as float32 (exact).  The MMA then sums
// integers times 2^-F exactly as long as every row's sum stays below 2^24 units.
int build_fixed_images(pim_instance* p, int W, int I) {
  if (p->d_fix && p->fix_w == W && p->fix_i == I) return PIM_OK;
  const int n = p->n, npad = p->npad;
  const double step = std::ldexp(1.0, I - W);
  const size_t nn = static_cast<size_t>(n) * n;
  std::vector<uint16_t> bits(2 * nn);
  std::vector<float> hq(npad, 0.0f);
  for (int i = 0; i < n; ++i) {
    long long units = 0;
    for (int j = 0; j < n; ++j) {
      const int32_t m = fixed_units(p->c * p->host_J[static_cast<size_t>(i) * n + j], W, I);
      const double v = static_cast<double>(m) * step;
      const uint16_t hb = bf16_bits_rne(v);
      const double lv = v - bf16_value(hb);
      const uint16_t lb = bf16_bits_rne(lv);
      if (bf16_value(lb) != lv)
        return fail(PIM_ERR_UNSUPPORTED, "pim_set_schedule_fixed: Q(c J[%d][%d]) needs more than "
                                         "two BF16 parts", i, j);
      bits[static_cast<size_t>(i) * n + j] = hb;
      bits[nn + static_cast<size_t>(i) * n + j] = lb;
      units += m < 0 ? -m : m;
    }
    const int32_t mh = fixed_units(p->c * p->host_h[i], W, I);
    hq[i] = static_cast<float>(static_cast<double>(mh) * step);
    units += mh < 0 ? -mh : mh;
    if (units >= (1ll << 24))
      return fail(PIM_ERR_UNSUPPORTED, "pim_set_schedule_fixed: row %d of Q(c J) sums to %lld "
                                       "units of 2^-%d (FP32 accumulation exact below 2^24)",
                  i, units, W - I);
  }
  DeviceCtx* ctx = device_ctx(p->device);
  if (!ctx) return fail(PIM_ERR_NOMEM, "pim_set_schedule_fixed: device context");
  const size_t o_lo_bits = align256(nn * 2), o_hi = o_lo_bits + align256(nn * 2);
  const size_t img = static_cast<size_t>(npad) * npad * 2;
  const size_t o_lo = o_hi + align256(img), o_h = o_lo + align256(img);
  void* block = nullptr;
  CK(pool_alloc(&block, o_h + align256(npad * sizeof(float)), p->device, ctx->upload),
     "allocating fixed-point images");
  char* d = static_cast<char*>(block);
  CK(cudaMemcpyAsync(d, bits.data(), nn * 2, cudaMemcpyHostToDevice, ctx->upload), "upload Q(c J)");
  CK(cudaMemcpyAsync(d + o_lo_bits, bits.data() + nn, nn * 2, cudaMemcpyHostToDevice, ctx->upload),
     "upload Q(c J)");
  CK(cudaMemcpyAsync(d + o_h, hq.data(), npad * sizeof(float), cudaMemcpyHostToDevice, ctx->upload),
     "upload Q(c h)");
  CK(staging_after_upload(ctx, p->device), "staging order");
  CK(launch_stage_bf16_image(reinterpret_cast<const uint16_t*>(d), n, npad,
                             reinterpret_cast<uint8_t*>(d + o_hi), ctx->staging),
     "stage high part");
  CK(launch_stage_bf16_image(reinterpret_cast<const uint16_t*>(d + o_lo_bits), n, npad,
                             reinterpret_cast<uint8_t*>(d + o_lo), ctx->staging),
     "stage low part");
  {
    std::lock_guard<std::mutex> lk(ctx->stage_mu);
    CK(cudaEventRecord(p->ready, ctx->staging), "cudaEventRecord");
    p->ready_seq = ++ctx->stage_seq;
  }
  pool_free_after(p->d_fix, p->device, p->done ? p->done->ev : nullptr);
  p->d_fix = d;
  p->d_fix_hi = reinterpret_cast<uint8_t*>(d + o_hi);
  p->d_fix_lo = reinterpret_cast<uint8_t*>(d + o_lo);
  p->d_fix_h = reinterpret_cast<float*>(d + o_h);
  p->fix_w = W;
  p->fix_i = I;
  return PIM_OK;
}

// Schedule of the fixed-point datapath for real couplings: fl32(beta_t) per step and the
// integer tables of the decision (fixed_real_tables), uploaded once.
int build_fixed_real_schedule(std::shared_ptr<Schedule>& out, int steps, const float* beta,
                              const float* eta, float xi, int noise, int act, int lut, int W,
                              int I, int device) {
  auto s = std::make_shared<Schedule>();
  s->steps = steps;
  s->device = device;
  s->xi = xi;
  s->act = act;
  s->lut = lut;
  s->fix_w = W;
  s->fix_i = I;
  std::vector<float> z(kNoiseLevels);
  noise_levels(noise == PIM_NOISE_GAUSS ? 0 : 1, z.data());
  std::vector<int32_t> tau(static_cast<size_t>(1) << W), qz(kNoiseLevels), qeta(steps);
  fixed_real_tables(W, I, act, lut, xi, z.data(), tau.data(), qz.data(), &s->fix_xi);
  for (int t = 0; t < steps; ++t) qeta[t] = fixed_units(static_cast<double>(eta[t]), W, I);
  CK(cudaMalloc(&s->d_bt, steps * 4), "cudaMalloc schedule");
  CK(cudaMalloc(&s->d_eta, steps * 4), "cudaMalloc schedule");
  CK(cudaMalloc(&s->d_z, kNoiseLevels * 4), "cudaMalloc schedule");
  CK(cudaMalloc(&s->d_fix_tau, tau.size() * 4), "cudaMalloc schedule");
  CK(cudaMalloc(&s->d_fix_eta, steps * 4), "cudaMalloc schedule");
  CK(cudaMalloc(&s->d_fix_z, kNoiseLevels * 4), "cudaMalloc schedule");
  CK(cudaMemcpy(s->d_bt, beta, steps * 4, cudaMemcpyHostToDevice), "upload schedule");
  CK(cudaMemcpy(s->d_eta, eta, steps * 4, cudaMemcpyHostToDevice), "upload schedule");
  CK(cudaMemcpy(s->d_z, z.data(), kNoiseLevels * 4, cudaMemcpyHostToDevice), "upload schedule");
  CK(cudaMemcpy(s->d_fix_tau, tau.data(), tau.size() * 4, cudaMemcpyHostToDevice), "upload schedule");
  CK(cudaMemcpy(s->d_fix_eta, qeta.data(), steps * 4, cudaMemcpyHostToDevice), "upload schedule");
  CK(cudaMemcpy(s->d_fix_z, qz.data(), kNoiseLevels * 4, cudaMemcpyHostToDevice), "upload schedule");
  out = s;
  return PIM_OK;
}

}  // namespace

PIM_API int pim_set_schedule_fixed(pim_instance* inst, int steps, const float* beta,
                                   const float* eta, float xi, int noise_kind, int act_kind,
                                   int lut_levels, int total_bits, int int_bits) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_set_schedule_fixed: instance is NULL");
  if (total_bits < 2 || total_bits > 32 || int_bits < 1 || int_bits > total_bits)
    return fail(PIM_ERR_INVALID, "pim_set_schedule_fixed: need 2 <= W <= 32, 1 <= I <= W");
  if (inst->real && inst->n > kMaxNFixedReal)
    return fail(PIM_ERR_UNSUPPORTED, "pim_set_schedule_fixed: real couplings need n <= %d",
                kMaxNFixedReal);
  if (inst->real && total_bits > 16)
    return fail(PIM_ERR_UNSUPPORTED, "pim_set_schedule_fixed: real couplings need W <= 16");
  if (steps < 1 || !beta || !eta) return fail(PIM_ERR_INVALID, "pim_set_schedule_fixed: bad steps/arrays");
  if (!std::isfinite(xi) || xi < 0.0f) return fail(PIM_ERR_INVALID, "pim_set_schedule_fixed: xi must be finite, >= 0");
  if (noise_kind != PIM_NOISE_GAUSS && noise_kind != PIM_NOISE_UNIFORM)
    return fail(PIM_ERR_INVALID, "pim_set_schedule_fixed: unknown noise kind %d", noise_kind);
  if (act_kind != PIM_ACT_TANH && act_kind != PIM_ACT_LUT)
    return fail(PIM_ERR_INVALID, "pim_set_schedule_fixed: unknown activation %d", act_kind);
  if (act_kind == PIM_ACT_LUT && lut_levels < 2)
    return fail(PIM_ERR_INVALID, "pim_set_schedule_fixed: lut_levels must be >= 2");
  if (act_kind == PIM_ACT_TANH) lut_levels = 0;
  for (int t = 0; t < steps; ++t)
    if (!std::isfinite(beta[t]) || beta[t] < 0.0f || !std::isfinite(eta[t]) || eta[t] < 0.0f)
      return fail(PIM_ERR_INVALID, "pim_set_schedule_fixed: beta/eta[%d] must be finite and >= 0", t);
  if (inst->real) {
    const int rc = build_fixed_images(inst, total_bits, int_bits);
    if (rc != PIM_OK) return rc;
  }
  const int imax = inst->real ? -1 : table_imax(inst);
  std::string key = schedule_key(steps, beta, eta, xi, noise_kind, act_kind, lut_levels, inst->c,
                                 imax, inst->device);
  key += inst->real ? "fixedreal" : "fixed";
  key.append(reinterpret_cast<const char*>(&total_bits), sizeof total_bits);
  key.append(reinterpret_cast<const char*>(&int_bits), sizeof int_bits);
  std::shared_ptr<Schedule> s;
  {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    auto it = g_sched_cache.find(key);
    if (it != g_sched_cache.end()) s = it->second.lock();
  }
  if (!s) {
    const int rc = inst->real
                       ? build_fixed_real_schedule(s, steps, beta, eta, xi, noise_kind, act_kind,
                                                   lut_levels, total_bits, int_bits, inst->device)
                       : build_fixed_schedule(s, steps, beta, eta, xi, noise_kind, act_kind,
                                              lut_levels, inst->c, imax, total_bits, int_bits,
                                              inst->device);
    if (rc != PIM_OK) return rc;
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched_cache[key] = s;
  }
  if (inst->done) cudaEventSynchronize(inst->done->ev);
  inst->sched = s;
  return PIM_OK;
}

namespace {

// Tile plan of the large-N kernel for one instance.
struct BigPlan {
  int nt = 0;                // output spins per CTA (64 or 128)
  int op = kBigFp8;          // operand variant (BigOp)
  int tiles_per_launch = 0;  // 128-replica tiles per cooperative launch
  int launches = 0;
  double us_per_sweep = 0.0;  // model estimate
};

// Per-sweep time model of the large-N kernel.  Every CTA streams K-blocks of 128 x 128 B
// spins (128 FP8, 64 BF16 or 256 E2M1 spins per row) plus, unless they are resident, nt x
// 128 B of couplings; a K-block costs the larger of its ingest time at the per-SM bulk-copy
// rate (about 64 GB/s per SM when all SMs stream, as measured for this kernel on GB300) and
// its MMA time at the per-SM tensor rate (1889 TFLOP/s BF16, twice that for FP8, four times
// for FP4, over 152 SMs); replica tiles that do not fit the co-resident grid run as further
// launches, each with its own ~3 us grid barrier per sweep.
// ---- Autotuning: measured kernel times per shape class -----------------------------------
// pim_batch_create (mode 1) times, on the batch's own instances, every shape class it has
// not seen on this device before: the persistent mid-N kernel per (npad, decision path)
// unit, the fused kernel per unit, and the large-N kernel per (real, npad, replica tiles,
// NT) instance sweep.  The router and the large-N tile plan use a measured time wherever
// the cache has one and the analytic model otherwise.  Entries are kept per process and,
// when PIM_TUNE_CACHE names a file, appended to it and read back by later processes.
std::mutex g_tune_mu;
std::map<std::string, double> g_tune;  // key -> microseconds
bool g_tune_loaded = false;
std::atomic<int> g_tune_mode{1};
thread_local int t_force_nt = 0;            // measurement of one large-N tile width
thread_local int t_force_op = -1;           //   and operand variant
thread_local bool t_model_routes = false;   // measurement runs: no measured overrides

std::string device_name(int dev) {
  static std::mutex mu;
  static std::map<int, std::string> names;
  std::lock_guard<std::mutex> lk(mu);
  auto it = names.find(dev);
  if (it != names.end()) return it->second;
  cudaDeviceProp prop{};
  std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
  for (char& ch : name)
    if (ch == ' ' || ch == '|') ch = '_';
  names[dev] = name;
  return name;
}

std::string tune_key(const char* what, int a, int b, int c = 0, int d = 0) {
  int dev = 0;
  cudaGetDevice(&dev);
  char buf[160];
  std::snprintf(buf, sizeof buf, "%s|%s|%d|%d|%d|%d", device_name(dev).c_str(), what, a, b, c, d);
  return buf;
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("PIM_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    char key[200];
    double us = 0.0;
    if (std::sscanf(line, "%199s %lf", key, &us) == 2 && us > 0.0) g_tune[key] = us;
  }
  std::fclose(f);
}

bool tune_lookup(const std::string& key, double* us) {
  if (t_model_routes || g_tune_mode.load() == 0) return false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *us = it->second;
  return true;
}

bool tune_known(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  return g_tune.count(key) != 0;
}

void tune_store(const std::string& key, double us) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  g_tune[key] = us;
  const char* path = std::getenv("PIM_TUNE_CACHE");
  if (path && *path) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%s %.6g\n", key.c_str(), us);
      std::fclose(f);
    }
  }
}

constexpr double kIngestBytesPerUs = 64e3;
constexpr double kBf16FlopsPerUs = 1889e6 / 152;

int plan_big(int n, int npad, int R, bool real, bool fp4, int stride_words, BigPlan* out) {
  const int tiles_total = (R + 127) / 128;
  const int base = real ? kBigBf16 : kBigFp8;
  const std::pair<int, int> cands[3] = {{64, base}, {128, base}, {64, kBigFp4}};
  BigPlan best;
  for (const auto& cand : cands) {
    const int nt = cand.first, op = cand.second;
    if (op == kBigFp4 && !fp4) continue;
    if (npad % nt || (t_force_nt && nt != t_force_nt) || (t_force_op >= 0 && op != t_force_op))
      continue;
    const int ncb = npad / nt;
    const int cap = sweep_big_max_blocks(nt, op, npad, stride_words);
    if (cap < ncb) continue;
    BigPlan p;
    p.nt = nt;
    p.op = op;
    p.tiles_per_launch = std::min(tiles_total, cap / ncb);
    p.launches = (tiles_total + p.tiles_per_launch - 1) / p.tiles_per_launch;
    double measured = 0.0;
    if (tune_lookup(tune_key("big", op, npad, tiles_total, nt), &measured)) {
      p.us_per_sweep = measured;
      if (best.nt == 0 || p.us_per_sweep < best.us_per_sweep) best = p;
      continue;
    }
    const int spins_per_kb = op == kBigFp4 ? 256 : (real ? 64 : 128);
    const double rate = kBf16FlopsPerUs * (op == kBigFp4 ? 4 : (real ? 1 : 2));
    const double bytes = 128.0 * 128 + (op == kBigFp4 ? 0.0 : nt * 128.0);
    const double flops = 2.0 * 128 * nt * spins_per_kb;
    const double per_kb = std::max(bytes / kIngestBytesPerUs, flops / rate);
    p.us_per_sweep = p.launches * ((npad / spins_per_kb) * per_kb + 3.0);
    if (best.nt == 0 || p.us_per_sweep < best.us_per_sweep) best = p;
  }
  if (best.nt == 0)
    return fail(PIM_ERR_UNSUPPORTED, "anneal: n = %d needs more co-resident CTAs than the device holds", n);
  *out = best;
  return PIM_OK;
}

// Large-N anneal of one instance: the replicas are split into groups of tiles that fit the
// co-resident grid (each group is an independent cooperative launch); per launch scratch
// (two spin images, energy accumulators, barrier words) comes from the stream-ordered pool.
// Bytes of one large-N spin image of rpad replica rows.
size_t big_image_bytes(int rpad, int npad, int op) {
  const size_t cells = static_cast<size_t>(rpad) * npad;
  return op == kBigFp4 ? cells / 2 : (op == kBigBf16 ? 2 * cells : cells);
}

int launch_big(const Problem& P, bool real, int t_begin, int sweeps, uint64_t seed, bool cont,
               int* d_err, char* scratch, int* launches, cudaStream_t st) {
  BigPlan plan;
  const int rc = plan_big(P.n, P.npad, P.R, real, P.jimg4 != nullptr, P.stride_words, &plan);
  if (rc != PIM_OK) return rc;
  const BigSmem smem = sweep_big_smem(plan.nt, plan.op, P.npad, P.stride_words);
  if (!smem.ok) return fail(PIM_ERR_UNSUPPORTED, "anneal: large-N variant does not fit");
  const int ncb = P.npad / plan.nt;
  const int tiles_total = (P.R + 127) / 128;
  for (int tile0 = 0; tile0 < tiles_total; tile0 += plan.tiles_per_launch) {
    const int tiles = std::min(plan.tiles_per_launch, tiles_total - tile0);
    const int rpad = tiles * 128;
    const size_t img_bytes = big_image_bytes(rpad, P.npad, plan.op);
    const size_t energy_bytes = sizeof(float) * 3 * rpad;
    const size_t bytes = 2 * img_bytes + energy_bytes + 256;
    char* d = scratch;
    if (!scratch)
      CK(run_alloc(reinterpret_cast<void**>(&d), bytes, st), "cudaMallocAsync large-N scratch");
    CK(cudaMemsetAsync(d + 2 * img_bytes, 0, energy_bytes + 256, st), "clear large-N scratch");
    BigLaunch L{};
    L.P = P;
    L.s_img[0] = reinterpret_cast<uint8_t*>(d);
    L.s_img[1] = reinterpret_cast<uint8_t*>(d + img_bytes);
    L.j4 = plan.op == kBigFp4 ? P.jimg4 : nullptr;
    L.stages = smem.stages;
    L.tab_smem = smem.tab_smem;
    L.energy = reinterpret_cast<float*>(d + 2 * img_bytes);
    L.bar = reinterpret_cast<unsigned int*>(d + 2 * img_bytes + energy_bytes);
    L.nt = plan.nt;
    L.rbase = tile0 * 128;
    L.rpad = rpad;
    L.ncb = ncb;
    L.t_begin = t_begin;
    L.sweeps = sweeps;
    L.cont = cont ? 1 : 0;
    philox_round_keys(seed, L.round_keys);
    L.err = d_err;
    L.wait_ns = g_wait_ns.load();
    L.inject = g_inject.load();
    CK(launch_sweep_big(L, plan.nt, plan.op, tiles * ncb, st), "large-N sweep kernel");
    if (!scratch) CK(cudaFreeAsync(d, st), "cudaFreeAsync large-N scratch");
    if (launches) ++*launches;
  }
  return PIM_OK;
}

// Kernel of each instance of a batch: kFused (n <= 256, one CTA per 128-replica panel with
// J resident in shared memory), kMid (integer n <= 1024, persistent, J streamed from L2) or
// kBig (n > 256, cooperative grid per instance).  Integer instances with 256 < n <= 1024
// can run on kMid or kBig; the choice minimises a time model of the batch:
//   kMid   a unit (instance, 128-replica panel) takes about (chunks + 1) x max(epilogue of
//          a 128 x 128 chunk, ingest of the chunk's 128 x npad couplings) per sweep; the
//          persistent grid finishes after max(longest unit, total / SMs);
//   kBig   plan_big's per-sweep estimate, launches run one after another.
// Starting from every eligible instance on kMid, the largest instances move to kBig while
// that lowers the modelled time (a lone large instance fills more SMs on kBig).
enum Route { kFused = 0, kMid = 1, kBig = 2 };
constexpr double kEpiUsPerChunk = 2.0;  // 128 x 128 decisions at ~8.5e9 spin updates/s/SM

double mid_unit_us(int npad) {
  const int chunks = npad / 128;
  const double ingest = 128.0 * npad / kIngestBytesPerUs;
  return (chunks + 1) * std::max(kEpiUsPerChunk, ingest);
}

// Decision path a mid-N unit of instance p takes (0 general table, else the diagonal K).
int mid_path(const pim_instance* p) {
  if (p->diag && p->sched && p->sched->d_thr_diag) return 256;
  if (p->d_img5 && p->sched &&
      (p->dk5 == 256 ? p->sched->d_thr_diag != nullptr : p->sched->dk == p->dk5))
    return p->dk5;
  return 0;
}

// Mid-N unit time of instance p: measured when the cache has it, else the model.
double mid_unit_us(const pim_instance* p) {
  double us = 0.0;
  if (tune_lookup(tune_key("mid", p->npad, mid_path(p)), &us)) return us;
  return mid_unit_us(p->npad);
}

int route_batch(pim_instance* const* insts, const int* replicas, int count, int flags,
                std::vector<int>& route) {
  route.assign(count, kFused);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int mid_blocks = std::max(1, std::min(sms, sweep_mid_max_blocks()));
  std::vector<int> eligible;
  for (int k = 0; k < count; ++k) {
    const pim_instance* p = insts[k];
    if (p->real) {
      route[k] = p->n <= kMaxNTensor ? kFused : kBig;
    } else if (p->n <= kMaxNTensor) {
      route[k] = (flags & PIM_PATH_MID) ? kMid : kFused;
      // measured: a fused unit runs two CTAs per SM, a mid-N unit one, so the per-SM
      // throughputs compare fused_us / 2 with mid_us
      double fused_us = 0.0, mid_us = 0.0;
      if (route[k] == kFused && p->npad <= sweep_mid_max_npad() &&
          p->sched->imax <= kMaxImaxTensor &&
          tune_lookup(tune_key("fused", p->npad, p->diag ? 1 : 0), &fused_us) &&
          tune_lookup(tune_key("mid", p->npad, mid_path(p)), &mid_us) && mid_us < 0.5 * fused_us)
        route[k] = kMid;
    } else if (p->npad > sweep_mid_max_npad() || (flags & PIM_PATH_BIG)) {
      route[k] = kBig;
    } else {
      route[k] = kMid;
      if (!(flags & PIM_PATH_MID)) eligible.push_back(k);
    }
  }
  if (eligible.empty()) return PIM_OK;
  // time model (per sweep) of the kMid launch and of the instances moved to kBig
  double mid_total = 0.0, mid_max = 0.0;
  for (int k = 0; k < count; ++k)
    if (route[k] == kMid) {
      const double u = mid_unit_us(insts[k]);
      mid_total += u * ((replicas[k] + 127) / 128);
      mid_max = std::max(mid_max, u);
    }
  std::sort(eligible.begin(), eligible.end(), [&](int a, int b) {
    return static_cast<long long>(insts[a]->npad) * replicas[a] >
           static_cast<long long>(insts[b]->npad) * replicas[b];
  });
  double big_total = 0.0;
  for (size_t e = 0; e < eligible.size(); ++e) {
    const int k = eligible[e];
    BigPlan plan;
    const bool fp4 = insts[k]->d_img4 != nullptr && !(flags & PIM_PATH_FP8);
    if (plan_big(insts[k]->n, insts[k]->npad, replicas[k], false, fp4, insts[k]->sched->stride_words,
                 &plan) != PIM_OK)
      continue;
    const double u = mid_unit_us(insts[k]);
    const double rest_total = mid_total - u * ((replicas[k] + 127) / 128);
    double rest_max = 0.0;
    for (size_t f2 = e + 1; f2 < eligible.size(); ++f2)
      rest_max = std::max(rest_max, mid_unit_us(insts[eligible[f2]]));
    for (int j = 0; j < count; ++j)
      if (route[j] == kMid && insts[j]->n <= kMaxNTensor)
        rest_max = std::max(rest_max, mid_unit_us(insts[j]));
    const double before = big_total + std::max(mid_max, mid_total / mid_blocks);
    const double after = big_total + plan.us_per_sweep + std::max(rest_max, rest_total / mid_blocks);
    if (after >= before) break;
    route[k] = kBig;
    big_total += plan.us_per_sweep;
    mid_total = rest_total;
    mid_max = rest_max;
  }
  return PIM_OK;
}

// fused 0-5, mid-N general path 6, mid-N diagonal-encoded 7
constexpr int kGroups = 8, kMidGroup = 6, kMidDiagGroup = 7;


// Launch description of one batch: problem descriptors, the unit lists of each kernel group
// (fused: npad 128 | 256 x diagonal-encoded | general bias | real-valued; persistent mid-N),
// the large-N instances, and the layout of the one device buffer that holds them.
struct BatchPlan {
  std::vector<Problem> probs;
  std::vector<int> route;
  std::vector<WorkItem> work[kGroups];
  int maxR = 0, max_words = 0, stride_max = 4;
  size_t work_off[kGroups] = {};
  size_t ready_off[kGroups] = {};  // fused groups: chunked-queue counter and ready flags
  size_t init_off = 0, init_bytes = 0, counters_off = 0, total = 0;
  size_t big_scratch = 0;  // largest scratch one large-N launch of this batch needs
};

// Argument checks shared by pim_anneal, pim_anneal_batch and pim_batch_run.
int check_batch(pim_instance* const* insts, int count, const int* replicas, int t_begin,
                int sweeps, const double* targets, int flags, bool check_steps) {
  if (!insts || count < 1 || !replicas) return fail(PIM_ERR_INVALID, "anneal: empty batch");
  if (sweeps < 0 || t_begin < 0) return fail(PIM_ERR_INVALID, "anneal: negative t_begin/sweeps");
  if (flags & ~(PIM_CONTINUE | PIM_PATH_FP32REF | PIM_PATH_MID | PIM_PATH_BIG | PIM_RESULTS_TO_HOST |
                PIM_PATH_FP8))
    return fail(PIM_ERR_INVALID, "anneal: unknown flags");
  const bool cont = (flags & PIM_CONTINUE) != 0;
  const bool ref = (flags & PIM_PATH_FP32REF) != 0;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int k = 0; k < count; ++k) {
    pim_instance* p = insts[k];
    if (!p) return fail(PIM_ERR_INVALID, "anneal: instance %d is NULL", k);
    if (p->device != dev) return fail(PIM_ERR_INVALID, "anneal: instance %d lives on device %d", k, p->device);
    if (!p->sched) return fail(PIM_ERR_STATE, "anneal: instance %d has no schedule", k);
    if (replicas[k] < 1) return fail(PIM_ERR_INVALID, "anneal: replicas[%d] = %d < 1", k, replicas[k]);
    if (check_steps && static_cast<long long>(t_begin) + sweeps > p->sched->steps)
      return fail(PIM_ERR_INVALID, "anneal: t_begin + sweeps = %lld exceeds the %d schedule steps",
                  static_cast<long long>(t_begin) + sweeps, p->sched->steps);
    if (cont && (!p->has_results || p->R != replicas[k]))
      return fail(PIM_ERR_STATE, "anneal: CONTINUE needs a previous run with the same replicas");
    if (ref && p->real)
      return fail(PIM_ERR_UNSUPPORTED, "anneal: the plain path takes integer couplings only");
    if (!ref && !p->real && p->n <= kMaxNTensor && !(flags & PIM_PATH_MID) &&
        p->sched->imax > kMaxImaxTensor)
      return fail(PIM_ERR_UNSUPPORTED, "anneal: field range %d too large for the fused kernel",
                  p->sched->imax);
    for (int j = 0; j < k; ++j)
      if (insts[j] == p) return fail(PIM_ERR_INVALID, "anneal: instance listed twice");
    if (targets && std::isnan(targets[k]) == false && !std::isfinite(targets[k]))
      return fail(PIM_ERR_INVALID, "anneal: target %d not finite", k);
  }
  return PIM_OK;
}

// Streaming multiprocessors of the current device.
int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, sms);
}

// Host side of a batch: descriptors (instances must have their result buffers), routing,
// unit lists and the device buffer layout.
int build_plan(pim_instance* const* insts, int count, const int* replicas, const uint32_t* ids,
               const double* targets, int flags, size_t init_bytes, BatchPlan& B) {
  const bool ref = (flags & PIM_PATH_FP32REF) != 0;
  B.probs.assign(count, Problem{});
  for (int k = 0; k < count; ++k) {
    pim_instance* p = insts[k];
    Problem& P = B.probs[k];
    P.jimg = p->d_img;
    P.jimg4 = (flags & PIM_PATH_FP8) ? nullptr : p->d_img4;
    P.jf = p->d_jf;
    P.j8 = p->d_J8;
    P.h = p->d_h;
    P.thr = p->sched->d_thr;
    P.thr_diag = p->sched->d_thr_diag;
    P.diag_img = p->diag ? 1 : 0;
    P.best_E = p->d_bestE;
    P.final_E = p->d_finalE;
    P.best_t = p->d_bestT;
    P.first_hit = p->d_first;
    P.best_bits = p->d_best_bits;
    P.cur_bits = p->d_cur_bits;
    P.n = p->n;
    P.npad = p->npad;
    P.words = p->words;
    P.imax = p->sched->imax;
    P.stride_words = p->sched->stride_words;
    P.R = replicas[k];
    P.q = ids ? ids[k] : static_cast<uint32_t>(k);
    P.hf = p->d_hf;
    P.sched_b = p->sched->d_bt;
    P.sched_eta = p->sched->d_eta;
    P.zlev = p->sched->d_z;
    P.xi = p->sched->xi;
    P.act = p->sched->act;
    P.lut_levels = p->sched->lut;
    if (p->real && p->sched->fix_w > 0) {
      P.jimg = p->d_fix_hi;
      P.jimg_lo = p->d_fix_lo;
      P.hf = p->d_fix_h;
      P.fix_w = p->sched->fix_w;
      P.fix_f = p->sched->fix_w - p->sched->fix_i;
      P.fix_tau = p->sched->d_fix_tau;
      P.fix_eta = p->sched->d_fix_eta;
      P.fix_z = p->sched->d_fix_z;
      P.fix_xi = p->sched->fix_xi;
    }
    const double tg = targets ? targets[k] : NAN;
    P.has_target = std::isnan(tg) ? 0 : 1;
    P.target = std::isnan(tg) ? 0 : static_cast<long long>(std::floor(tg));
    P.target_f = std::isnan(tg) ? 0.0 : tg;
    B.maxR = std::max(B.maxR, replicas[k]);
    B.max_words = std::max(B.max_words, p->words);
    B.stride_max = std::max(B.stride_max, p->sched->stride_words);
  }
  B.route.assign(count, kFused);
  if (!ref) {
    const int rc = route_batch(insts, replicas, count, flags, B.route);
    if (rc != PIM_OK) return rc;
  }
  // Mid-N units decide from the diagonal-encoded image when the instance has one: the
  // E4M3 image with 256 on the diagonal, or the E5M2 image with dk5 and its schedule's table.
  for (int k = 0; k < count && !ref; ++k) {
    if (B.route[k] != kMid) continue;
    const pim_instance* p = insts[k];
    Problem& P = B.probs[k];
    if (p->diag && p->sched->d_thr_diag) {
      P.dk = 256;
    } else if (p->d_img5) {
      const uint32_t* tab = p->dk5 == 256 ? p->sched->d_thr_diag
                                          : (p->sched->dk == p->dk5 ? p->sched->d_thr_dk : nullptr);
      if (tab) {
        P.jimg = p->d_img5;
        P.thr_diag = tab;
        P.dk = p->dk5;
        P.e5m2 = 1;
      }
    }
  }
  for (auto& w : B.work) w.clear();
  for (int k = 0; k < count && !ref; ++k) {
    if (B.route[k] == kBig) {
      BigPlan plan;
      const Problem& P = B.probs[k];
      const int rc = plan_big(P.n, P.npad, P.R, insts[k]->real, P.jimg4 != nullptr, P.stride_words, &plan);
      if (rc != PIM_OK) return rc;
      const int rpad = plan.tiles_per_launch * 128;
      B.big_scratch = std::max(B.big_scratch, 2 * big_image_bytes(rpad, P.npad, plan.op) +
                                                  sizeof(float) * 3 * rpad + 256);
      continue;
    }
    const int g = B.route[k] == kMid ? (B.probs[k].dk > 0 ? kMidDiagGroup : kMidGroup)
                                     : (insts[k]->npad <= 128 ? 0 : 1) +
                                           (insts[k]->real ? 4 : (insts[k]->diag ? 0 : 2));
    for (int rb = 0; rb < replicas[k]; rb += 128) B.work[g].push_back({k, rb});
  }
  // persistent launch: largest units first so the last wave is short
  for (int g : {kMidGroup, kMidDiagGroup})
    std::stable_sort(B.work[g].begin(), B.work[g].end(), [&](const WorkItem& a, const WorkItem& b) {
      return insts[a.prob]->npad > insts[b.prob]->npad;
    });
  size_t off = align256(B.probs.size() * sizeof(Problem));
  for (int g = 0; g < kGroups; ++g) {
    B.work_off[g] = off;
    off += B.work[g].size() * sizeof(WorkItem);
    if (g < 4 && !B.work[g].empty()) {
      off = align256(off);
      B.ready_off[g] = off;
      off += (B.work[g].size() + 1) * sizeof(unsigned int);
    }
  }
  B.init_off = align256(off);
  B.init_bytes = init_bytes;
  B.counters_off = align256(B.init_off + init_bytes);
  B.total = B.counters_off + 256;
  return PIM_OK;
}

void pack_plan(const BatchPlan& B, const int8_t* init_spins, std::vector<char>& h) {
  h.assign(B.total, 0);
  std::memcpy(h.data(), B.probs.data(), B.probs.size() * sizeof(Problem));
  for (int g = 0; g < kGroups; ++g)
    if (!B.work[g].empty())
      std::memcpy(h.data() + B.work_off[g], B.work[g].data(), B.work[g].size() * sizeof(WorkItem));
  if (B.init_bytes) std::memcpy(h.data() + B.init_off, init_spins, B.init_bytes);
}

// Event record that also works inside stream capture: there it becomes an event-record
// node of the graph, so the host can time and wait on replays.
cudaError_t record_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, st);
}

// Every device operation of one run of a batch, in stream order: initial spins (unless
// continuing), the timer start, the kernel groups, the large-N launches, the timer stop.
// `big_scratch` (may be null) is a preallocated scratch of B.big_scratch bytes.
int enqueue_plan(const BatchPlan& B, char* d_buf, char* big_scratch, pim_instance* const* insts,
                 int count, int t_begin, int sweeps, uint64_t seed, bool cont, bool ref,
                 LaunchTimer* timer, int* d_err, int* launches, cudaStream_t st) {
  const Problem* d_probs = reinterpret_cast<const Problem*>(d_buf);
  const int8_t* d_init = B.init_bytes ? reinterpret_cast<const int8_t*>(d_buf + B.init_off) : nullptr;
  int nl = 0;
  if (!cont) {
    CK(launch_init_bits(d_probs, count, B.maxR, B.max_words, d_init, static_cast<uint32_t>(seed),
                        static_cast<uint32_t>(seed >> 32), st),
       "init kernel");
    ++nl;
  }
  if (ref) {
    float *d_S = nullptr, *d_I = nullptr;
    size_t maxRn = 0;
    for (int k = 0; k < count; ++k)
      maxRn = std::max(maxRn, static_cast<size_t>(B.probs[k].R) * insts[k]->n);
    CK(run_alloc(reinterpret_cast<void**>(&d_S), maxRn * 4, st), "cudaMallocAsync S");
    CK(run_alloc(reinterpret_cast<void**>(&d_I), maxRn * 4, st), "cudaMallocAsync I");
    CK(record_event(timer->start, st), "cudaEventRecord");
    CK(launch_ref_anneal(B.probs.data(), d_probs, count, t_begin, sweeps, static_cast<uint32_t>(seed),
                         static_cast<uint32_t>(seed >> 32), cont ? 1 : 0, d_S, d_I, d_err, st),
       "plain path");
    CK(record_event(timer->stop, st), "cudaEventRecord");
    CK(cudaFreeAsync(d_S, st), "cudaFreeAsync");
    CK(cudaFreeAsync(d_I, st), "cudaFreeAsync");
    nl += 2 * (sweeps + 1) * count;
  } else {
    CK(record_event(timer->start, st), "cudaEventRecord");
    for (int g = 0; g < kGroups; ++g) {
      if (B.work[g].empty()) continue;
      Launch L{};
      L.probs = d_probs;
      L.work = reinterpret_cast<const WorkItem*>(d_buf + B.work_off[g]);
      L.nwork = static_cast<int>(B.work[g].size());
      L.t_begin = t_begin;
      L.sweeps = sweeps;
      L.key_lo = static_cast<uint32_t>(seed);
      L.key_hi = static_cast<uint32_t>(seed >> 32);
      philox_round_keys(seed, L.round_keys);
      L.cont = cont ? 1 : 0;
      L.stride_words_max = B.stride_max;
      L.err = d_err;
      L.wait_ns = g_wait_ns.load();
      L.inject = g_inject.load();
      L.next = reinterpret_cast<unsigned int*>(d_buf + B.counters_off);
      int blocks = L.nwork;
      if (g < 4) {
        // More units than the two CTAs per SM that run at once: cut every unit's sweeps into
        // chunks and let persistent CTAs take them from a queue, so that no SM idles or
        // runs a lone CTA while others finish a last partial wave (about kQueueDepth
        // segments per CTA bound the imbalance at the end to a small share of the run).
        constexpr int kQueueDepth = 24;
        const int ctas = 2 * device_sms();
        if (L.nwork > ctas && sweeps > 0) {
          L.chunks = std::min(sweeps, (kQueueDepth * ctas + L.nwork - 1) / L.nwork);
          L.ready = reinterpret_cast<unsigned int*>(d_buf + B.ready_off[g]);
          blocks = ctas;
        }
      }
      if (g == kMidGroup || g == kMidDiagGroup) {
        const int blocks = std::min(L.nwork, sweep_mid_max_blocks());
        if (blocks < 1) return fail(PIM_ERR_CUDA, "anneal: mid-N kernel cannot be resident");
        CK(launch_sweep_mid(L, blocks, st, g == kMidDiagGroup), "persistent mid-N sweep kernel");
      } else if (g >= 4) {
        CK(launch_sweep_float(L, (g & 1) ? 256 : 128, L.nwork, st), "real-valued sweep kernel");
      } else {
        CK(launch_sweep_tc(L, (g & 1) ? 256 : 128, blocks, st, g < 2), "fused sweep kernel");
      }
      ++nl;
    }
    for (int k = 0; k < count; ++k) {
      if (B.route[k] != kBig) continue;
      int n_big = 0;
      const int rc = launch_big(B.probs[k], insts[k]->real, t_begin, sweeps, seed, cont, d_err,
                                big_scratch, &n_big, st);
      if (rc != PIM_OK) return rc;
      nl += n_big;
    }
    CK(record_event(timer->stop, st), "cudaEventRecord");
  }
  if (launches) *launches = nl;
  return PIM_OK;
}

// Makes st wait for the staging of every instance (all on one device): one wait on the
// ready event recorded last, which follows every earlier one on the staging stream.
cudaError_t wait_staged(pim_instance* const* insts, int count, cudaStream_t st) {
  const pim_instance* last = nullptr;
  for (int k = 0; k < count; ++k)
    if (!last || insts[k]->ready_seq > last->ready_seq) last = insts[k];
  return last ? cudaStreamWaitEvent(st, last->ready, 0) : cudaSuccess;
}

// Prerequisites of a run on stream st: staged inputs, float32 couplings for the plain path,
// result buffers for the replica counts.
int prepare_instances(pim_instance* const* insts, int count, const int* replicas, bool ref,
                      cudaStream_t st) {
  CK(wait_staged(insts, count, st), "cudaStreamWaitEvent");  // inputs staged
  for (int k = 0; k < count; ++k) {
    pim_instance* p = insts[k];
    if (ref && !p->d_jf) {  // float32 couplings of the plain path, built on first use
      void* d = nullptr;
      CK(pool_alloc(&d, static_cast<size_t>(p->n) * p->n * sizeof(float), p->device, st),
         "allocating float32 J");
      p->d_jf = static_cast<float*>(d);
      CK(launch_stage_f32(p->d_J8, p->n, p->d_jf, st), "stage float32 J");
    }
    const int rc = ensure_results(p, replicas[k], st);
    if (rc != PIM_OK) return rc;
  }
  return PIM_OK;
}

// Pinned host buffer for the instance's result block (PIM_RESULTS_TO_HOST), with its device
// address when the GPU can write it directly.
int ensure_host_copy(pim_instance* p) {
  if (p->h_res_cap >= p->res_bytes) return PIM_OK;
  // the previous block may still be the target of an earlier run's copy
  if (p->h_res) {
    if (p->done) CK(cudaEventSynchronize(p->done->ev), "cudaEventSynchronize");
    give_pinned(p->h_res, p->h_res_cap);
  }
  p->h_res_cap = pinned_class(p->res_bytes);
  p->h_res = static_cast<char*>(take_pinned(p->h_res_cap));
  p->h_res_dev = nullptr;
  if (!p->h_res) {
    p->h_res_cap = 0;
    return fail(PIM_ERR_NOMEM, "pinned results buffer of %zu bytes", p->res_bytes);
  }
  if (cudaHostGetDevicePointer(&p->h_res_dev, p->h_res, 0) != cudaSuccess) {
    cudaGetLastError();
    p->h_res_dev = nullptr;
  }
  return PIM_OK;
}

// End of a run on st: results to host (unless `copied` says a gather launch already did
// it), the error-word mirror, one completion event for all the run's instances.
int finish_run(pim_instance* const* insts, int count, const int* replicas,
               const std::shared_ptr<LaunchTimer>& timer, cudaStream_t st, bool to_host,
               bool copied = false) {
  for (int k = 0; k < count && to_host && !copied; ++k) {
    pim_instance* p = insts[k];
    const int rc = ensure_host_copy(p);
    if (rc != PIM_OK) return rc;
    CK(cudaMemcpyAsync(p->h_res, p->d_res, p->res_bytes, cudaMemcpyDeviceToHost, st), "results to host");
  }
  ErrWord* w = error_word(insts[0]->device);
  if (w && w->h_dev) CK(launch_mirror_word(w->d, w->h_dev, st), "error word mirror");
  auto done = std::make_shared<RunEvent>();
  done->device = insts[0]->device;
  CK(take_event(done->device, &done->ev), "cudaEventCreate");
  CK(cudaEventRecord(done->ev, st), "cudaEventRecord");
  for (int k = 0; k < count; ++k) {
    insts[k]->h_res_valid = to_host;
    insts[k]->R = replicas[k];
    insts[k]->has_results = true;
    insts[k]->timer = timer;
    insts[k]->done = done;
  }
  return PIM_OK;
}

// Results to host: one gather launch on st writes every instance's result block into its
// mapped pinned buffer, whatever the instance count (a single instance included): a copy
// command per instance would fill the launch queue behind a long run, and copy-engine
// commands from different streams queue behind each other.  *copied = false when some
// buffer has no device address; finish_run then copies instance by instance instead.

int gather_results(pim_instance* const* insts, int count, cudaStream_t st, bool* copied) {
  *copied = false;
  std::vector<CopyJob> jobs;
  for (int k = 0; k < count; ++k) {
    const int rc = ensure_host_copy(insts[k]);
    if (rc != PIM_OK) return rc;
    if (!insts[k]->h_res_dev) return PIM_OK;
    jobs.push_back(CopyJob{insts[k]->d_res, insts[k]->h_res_dev, insts[k]->res_bytes});
  }
  CopyJob* d_jobs = nullptr;
  const size_t bytes = jobs.size() * sizeof(CopyJob);
  CK(run_alloc(reinterpret_cast<void**>(&d_jobs), bytes, st), "cudaMallocAsync gather table");
  CK(upload_async(d_jobs, jobs.data(), bytes, st), "upload gather table");
  CK(launch_gather_copy(d_jobs, static_cast<int>(jobs.size()), st), "results gather");
  CK(cudaFreeAsync(d_jobs, st), "cudaFreeAsync gather table");
  *copied = true;
  return PIM_OK;
}

int anneal_impl(pim_instance* const* insts, int count, const int* replicas, int t_begin,
                int sweeps, uint64_t seed, const uint32_t* ids, const double* targets,
                const int8_t* init_spins, int flags, cudaStream_t st, float* d_fields = nullptr) {
  int rc = check_batch(insts, count, replicas, t_begin, sweeps, targets, flags, true);
  if (rc != PIM_OK) return rc;
  if (init_spins && count != 1) return fail(PIM_ERR_INVALID, "anneal: init spins need one instance");
  const bool cont = (flags & PIM_CONTINUE) != 0;
  const bool ref = (flags & PIM_PATH_FP32REF) != 0;
  if ((rc = prepare_instances(insts, count, replicas, ref, st)) != PIM_OK) return rc;
  int dev = 0;
  cudaGetDevice(&dev);
  int* d_err = device_error_word(dev);
  if (!d_err) return fail(PIM_ERR_NOMEM, "anneal: error word allocation failed");
  BatchPlan B;
  const size_t init_bytes = init_spins ? static_cast<size_t>(replicas[0]) * insts[0]->n : 0;
  if ((rc = build_plan(insts, count, replicas, ids, targets, flags, init_bytes, B)) != PIM_OK) return rc;
  if (d_fields) B.probs[0].fields_out = d_fields;
  char* d_buf = nullptr;
  CK(run_alloc(reinterpret_cast<void**>(&d_buf), B.total, st), "cudaMallocAsync launch buffer");
  std::vector<char> h_buf;
  pack_plan(B, init_spins, h_buf);
  CK(upload_async(d_buf, h_buf.data(), B.total, st), "upload launch buffer");
  auto timer = std::make_shared<LaunchTimer>();
  CK(cudaEventCreate(&timer->start), "cudaEventCreate");
  CK(cudaEventCreate(&timer->stop), "cudaEventCreate");
  rc = enqueue_plan(B, d_buf, nullptr, insts, count, t_begin, sweeps, seed, cont, ref, timer.get(),
                    d_err, nullptr, st);
  if (rc != PIM_OK) return rc;
  CK(cudaFreeAsync(d_buf, st), "cudaFreeAsync launch buffer");
  const bool to_host = (flags & PIM_RESULTS_TO_HOST) != 0;
  bool copied = false;
  if (to_host && (rc = gather_results(insts, count, st, &copied)) != PIM_OK)
    return rc;
  return finish_run(insts, count, replicas, timer, st, to_host, copied);
}

}  // namespace

namespace {

// Device time (ms) of the sweep kernels of `sweeps` sweeps of a clone of `rep` with R
// replicas, routed by `flags` (the clone shares rep's staged couplings and schedule and has
// result buffers of its own, so rep's records are untouched).
int tune_time(pim_instance* rep, int R, int sweeps, int flags, int force_nt, cudaStream_t st,
              double* ms) {
  pim_instance tmp = *rep;
  tmp.d_res = nullptr;
  tmp.R = tmp.R_cap = 0;
  tmp.has_results = false;
  tmp.res_bytes = 0;
  tmp.h_res = nullptr;
  tmp.h_res_dev = nullptr;
  tmp.h_res_cap = 0;
  tmp.h_res_valid = false;
  tmp.done.reset();
  tmp.timer.reset();
  tmp.ticket = 0;
  pim_instance* pt = &tmp;
  t_force_nt = force_nt;
  t_model_routes = true;
  int rc = anneal_impl(&pt, 1, &R, 0, sweeps, 0, nullptr, nullptr, nullptr, flags, st);
  t_force_nt = 0;
  t_model_routes = false;
  if (rc == PIM_OK) rc = sync_instance(pt);
  if (rc == PIM_OK) {
    float k = 0.0f;
    const cudaError_t e = cudaEventElapsedTime(&k, tmp.timer->start, tmp.timer->stop);
    if (e != cudaSuccess) rc = cuda_fail(e, "tuning timer");
    *ms = k;
  }
  free_results(pt);
  return rc;
}

// A candidate's time per sweep is the slope between a short and a longer run (each the
// faster of two, so first-launch costs such as loading the kernel's code drop out), which
// also removes the per-launch prologue and epilogue from the comparison.
constexpr int kTuneShort = 8, kTuneLong = 40;

int tune_slope(pim_instance* rep, int R, int flags, int force_nt, cudaStream_t st, double* us) {
  const int steps = rep->sched->steps;
  const int s_long = std::min(kTuneLong, steps), s_short = std::min(kTuneShort, s_long / 2);
  double best[2] = {1e30, 1e30};
  const int sweeps[2] = {s_short, s_long};
  for (int pass = 0; pass < 2; ++pass)
    for (int v = 0; v < 2; ++v) {
      if (v == 0 && s_short < 1) continue;
      double ms = 0.0;
      const int rc = tune_time(rep, R, sweeps[v], flags, force_nt, st, &ms);
      if (rc != PIM_OK) return rc;
      best[v] = std::min(best[v], ms);
    }
  *us = s_short >= 1 && s_long > s_short ? 1000.0 * (best[1] - best[0]) / (s_long - s_short)
                                         : 1000.0 * best[1] / s_long;
  if (!(*us > 0.0)) *us = 1000.0 * best[1] / s_long;
  return PIM_OK;
}

// Measures every shape class of the batch that the cache does not hold yet (see the tuning
// cache above): fused and mid-N unit times for integer n <= 256, mid-N unit and large-N
// instance sweeps (both tile widths) for integer n <= 1024, large-N sweeps above.
int tune_batch(pim_instance* const* insts, int count, const int* replicas, cudaStream_t st) {
  const int sms = device_sms();
  for (int k = 0; k < count; ++k) {
    pim_instance* p = insts[k];
    if (p->sched->steps < 2) continue;
    double us = 0.0;
    int rc = PIM_OK;
    const bool mid_ok = !p->real && p->npad <= sweep_mid_max_npad();
    if (!p->real && p->n <= kMaxNTensor && p->sched->imax <= kMaxImaxTensor) {
      const std::string key = tune_key("fused", p->npad, p->diag ? 1 : 0);
      if (!tune_known(key)) {  // one full wave: two CTAs per SM, one unit each
        if ((rc = tune_slope(p, 2 * sms * 128, 0, 0, st, &us)) != PIM_OK) return rc;
        tune_store(key, us);
      }
    }
    if (mid_ok) {
      const std::string key = tune_key("mid", p->npad, mid_path(p));
      if (!tune_known(key)) {  // one unit per SM
        if ((rc = tune_slope(p, sms * 128, PIM_PATH_MID, 0, st, &us)) != PIM_OK) return rc;
        tune_store(key, us);
      }
    }
    if (p->n > kMaxNTensor) {
      const int tiles = (replicas[k] + 127) / 128;
      const int base = p->real ? kBigBf16 : kBigFp8;
      const std::pair<int, int> cands[3] = {{64, base}, {128, base}, {64, kBigFp4}};
      for (const auto& cand : cands) {
        const int nt = cand.first, op = cand.second;
        if (p->npad % nt || (op == kBigFp4 && !p->d_img4)) continue;
        const std::string key = tune_key("big", op, p->npad, tiles, nt);
        if (tune_known(key)) continue;
        BigPlan plan;
        t_force_nt = nt;
        t_force_op = op;
        const int prc = plan_big(p->n, p->npad, replicas[k], p->real, p->d_img4 != nullptr,
                                 p->sched->stride_words, &plan);
        if (prc == PIM_OK)  // else this variant cannot be co-resident
          rc = tune_slope(p, replicas[k], PIM_PATH_BIG, nt, st, &us);
        t_force_nt = 0;
        t_force_op = -1;
        if (prc != PIM_OK) continue;
        if (rc != PIM_OK) return rc;
        tune_store(key, us);
      }
    }
  }
  return PIM_OK;
}

}  // namespace

PIM_API int pim_autotune(int mode) {
  if (mode != 0 && mode != 1) return fail(PIM_ERR_INVALID, "pim_autotune: mode must be 0 or 1");
  g_tune_mode = mode;
  return PIM_OK;
}

PIM_API int pim_tune_report(char* out, size_t cap, size_t* needed) {
  std::string text;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    for (const auto& kv : g_tune) {
      char line[256];
      std::snprintf(line, sizeof line, "%s %.4g\n", kv.first.c_str(), kv.second);
      text += line;
    }
  }
  if (needed) *needed = text.size() + 1;
  if (out && cap > 0) {
    const size_t n = std::min(cap - 1, text.size());
    std::memcpy(out, text.data(), n);
    out[n] = '\0';
  }
  return PIM_OK;
}

PIM_API int pim_anneal(pim_instance* inst, int replicas, int t_begin, int sweeps, uint64_t seed,
                       uint32_t instance_id, const int8_t* init_spins, double target_energy,
                       int flags, void* cuda_stream) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_anneal: instance is NULL");
  if (init_spins && !(flags & PIM_CONTINUE)) {
    const size_t tot = static_cast<size_t>(replicas > 0 ? replicas : 0) * inst->n;
    for (size_t k = 0; k < tot; ++k)
      if (init_spins[k] != 1 && init_spins[k] != -1)
        return fail(PIM_ERR_INVALID, "pim_anneal: init_spins must hold -1/+1");
  }
  return anneal_impl(&inst, 1, &replicas, t_begin, sweeps, seed, &instance_id, &target_energy,
                     (flags & PIM_CONTINUE) ? nullptr : init_spins, flags,
                     static_cast<cudaStream_t>(cuda_stream));
}

PIM_API int pim_fields(pim_instance* inst, int replicas, const int8_t* spins, float* fields,
                       int flags, void* cuda_stream) {
  if (!inst || !spins || !fields) return fail(PIM_ERR_INVALID, "pim_fields: NULL argument");
  if (!inst->real)
    return fail(PIM_ERR_UNSUPPORTED, "pim_fields: integer couplings give exact integer fields; "
                                     "the diagnostic serves real couplings");
  if (replicas < 1) return fail(PIM_ERR_INVALID, "pim_fields: replicas = %d < 1", replicas);
  if (flags & ~PIM_PATH_BIG) return fail(PIM_ERR_INVALID, "pim_fields: flags may only hold PIM_PATH_BIG");
  const size_t tot = static_cast<size_t>(replicas) * inst->n;
  for (size_t k = 0; k < tot; ++k)
    if (spins[k] != 1 && spins[k] != -1)
      return fail(PIM_ERR_INVALID, "pim_fields: spins must hold -1/+1");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  float* d_fields = nullptr;
  CK(run_alloc(reinterpret_cast<void**>(&d_fields), tot * sizeof(float), st), "cudaMallocAsync fields");
  const uint32_t id = 0;
  const double no_target = NAN;
  int rc = anneal_impl(&inst, 1, &replicas, 0, 1, 0, &id, &no_target, spins, flags, st, d_fields);
  if (rc == PIM_OK) {
    const cudaError_t e = cudaMemcpyAsync(fields, d_fields, tot * sizeof(float),
                                          cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "fields to host");
  }
  cudaFreeAsync(d_fields, st);
  if (rc != PIM_OK) return rc;
  CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  return sync_instance(inst);
}

PIM_API int pim_anneal_batch(pim_instance* const* insts, int count, const int* replicas,
                             int t_begin, int sweeps, uint64_t seed, const uint32_t* instance_ids,
                             const double* targets, int flags, void* cuda_stream) {
  return anneal_impl(insts, count, replicas, t_begin, sweeps, seed, instance_ids, targets, nullptr,
                     flags, static_cast<cudaStream_t>(cuda_stream));
}

// ----------------------------------------------------------------------------------------
// Batch plans: routing, descriptors and scratch built once; every run replays one CUDA graph
// of the batch's launches (re-captured and updated in place when the run parameters change).
struct pim_batch {
  int device = 0;
  std::vector<pim_instance*> insts;
  std::vector<int> replicas;
  std::vector<uint32_t> ids;
  std::vector<double> targets;
  int flags = 0;
  BatchPlan plan;
  std::vector<std::shared_ptr<Schedule>> scheds;  // schedules the descriptors point into
  std::vector<char*> res;                         // result blocks the descriptors point into
  char* d_buf = nullptr;
  char* d_big = nullptr;
  cudaStream_t cap = nullptr;  // private capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  std::string key;  // run parameters of the instantiated graph
  int launches = 0;
  std::shared_ptr<LaunchTimer> timer;
};

namespace {

void batch_release(pim_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) {
    cudaStreamSynchronize(b->cap);
    cudaStreamDestroy(b->cap);
  }
  // cudaFree waits for the device, so no replay still reads these buffers
  if (b->d_buf) cudaFree(b->d_buf);
  if (b->d_big) cudaFree(b->d_big);
  delete b;
}

}  // namespace

PIM_API int pim_batch_create(pim_batch** out, pim_instance* const* insts, int count,
                             const int* replicas, const uint32_t* instance_ids,
                             const double* targets, int flags) {
  if (!out) return fail(PIM_ERR_INVALID, "pim_batch_create: out is NULL");
  *out = nullptr;
  if (flags & (PIM_CONTINUE | PIM_PATH_FP32REF))
    return fail(PIM_ERR_INVALID, "pim_batch_create: flags take only PIM_PATH_MID / PIM_PATH_BIG");
  int rc = check_batch(insts, count, replicas, 0, 0, targets, flags, false);
  if (rc != PIM_OK) return rc;
  auto* b = new (std::nothrow) pim_batch();
  if (!b) return fail(PIM_ERR_NOMEM, "pim_batch_create: host allocation failed");
  cudaGetDevice(&b->device);
  b->insts.assign(insts, insts + count);
  b->replicas.assign(replicas, replicas + count);
  b->flags = flags;
  for (int k = 0; k < count; ++k) {
    b->ids.push_back(instance_ids ? instance_ids[k] : static_cast<uint32_t>(k));
    b->targets.push_back(targets ? targets[k] : NAN);
  }
  auto bail = [&](int code) {
    batch_release(b);
    return code;
  };
  auto bail_cuda = [&](cudaError_t e, const char* what) {
    const int code = cuda_fail(e, what);
    batch_release(b);
    return code;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
    return bail_cuda(e, "cudaStreamCreate");
  if ((rc = prepare_instances(b->insts.data(), count, b->replicas.data(), false, b->cap)) != PIM_OK)
    return bail(rc);
  if (g_tune_mode.load() == 1 && !(flags & (PIM_PATH_MID | PIM_PATH_BIG)) &&
      (rc = tune_batch(b->insts.data(), count, b->replicas.data(), b->cap)) != PIM_OK)
    return bail(rc);
  if ((rc = build_plan(b->insts.data(), count, b->replicas.data(), b->ids.data(), b->targets.data(),
                       flags, 0, b->plan)) != PIM_OK)
    return bail(rc);
  for (int k = 0; k < count; ++k) {
    b->scheds.push_back(insts[k]->sched);
    b->res.push_back(insts[k]->d_res);
  }
  if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_buf), b->plan.total)) != cudaSuccess)
    return bail_cuda(e, "allocating batch descriptors");
  if (b->plan.big_scratch &&
      (e = cudaMalloc(reinterpret_cast<void**>(&b->d_big), b->plan.big_scratch)) != cudaSuccess)
    return bail_cuda(e, "allocating large-N scratch");
  std::vector<char> h;
  pack_plan(b->plan, nullptr, h);
  if ((e = cudaMemcpyAsync(b->d_buf, h.data(), b->plan.total, cudaMemcpyHostToDevice, b->cap)) != cudaSuccess ||
      (e = cudaStreamSynchronize(b->cap)) != cudaSuccess)
    return bail_cuda(e, "uploading batch descriptors");
  b->timer = std::make_shared<LaunchTimer>();
  if ((e = cudaEventCreate(&b->timer->start)) != cudaSuccess ||
      (e = cudaEventCreate(&b->timer->stop)) != cudaSuccess)
    return bail_cuda(e, "cudaEventCreate");
  *out = b;
  return PIM_OK;
}

PIM_API int pim_batch_run(pim_batch* b, int t_begin, int sweeps, uint64_t seed, int run_flags,
                          void* cuda_stream) {
  if (!b) return fail(PIM_ERR_INVALID, "pim_batch_run: batch is NULL");
  if (run_flags & ~(PIM_CONTINUE | PIM_RESULTS_TO_HOST))
    return fail(PIM_ERR_INVALID, "pim_batch_run: run flags take only PIM_CONTINUE, PIM_RESULTS_TO_HOST");
  const int count = static_cast<int>(b->insts.size());
  int rc = check_batch(b->insts.data(), count, b->replicas.data(), t_begin, sweeps, b->targets.data(),
                       b->flags | run_flags, true);
  if (rc != PIM_OK) return rc;
  for (int k = 0; k < count; ++k)
    if (b->insts[k]->sched != b->scheds[k] || b->insts[k]->d_res != b->res[k])
      return fail(PIM_ERR_STATE, "pim_batch_run: instance %d changed schedule or result buffers "
                  "since the batch was created", k);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != b->device) return fail(PIM_ERR_INVALID, "pim_batch_run: batch lives on device %d", b->device);
  int* d_err = device_error_word(dev);
  if (!d_err) return fail(PIM_ERR_NOMEM, "anneal: error word allocation failed");
  const bool cont = (run_flags & PIM_CONTINUE) != 0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  CK(wait_staged(b->insts.data(), count, st), "cudaStreamWaitEvent");
  // run parameters that the captured launches bake in
  std::string key;
  const uint64_t wait_ns = g_wait_ns.load();
  const int inject = g_inject.load();
  auto put = [&](const void* v, size_t bytes) { key.append(static_cast<const char*>(v), bytes); };
  put(&t_begin, sizeof t_begin);
  put(&sweeps, sizeof sweeps);
  put(&seed, sizeof seed);
  put(&cont, sizeof cont);
  put(&wait_ns, sizeof wait_ns);
  put(&inject, sizeof inject);
  if (b->use_graph && (key != b->key || !b->exec)) {
    cudaGraph_t g = nullptr;
    int nl = 0;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = enqueue_plan(b->plan, b->d_buf, b->d_big, b->insts.data(), count, t_begin, sweeps, seed,
                        cont, false, b->timer.get(), d_err, &nl, b->cap);
      e = cudaStreamEndCapture(b->cap, &g);
    }
    if (e != cudaSuccess || rc != PIM_OK || !g) {
      // a launch of this batch cannot be captured: run it without a graph from now on
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      b->use_graph = false;
    } else {
      cudaGraphExecUpdateResultInfo info;
      if (!b->exec || cudaGraphExecUpdate(b->exec, g, &info) != cudaSuccess) {
        cudaGetLastError();
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        CK(cudaGraphInstantiate(&b->exec, g, 0), "cudaGraphInstantiate");
      }
      if (b->graph) cudaGraphDestroy(b->graph);
      b->graph = g;
      b->key = key;
      b->launches = nl;
    }
  }
  if (b->use_graph) {
    CK(cudaGraphLaunch(b->exec, st), "cudaGraphLaunch");
  } else {
    rc = enqueue_plan(b->plan, b->d_buf, b->d_big, b->insts.data(), count, t_begin, sweeps, seed, cont,
                      false, b->timer.get(), d_err, &b->launches, st);
    if (rc != PIM_OK) return rc;
  }
  const bool to_host = (run_flags & PIM_RESULTS_TO_HOST) != 0;
  bool copied = false;
  if (to_host &&
      (rc = gather_results(b->insts.data(), count, st, &copied)) != PIM_OK)
    return rc;
  return finish_run(b->insts.data(), count, b->replicas.data(), b->timer, st, to_host, copied);
}

PIM_API int pim_batch_info(const pim_batch* b, int* kernel_launches, int* uses_graph) {
  if (!b) return fail(PIM_ERR_INVALID, "pim_batch_info: batch is NULL");
  if (kernel_launches) *kernel_launches = b->launches + 1;  // + the end-of-run error-word mirror
  if (uses_graph) *uses_graph = b->use_graph && b->exec ? 1 : 0;
  return PIM_OK;
}

PIM_API int pim_batch_route(const pim_batch* b, int index, int* kernel, int* tile_width,
                            int* operand) {
  if (!b) return fail(PIM_ERR_INVALID, "pim_batch_route: batch is NULL");
  if (index < 0 || index >= static_cast<int>(b->insts.size()))
    return fail(PIM_ERR_INVALID, "pim_batch_route: index %d out of range", index);
  const int route = b->plan.route[index];
  int nt = 0, op = -1;
  if (route == kBig) {
    const Problem& P = b->plan.probs[index];
    BigPlan plan;
    const int rc = plan_big(P.n, P.npad, P.R, b->insts[index]->real, P.jimg4 != nullptr,
                            P.stride_words, &plan);
    if (rc != PIM_OK) return rc;
    nt = plan.nt;
    op = plan.op;
  }
  if (kernel) *kernel = route;
  if (tile_width) *tile_width = nt;
  if (operand) *operand = op;
  return PIM_OK;
}

PIM_API void pim_batch_destroy(pim_batch* b) {
  if (!b) return;
  for (pim_instance* p : b->insts)
    if (p && p->done) cudaEventSynchronize(p->done->ev);
  batch_release(b);
}

PIM_API int pim_anneal_sequential(pim_instance* inst, int replicas, int t_begin, int sweeps,
                                  uint64_t seed, uint32_t instance_id, const int8_t* init_spins,
                                  double target_energy, int flags, void* cuda_stream) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_anneal_sequential: instance is NULL");
  if (flags & ~(PIM_CONTINUE | PIM_RESULTS_TO_HOST))
    return fail(PIM_ERR_INVALID, "pim_anneal_sequential: flags take only PIM_CONTINUE, PIM_RESULTS_TO_HOST");
  if (inst->real)
    return fail(PIM_ERR_UNSUPPORTED, "pim_anneal_sequential: integer couplings only");
  // (the plain-path flag only skips the fused kernel's field-range check)
  int rc = check_batch(&inst, 1, &replicas, t_begin, sweeps, &target_energy,
                       flags | PIM_PATH_FP32REF, true);
  if (rc != PIM_OK) return rc;
  const bool cont = (flags & PIM_CONTINUE) != 0;
  if (cont && init_spins) return fail(PIM_ERR_INVALID, "pim_anneal_sequential: CONTINUE takes no spins");
  int smem_max = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (sequential_smem_bytes(inst->n) > smem_max)
    return fail(PIM_ERR_UNSUPPORTED, "pim_anneal_sequential: n = %d too large", inst->n);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if ((rc = prepare_instances(&inst, 1, &replicas, false, st)) != PIM_OK) return rc;
  BatchPlan B;
  const uint32_t id = instance_id;
  const size_t init_bytes = init_spins ? static_cast<size_t>(replicas) * inst->n : 0;
  if ((rc = build_plan(&inst, 1, &replicas, &id, &target_energy, PIM_PATH_FP32REF, init_bytes, B)) != PIM_OK)
    return rc;
  char* d_buf = nullptr;
  CK(run_alloc(reinterpret_cast<void**>(&d_buf), B.total, st), "cudaMallocAsync launch buffer");
  std::vector<char> h_buf;
  pack_plan(B, init_spins, h_buf);
  CK(upload_async(d_buf, h_buf.data(), B.total, st), "upload launch buffer");
  if (!cont) {
    const int8_t* d_init = init_bytes ? reinterpret_cast<const int8_t*>(d_buf + B.init_off) : nullptr;
    CK(launch_init_bits(reinterpret_cast<const Problem*>(d_buf), 1, replicas, inst->words, d_init,
                        static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), st),
       "init kernel");
  }
  auto timer = std::make_shared<LaunchTimer>();
  CK(cudaEventCreate(&timer->start), "cudaEventCreate");
  CK(cudaEventCreate(&timer->stop), "cudaEventCreate");
  SeqLaunch L{};
  L.P = B.probs[0];
  L.t_begin = t_begin;
  L.sweeps = sweeps;
  L.cont = cont ? 1 : 0;
  philox_round_keys(seed, L.round_keys);
  CK(cudaEventRecord(timer->start, st), "cudaEventRecord");
  CK(launch_sequential(L, st), "sequential kernel");
  CK(cudaEventRecord(timer->stop, st), "cudaEventRecord");
  CK(cudaFreeAsync(d_buf, st), "cudaFreeAsync launch buffer");
  return finish_run(&inst, 1, &replicas, timer, st, (flags & PIM_RESULTS_TO_HOST) != 0);
}

PIM_API int pim_sync(pim_instance* inst) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_sync: instance is NULL");
  return sync_instance(inst);
}

PIM_API int pim_replicas(const pim_instance* inst) { return inst ? inst->R : 0; }

PIM_API int pim_set_fault_injection(int mode, uint64_t wait_limit_ns) {
  if (mode < 0 || mode > 1) return fail(PIM_ERR_INVALID, "pim_set_fault_injection: mode %d", mode);
  g_inject.store(mode);
  g_wait_ns.store(wait_limit_ns);
  return PIM_OK;
}

PIM_API int pim_kernel_ms(pim_instance* inst, float* ms) {
  if (!inst || !ms) return fail(PIM_ERR_INVALID, "pim_kernel_ms: NULL argument");
  if (!inst->timer) return fail(PIM_ERR_STATE, "pim_kernel_ms: no anneal has run");
  CK(cudaEventSynchronize(inst->timer->stop), "cudaEventSynchronize");
  CK(cudaEventElapsedTime(ms, inst->timer->start, inst->timer->stop), "cudaEventElapsedTime");
  return PIM_OK;
}

PIM_API int pim_energies(pim_instance* inst, double* best_E, int32_t* best_t,
                         int32_t* first_hit_t, double* final_E) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_energies: instance is NULL");
  if (!inst->has_results) return fail(PIM_ERR_STATE, "pim_energies: no anneal has run");
  int rc = sync_instance(inst);
  if (rc != PIM_OK) return rc;
  // The four per-replica arrays are contiguous on the device: one copy.
  const size_t R = inst->R, cap = inst->R_cap;
  std::vector<char> hv;
  const char* h = inst->h_res;
  if (!inst->h_res_valid) {
    hv.resize(cap * 24);
    CK(cudaMemcpy(hv.data(), inst->d_res, cap * 24, cudaMemcpyDeviceToHost), "copy energies");
    h = hv.data();
  }
  if (best_E) std::memcpy(best_E, h, R * 8);
  if (final_E) std::memcpy(final_E, h + cap * 8, R * 8);
  if (best_t) std::memcpy(best_t, h + cap * 16, R * 4);
  if (first_hit_t) std::memcpy(first_hit_t, h + cap * 20, R * 4);
  return PIM_OK;
}

namespace {
int copy_state(pim_instance* inst, const uint32_t* d_bits, int8_t* out) {
  if (!out) return fail(PIM_ERR_INVALID, "state copy: out is NULL");
  if (!inst->has_results) return fail(PIM_ERR_STATE, "state copy: no anneal has run");
  int rc = sync_instance(inst);
  if (rc != PIM_OK) return rc;
  std::vector<uint32_t> bv;
  const uint32_t* bits = nullptr;
  if (inst->h_res_valid) {
    bits = reinterpret_cast<const uint32_t*>(inst->h_res + (reinterpret_cast<const char*>(d_bits) - inst->d_res));
  } else {
    bv.resize(static_cast<size_t>(inst->R) * inst->words);
    CK(cudaMemcpy(bv.data(), d_bits, bv.size() * 4, cudaMemcpyDeviceToHost), "copy state bits");
    bits = bv.data();
  }
  // Byte -> eight int8 spins (+1 where the bit is set, -1 elsewhere), 8 spins per lookup.
  static const std::vector<uint64_t> expand = [] {
    std::vector<uint64_t> tab(256);
    for (int b = 0; b < 256; ++b) {
      uint64_t v = 0;
      for (int k = 0; k < 8; ++k) v |= static_cast<uint64_t>(((b >> k) & 1) ? 0x01 : 0xFF) << (8 * k);
      tab[b] = v;
    }
    return tab;
  }();
  const int n = inst->n, full = n / 8;
  for (int r = 0; r < inst->R; ++r) {
    const uint8_t* src = reinterpret_cast<const uint8_t*>(&bits[static_cast<size_t>(r) * inst->words]);
    int8_t* dst = out + static_cast<size_t>(r) * n;
    for (int b = 0; b < full; ++b) std::memcpy(dst + 8 * b, &expand[src[b]], 8);
    for (int i = 8 * full; i < n; ++i) dst[i] = ((src[i >> 3] >> (i & 7)) & 1) ? 1 : -1;
  }
  return PIM_OK;
}
}  // namespace

PIM_API int pim_results_dev(pim_instance* inst, double* best_E, int32_t* best_t,
                            int32_t* first_hit_t, double* final_E, uint32_t* best_bits,
                            uint32_t* final_bits, void* cuda_stream) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_results_dev: instance is NULL");
  if (!inst->has_results) return fail(PIM_ERR_STATE, "pim_results_dev: no anneal has run");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (inst->done) CK(cudaStreamWaitEvent(st, inst->done->ev, 0), "cudaStreamWaitEvent");
  const size_t R = inst->R, bits = R * inst->words * sizeof(uint32_t);
  auto d2d = [&](void* dst, const void* src, size_t bytes) {
    return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
  };
  CK(d2d(best_E, inst->d_bestE, R * 8), "copy best energies");
  CK(d2d(final_E, inst->d_finalE, R * 8), "copy final energies");
  CK(d2d(best_t, inst->d_bestT, R * 4), "copy best steps");
  CK(d2d(first_hit_t, inst->d_first, R * 4), "copy first hits");
  CK(d2d(best_bits, inst->d_best_bits, bits), "copy best states");
  CK(d2d(final_bits, inst->d_cur_bits, bits), "copy final states");
  return PIM_OK;
}

PIM_API int pim_state_words(const pim_instance* inst) { return inst ? inst->words : 0; }

PIM_API int pim_best_state(pim_instance* inst, int8_t* out) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_best_state: instance is NULL");
  return copy_state(inst, inst->d_best_bits, out);
}

PIM_API int pim_final_state(pim_instance* inst, int8_t* out) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_final_state: instance is NULL");
  return copy_state(inst, inst->d_cur_bits, out);
}

namespace {
std::mutex g_ticket_mu;
std::map<uint64_t, pim_instance*> g_tickets;
uint64_t g_next_ticket = 1;
cudaStream_t g_submit_stream = nullptr;
}  // namespace

PIM_API int pim_submit(pim_instance* inst, int replicas, int sweeps, uint64_t seed, uint64_t* ticket) {
  if (!inst || !ticket) return fail(PIM_ERR_INVALID, "pim_submit: NULL argument");
  std::lock_guard<std::mutex> lk(g_ticket_mu);
  if (!g_submit_stream)
    CK(cudaStreamCreateWithFlags(&g_submit_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  const int rc = pim_anneal(inst, replicas, 0, sweeps, seed, 0, nullptr, NAN, 0, g_submit_stream);
  if (rc != PIM_OK) return rc;
  if (inst->ticket) g_tickets.erase(inst->ticket);
  inst->ticket = g_next_ticket++;
  g_tickets[inst->ticket] = inst;
  *ticket = inst->ticket;
  return PIM_OK;
}

PIM_API int pim_poll(uint64_t ticket) {
  pim_instance* inst = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_ticket_mu);
    auto it = g_tickets.find(ticket);
    if (it == g_tickets.end()) return fail(PIM_ERR_INVALID, "pim_poll: unknown ticket %llu",
                                           static_cast<unsigned long long>(ticket));
    inst = it->second;
  }
  const cudaError_t e = inst->done ? cudaEventQuery(inst->done->ev) : cudaSuccess;
  if (e == cudaErrorNotReady) return PIM_PENDING;
  if (e != cudaSuccess) return cuda_fail(e, "pim_poll");
  return check_device_errors(inst->device);
}

PIM_API void pim_destroy(pim_instance* inst) {
  if (!inst) return;
  if (inst->done) cudaEventSynchronize(inst->done->ev);
  {
    std::lock_guard<std::mutex> lk(g_ticket_mu);
    if (inst->ticket) g_tickets.erase(inst->ticket);
  }
  // Blocks go back to the pool on the release stream once the last anneal has finished.
  free_results(inst);
  give_pinned(inst->h_res, inst->h_res_cap);  // its copies ended with the synchronised run
  // after its last run, or (never run) after its own staging on the staging stream
  cudaEvent_t after = inst->done ? inst->done->ev : inst->ready;
  pool_free_after(inst->d_slab, inst->device, after);
  pool_free_after(inst->d_jf, inst->device, after);
  pool_free_after(inst->d_fix, inst->device, after);
  inst->done.reset();
  give_event(inst->device, inst->ready);
  inst->sched.reset();
  delete inst;
}

PIM_API int pim_thresholds(pim_instance* inst, uint32_t* out, size_t cap_words, int* steps,
                           int* imax, int* stride_words) {
  if (!inst) return fail(PIM_ERR_INVALID, "pim_thresholds: instance is NULL");
  if (!inst->sched) return fail(PIM_ERR_STATE, "pim_thresholds: no schedule");
  if (inst->real) return fail(PIM_ERR_STATE, "pim_thresholds: real-valued couplings have no tables");
  const Schedule& s = *inst->sched;
  if (steps) *steps = s.steps;
  if (imax) *imax = s.imax;
  if (stride_words) *stride_words = s.stride_words;
  if (!out) return PIM_OK;
  const size_t need = static_cast<size_t>(s.steps) * s.stride_words;
  if (cap_words < need) return fail(PIM_ERR_INVALID, "pim_thresholds: need %zu words", need);
  CK(cudaMemcpy(out, s.d_thr, need * 4, cudaMemcpyDeviceToHost), "copy thresholds");
  return PIM_OK;
}
