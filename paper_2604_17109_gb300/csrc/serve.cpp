// MIMO-detection serving engine (supplementary "Kernel execution" and "Host-side task
// scheduling" subsections, re-designed for one GPU): requests (H, y) are queued on the
// host; a dispatcher thread admits them while a stream slot is free and their device
// memory fits the budget, formulates each (FP64 DI-MIMO), stages it as a BF16 instance and
// launches every admitted request of the moment as one batch on a free stream, so batches
// admitted while others run overlap on the device (continuous batching).  A completion
// thread waits for each batch, selects every request's minimum-energy replica by its FP64
// energy, reconstructs the symbols and records the request's latency (submit -> result).
// The Ising solving runs in the library's sweep kernels through the public entry points.
//
// Device-queue mode (cfg.device_queue): the dispatcher writes each formulated request into a
// slot of a queue in mapped pinned host memory and publishes it; a persistent serving kernel
// (launch_serve_float) claims requests from a device counter and flags each slot done; the
// completion thread polls the flags.  The kernel ends after idle_s without requests and is
// launched again by whichever thread next finds requests in flight and the kernel ended.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels.h"
#include "mimo.h"
#include "pim.h"

#define PIM_API extern "C" __attribute__((visibility("default")))

using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket = 0;
  uint32_t id = 0;
  std::vector<double> H, y;
  double reg = 0.0;
  Clock::time_point t_submit, t_done;
  pim_instance* inst = nullptr;
  std::vector<double> J, h, xm;
  size_t bytes = 0;
  std::vector<double> x_hat;
  double best_E = NAN;
  int status = PIM_PENDING;
  uint64_t seq = 0;  // device queue: position in the queue (slot seq % nslots)
};

struct Batch {
  std::vector<std::shared_ptr<Request>> reqs;
  cudaEvent_t done = nullptr;
  int slot = -1;
  size_t bytes = 0;
};

int fail_msg(int code, const char* msg) {
  pim::set_last_error(msg);
  return code;
}

// BF16 bits of v rounded to nearest (ties to even) from float64 directly: the float64
// significand is rounded to 8 bits, after which the conversion to float32 is exact.
uint16_t bf16_rne(double v) {
  uint64_t d;
  std::memcpy(&d, &v, sizeof d);
  d += ((1ull << 44) - 1) + ((d >> 45) & 1);
  d &= ~((1ull << 45) - 1);
  double r;
  std::memcpy(&r, &d, sizeof r);
  const float f = static_cast<float>(r);
  uint32_t b;
  std::memcpy(&b, &f, sizeof b);
  return static_cast<uint16_t>(b >> 16);
}

// Layout of one queue slot in the mapped block: descriptor, BF16 coupling image, bias,
// results (best / final energies, best step, first hit, best and final spin bits).
struct SlotLayout {
  size_t desc = 0, img = 0, bias = 0, bestE = 0, finalE = 0, bestT = 0, first = 0, best_bits = 0,
         cur_bits = 0, bytes = 0;
  SlotLayout(int npad, int R, int words) {
    auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    size_t o = up(sizeof(pim::Problem));
    img = o;
    o = up(o + static_cast<size_t>(npad) * npad * 2);
    bias = o;
    o = up(o + static_cast<size_t>(npad) * 4);
    bestE = o;
    o = up(o + static_cast<size_t>(R) * 8);
    finalE = o;
    o = up(o + static_cast<size_t>(R) * 8);
    bestT = o;
    o = up(o + static_cast<size_t>(R) * 4);
    first = o;
    o = up(o + static_cast<size_t>(R) * 4);
    best_bits = o;
    o = up(o + static_cast<size_t>(R) * words * 4);
    cur_bits = o;
    o = up(o + static_cast<size_t>(R) * words * 4);
    bytes = o;
  }
};

}  // namespace

struct pim_mimo_server {
  pim_mimo_server_config cfg{};
  std::vector<float> beta, eta;
  int device = 0, n = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> requests;
  std::deque<Batch> inflight;
  std::vector<cudaStream_t> streams;
  std::vector<bool> busy;
  size_t bytes_inflight = 0, peak_bytes = 0;
  uint64_t next_ticket = 1, completed = 0, batches = 0, batched = 0;
  std::vector<double> latencies_us;
  bool stop = false, dispatcher_done = false;
  int error = PIM_OK;
  pim_instance* keeper = nullptr;  // holds the schedule so the library keeps it cached
  std::thread dispatcher, completer;

  // ---- device-queue mode ----------------------------------------------------------------
  bool dq = false;
  int npad = 0, words = 0, nslots = 0, ctas = 0;
  SlotLayout lay{128, 1, 2};
  char* h_block = nullptr;       // mapped pinned: control words | slots
  char* d_block = nullptr;       // its device address
  unsigned int* h_tail = nullptr;
  unsigned int* h_stop = nullptr;
  unsigned int* h_done = nullptr;
  size_t slots_off = 0;
  unsigned int* d_head = nullptr;  // device memory: claimed requests
  int* d_exit = nullptr;           // device memory: why the kernel ended
  pim::ServeQueue Q{};
  pim::Launch L{};
  pim::Problem proto{};            // descriptor fields shared by every request
  cudaStream_t kstream = nullptr;
  cudaEvent_t kdone = nullptr;
  std::mutex kmu;                  // kernel launches
  bool kernel_launched = false;
  int last_exit = 0;               // 1 idle limit, 2 stopped
  uint64_t published = 0;          // requests written to the queue
  std::vector<std::shared_ptr<Request>> slot_req;  // in-flight request of each slot
  std::atomic<uint64_t> in_flight{0};

  char* slot_host(int k) { return h_block + slots_off + static_cast<size_t>(k) * lay.bytes; }
  char* slot_dev(int k) { return d_block + slots_off + static_cast<size_t>(k) * lay.bytes; }
  int ensure_kernel();  // launches the serving kernel unless it is running
  int setup_device_queue();
  void free_device_queue();
  void run_dq_dispatcher();
  void run_dq_completer();

  // device bytes one request holds while admitted: BF16 J and image, bias, results
  size_t request_bytes() const {
    const size_t npad = n <= 128 ? 128 : (n <= 256 ? 256 : ((n + 127) / 128) * 128);
    const size_t words = ((n + 63) / 64) * 2;
    return 2 * static_cast<size_t>(n) * n + 2 * npad * npad + 4 * n + 4096 +
           static_cast<size_t>(cfg.replicas) * (24 + 8 * words);
  }

  void run_dispatcher();
  void run_completer();
};

void pim_mimo_server::run_dispatcher() {
  cudaSetDevice(device);
  for (;;) {
    Batch b;
    {
      std::unique_lock<std::mutex> lk(mu);
      auto free_slot = [&]() {
        for (size_t k = 0; k < busy.size(); ++k)
          if (!busy[k]) return static_cast<int>(k);
        return -1;
      };
      cv_work.wait(lk, [&]() {
        return stop || (!queue.empty() && free_slot() >= 0 &&
                        bytes_inflight + request_bytes() <= cfg.mem_budget);
      });
      if (stop && queue.empty()) break;
      if (stop) break;
      b.slot = free_slot();
      while (!queue.empty() && static_cast<int>(b.reqs.size()) < cfg.max_batch &&
             bytes_inflight + b.bytes + request_bytes() <= cfg.mem_budget) {
        b.reqs.push_back(queue.front());
        queue.pop_front();
        b.bytes += request_bytes();
      }
      busy[b.slot] = true;
      bytes_inflight += b.bytes;
      peak_bytes = std::max(peak_bytes, bytes_inflight);
    }
    // formulate and stage every admitted request, then one batched anneal on the slot
    std::vector<pim_instance*> insts;
    std::vector<uint32_t> ids;
    int rc = PIM_OK;
    for (auto& r : b.reqs) {
      r->J.assign(static_cast<size_t>(n) * n, 0.0);
      r->h.assign(n, 0.0);
      r->xm.assign(2 * cfg.nt, 0.0);
      rc = pim::mimo_formulate(cfg.nt, cfg.nr, cfg.qam, r->H.data(), r->y.data(), r->reg,
                               r->J.data(), r->h.data(), r->xm.data());
      if (rc == PIM_OK) rc = pim_create(&r->inst, n, PIM_J_FP64, r->J.data(), r->h.data(), cfg.scale_c);
      if (rc == PIM_OK)
        rc = pim_set_schedule(r->inst, cfg.sweeps, beta.data(), eta.data(), cfg.xi,
                              PIM_NOISE_GAUSS, PIM_ACT_TANH, 0);
      if (rc != PIM_OK) break;
      insts.push_back(r->inst);
      ids.push_back(r->id);
    }
    cudaStream_t st = streams[b.slot];
    if (rc == PIM_OK) {
      std::vector<int> reps(insts.size(), cfg.replicas);
      rc = pim_anneal_batch(insts.data(), static_cast<int>(insts.size()), reps.data(), 0,
                            cfg.sweeps, cfg.seed, ids.data(), nullptr, 0, st);
    }
    if (rc == PIM_OK && cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess)
      rc = PIM_ERR_CUDA;
    if (rc == PIM_OK && cudaEventRecord(b.done, st) != cudaSuccess) rc = PIM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(mu);
    if (rc != PIM_OK) {
      error = rc;
      for (auto& r : b.reqs) r->status = rc;
    }
    inflight.push_back(std::move(b));
    ++batches;
    cv_done.notify_all();
  }
  std::lock_guard<std::mutex> lk(mu);
  dispatcher_done = true;
  cv_done.notify_all();
}

void pim_mimo_server::run_completer() {
  cudaSetDevice(device);
  const int R = cfg.replicas;
  std::vector<int8_t> states(static_cast<size_t>(R) * n);
  std::vector<double> Es(R);
  for (;;) {
    Batch b;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_done.wait(lk, [&]() { return !inflight.empty() || (dispatcher_done && inflight.empty()); });
      if (inflight.empty()) break;
      b = inflight.front();
      inflight.pop_front();
    }
    if (b.done) cudaEventSynchronize(b.done);
    std::vector<int> status(b.reqs.size(), PIM_OK);
    for (size_t q = 0; q < b.reqs.size(); ++q) {
      auto& r = b.reqs[q];
      status[q] = r->status;
      if (r->status == PIM_PENDING && r->inst) {
        // the replica of lowest reported energy (device FP32 sums; ties -> lowest index),
        // then its FP64 energy -1/2 s^T J s - h^T s
        int rc = pim_energies(r->inst, Es.data(), nullptr, nullptr, nullptr);
        if (rc == PIM_OK) rc = pim_best_state(r->inst, states.data());
        if (rc == PIM_OK) {
          const int best = static_cast<int>(std::min_element(Es.begin(), Es.end()) - Es.begin());
          const int8_t* s = states.data() + static_cast<size_t>(best) * n;
          double e = 0.0;
          for (int i = 0; i < n; ++i) {
            double f = 0.0;
            const double* Ji = r->J.data() + static_cast<size_t>(i) * n;
            for (int j = 0; j < n; ++j) f += Ji[j] * s[j];
            e -= s[i] * (0.5 * f + r->h[i]);
          }
          r->best_E = e;
          r->x_hat.assign(2 * cfg.nt, 0.0);
          pim::mimo_reconstruct(cfg.nt, cfg.qam, r->xm.data(), s, r->x_hat.data());
        }
        status[q] = rc;
      }
      if (r->inst) pim_destroy(r->inst);
      r->inst = nullptr;
    }
    if (b.done) cudaEventDestroy(b.done);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    for (size_t q = 0; q < b.reqs.size(); ++q) {
      auto& r = b.reqs[q];
      r->status = status[q];
      r->t_done = now;
      latencies_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
      ++completed;
    }
    batched += b.reqs.size();
    if (b.slot >= 0) busy[b.slot] = false;
    bytes_inflight -= b.bytes;
    cv_work.notify_all();
    cv_done.notify_all();
  }
}

int pim_mimo_server::setup_device_queue() {
  if (n > 256 || cfg.replicas > 128)
    return fail_msg(PIM_ERR_UNSUPPORTED, "pim_mimo_server_create: the device queue serves n <= 256 "
                                         "spins and at most 128 replicas");
  if (!(cfg.idle_s > 0.0) || !std::isfinite(cfg.idle_s))
    return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_create: idle_s must be > 0");
  dq = true;
  npad = n <= 128 ? 128 : 256;
  words = ((n + 63) / 64) * 2;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  ctas = std::max(1, std::min(sms, cfg.max_batch * cfg.max_inflight));
  nslots = 2 * ctas;
  lay = SlotLayout(npad, cfg.replicas, words);
  slots_off = 256 + ((static_cast<size_t>(nslots) * 4 + 255) & ~static_cast<size_t>(255));
  const size_t bytes = slots_off + static_cast<size_t>(nslots) * lay.bytes;
  if (cudaHostAlloc(reinterpret_cast<void**>(&h_block), bytes, cudaHostAllocMapped) != cudaSuccess)
    return fail_msg(PIM_ERR_NOMEM, "pim_mimo_server_create: mapped queue allocation failed");
  std::memset(h_block, 0, bytes);
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_block), h_block, 0) != cudaSuccess)
    return fail_msg(PIM_ERR_UNSUPPORTED, "pim_mimo_server_create: mapped memory has no device address");
  h_tail = reinterpret_cast<unsigned int*>(h_block);
  h_stop = h_tail + 1;
  h_done = reinterpret_cast<unsigned int*>(h_block + 256);
  if (cudaMalloc(reinterpret_cast<void**>(&d_head), 256) != cudaSuccess ||
      cudaMemset(d_head, 0, 256) != cudaSuccess)
    return fail_msg(PIM_ERR_NOMEM, "pim_mimo_server_create: device queue counters");
  d_exit = reinterpret_cast<int*>(d_head + 1);
  if (cudaStreamCreateWithFlags(&kstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&kdone, cudaEventDisableTiming) != cudaSuccess)
    return fail_msg(PIM_ERR_CUDA, "pim_mimo_server_create: serving stream");
  const float *bt = nullptr, *eta_d = nullptr, *z = nullptr;
  float xi = 0.0f;
  int act = 0, lut = 0;
  if (pim::schedule_device_arrays(keeper, &bt, &eta_d, &z, &xi, &act, &lut) != PIM_OK)
    return fail_msg(PIM_ERR_STATE, "pim_mimo_server_create: no real-valued schedule");
  proto = pim::Problem{};
  proto.n = n;
  proto.npad = npad;
  proto.words = words;
  proto.R = cfg.replicas;
  proto.sched_b = bt;
  proto.sched_eta = eta_d;
  proto.zlev = z;
  proto.xi = xi;
  proto.act = act;
  proto.lut_levels = lut;
  Q.tail = reinterpret_cast<const unsigned int*>(d_block);
  Q.stop = reinterpret_cast<const unsigned int*>(d_block) + 1;
  Q.done = reinterpret_cast<unsigned int*>(d_block + 256);
  Q.slots = d_block + slots_off;
  Q.slot_bytes = lay.bytes;
  Q.head = d_head;
  Q.exit_status = d_exit;
  Q.zlev = z;
  Q.nslots = nslots;
  Q.idle_ns = static_cast<uint64_t>(cfg.idle_s * 1e9);
  L = pim::Launch{};
  L.t_begin = 0;
  L.sweeps = cfg.sweeps;
  L.key_lo = static_cast<uint32_t>(cfg.seed);
  L.key_hi = static_cast<uint32_t>(cfg.seed >> 32);
  pim::philox_round_keys(cfg.seed, L.round_keys);
  L.err = d_exit + 1;
  slot_req.assign(nslots, nullptr);
  return PIM_OK;
}

void pim_mimo_server::free_device_queue() {
  if (kstream) cudaStreamSynchronize(kstream);
  if (kdone) cudaEventDestroy(kdone);
  if (kstream) cudaStreamDestroy(kstream);
  if (d_head) cudaFree(d_head);
  if (h_block) cudaFreeHost(h_block);
  kdone = nullptr;
  kstream = nullptr;
  d_head = nullptr;
  h_block = nullptr;
}

int pim_mimo_server::ensure_kernel() {
  std::lock_guard<std::mutex> lk(kmu);
  if (kernel_launched) {
    const cudaError_t q = cudaEventQuery(kdone);
    if (q == cudaErrorNotReady) return PIM_OK;  // still serving
    if (q != cudaSuccess) return PIM_ERR_CUDA;
    int why[2] = {0, 0};  // exit reason, device error bits
    if (cudaMemcpy(why, d_exit, sizeof why, cudaMemcpyDeviceToHost) != cudaSuccess) return PIM_ERR_CUDA;
    last_exit = why[0];
    kernel_launched = false;
    if (why[1] & pim::kDevErrTimeout) {
      pim::set_last_error("serving kernel: a device-side bounded wait gave up");
      return PIM_ERR_TIMEOUT;
    }
  }
  if (cudaMemsetAsync(d_exit, 0, 2 * sizeof(int), kstream) != cudaSuccess) return PIM_ERR_CUDA;
  if (pim::launch_serve_float(L, Q, npad, ctas, kstream) != cudaSuccess) return PIM_ERR_CUDA;
  if (cudaEventRecord(kdone, kstream) != cudaSuccess) return PIM_ERR_CUDA;
  kernel_launched = true;
  return PIM_OK;
}

void pim_mimo_server::run_dq_dispatcher() {
  cudaSetDevice(device);
  const size_t nn = static_cast<size_t>(n) * n;
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&]() { return stop || !queue.empty(); });
      if (stop) break;
      r = queue.front();
      queue.pop_front();
    }
    r->J.assign(nn, 0.0);
    r->h.assign(n, 0.0);
    r->xm.assign(2 * cfg.nt, 0.0);
    int rc = pim::mimo_formulate(cfg.nt, cfg.nr, cfg.qam, r->H.data(), r->y.data(), r->reg,
                                 r->J.data(), r->h.data(), r->xm.data());
    std::unique_lock<std::mutex> lk(mu);
    if (rc != PIM_OK) {
      r->status = rc;
      r->t_done = Clock::now();
      latencies_us.push_back(std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
      ++completed;
      cv_done.notify_all();
      continue;
    }
    const int slot = static_cast<int>(published % nslots);
    cv_work.wait(lk, [&]() { return stop || !slot_req[slot]; });  // the slot's last request is read
    if (stop) break;
    // the position first: the completion thread matches the slot's done flag against it as
    // soon as the request is in the slot table (the flag still holds the slot's previous
    // request's position + 1 until this one is done)
    r->seq = published;
    slot_req[slot] = r;
    lk.unlock();
    // the request into its slot: BF16 coupling image (K-major, 128-byte swizzle), bias and
    // descriptor, then the release store that publishes it
    char* base = slot_host(slot);
    uint16_t* img = reinterpret_cast<uint16_t*>(base + lay.img);
    std::memset(img, 0, static_cast<size_t>(npad) * npad * 2);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        img[pim::sw128_offset(i, 2 * j, npad) / 2] = bf16_rne(r->J[static_cast<size_t>(i) * n + j]);
    float* bias = reinterpret_cast<float*>(base + lay.bias);
    for (int i = 0; i < npad; ++i) bias[i] = i < n ? static_cast<float>(r->h[i]) : 0.0f;
    pim::Problem P = proto;
    char* dev = slot_dev(slot);
    P.jimg = reinterpret_cast<const uint8_t*>(dev + lay.img);
    P.hf = reinterpret_cast<const float*>(dev + lay.bias);
    P.best_E = reinterpret_cast<double*>(dev + lay.bestE);
    P.final_E = reinterpret_cast<double*>(dev + lay.finalE);
    P.best_t = reinterpret_cast<int32_t*>(dev + lay.bestT);
    P.first_hit = reinterpret_cast<int32_t*>(dev + lay.first);
    P.best_bits = reinterpret_cast<uint32_t*>(dev + lay.best_bits);
    P.cur_bits = reinterpret_cast<uint32_t*>(dev + lay.cur_bits);
    P.q = r->id;
    std::memcpy(base + lay.desc, &P, sizeof P);
    std::atomic_thread_fence(std::memory_order_release);
    lk.lock();
    ++published;
    __atomic_store_n(h_tail, static_cast<unsigned int>(published), __ATOMIC_RELEASE);
    ++in_flight;
    peak_bytes = std::max(peak_bytes, static_cast<size_t>(in_flight.load()) * lay.bytes);
    ++batches;
    lk.unlock();
    rc = ensure_kernel();
    if (rc != PIM_OK) {
      std::lock_guard<std::mutex> g(mu);
      error = rc;
    }
    cv_done.notify_all();
  }
  std::lock_guard<std::mutex> lk(mu);
  dispatcher_done = true;
  cv_done.notify_all();
}

void pim_mimo_server::run_dq_completer() {
  cudaSetDevice(device);
  const int R = cfg.replicas;
  std::vector<int8_t> s(n);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_done.wait(lk, [&]() { return in_flight.load() > 0 || dispatcher_done; });
      if (in_flight.load() == 0 && dispatcher_done) break;
    }
    bool progress = false;
    for (int slot = 0; slot < nslots; ++slot) {
      std::shared_ptr<Request> r;
      {
        std::lock_guard<std::mutex> lk(mu);
        r = slot_req[slot];
      }
      if (!r || __atomic_load_n(h_done + slot, __ATOMIC_ACQUIRE) != static_cast<unsigned int>(r->seq + 1))
        continue;
      const char* base = slot_host(slot);
      const double* bestE = reinterpret_cast<const double*>(base + lay.bestE);
      const uint32_t* bits = reinterpret_cast<const uint32_t*>(base + lay.best_bits);
      // the replica of lowest reported energy (ties -> lowest index), then its FP64 energy
      int best = 0;
      for (int q = 1; q < R; ++q)
        if (bestE[q] < bestE[best]) best = q;
      for (int i = 0; i < n; ++i)
        s[i] = ((bits[static_cast<size_t>(best) * words + (i >> 5)] >> (i & 31)) & 1u) ? 1 : -1;
      double e = 0.0;
      for (int i = 0; i < n; ++i) {
        double f = 0.0;
        const double* Ji = r->J.data() + static_cast<size_t>(i) * n;
        for (int j = 0; j < n; ++j) f += Ji[j] * s[j];
        e -= s[i] * (0.5 * f + r->h[i]);
      }
      r->best_E = e;
      r->x_hat.assign(2 * cfg.nt, 0.0);
      pim::mimo_reconstruct(cfg.nt, cfg.qam, r->xm.data(), s.data(), r->x_hat.data());
      const auto now = Clock::now();
      std::lock_guard<std::mutex> lk(mu);
      r->status = PIM_OK;
      r->t_done = now;
      latencies_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
      ++completed;
      ++batched;
      slot_req[slot].reset();
      --in_flight;
      progress = true;
      cv_work.notify_all();
      cv_done.notify_all();
    }
    if (!progress) {
      // requests in flight but the kernel ended (its wait for requests ran out just before
      // they were published): launch it again
      if (in_flight.load() > 0) {
        const int rc = ensure_kernel();
        if (rc != PIM_OK) {
          std::lock_guard<std::mutex> lk(mu);
          error = rc;
        }
      }
      std::this_thread::yield();
    }
  }
}

PIM_API int pim_mimo_server_create(pim_mimo_server** out, const pim_mimo_server_config* cfg) {
  if (!out || !cfg) return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_create: NULL argument");
  *out = nullptr;
  const int ncopy = pim::mimo_spins_per_component(cfg->qam);
  if (ncopy == 0 || cfg->nt < 1 || cfg->nr < cfg->nt || cfg->replicas < 1 || cfg->sweeps < 1 ||
      !cfg->beta || !cfg->eta || cfg->max_batch < 1 || cfg->max_inflight < 1 ||
      !(cfg->scale_c > 0.0))
    return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_create: bad configuration");
  const int n = ncopy * 2 * cfg->nt;
  if (n > 8192) return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_create: system too large");
  auto* s = new (std::nothrow) pim_mimo_server();
  if (!s) return fail_msg(PIM_ERR_NOMEM, "pim_mimo_server_create: host allocation failed");
  s->cfg = *cfg;
  s->n = n;
  s->beta.assign(cfg->beta, cfg->beta + cfg->sweeps);
  s->eta.assign(cfg->eta, cfg->eta + cfg->sweeps);
  if (s->cfg.mem_budget < s->request_bytes()) s->cfg.mem_budget = s->request_bytes();
  cudaGetDevice(&s->device);
  for (int k = 0; k < cfg->max_inflight; ++k) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      return fail_msg(PIM_ERR_CUDA, "pim_mimo_server_create: cudaStreamCreate failed");
    }
    s->streams.push_back(st);
  }
  s->busy.assign(cfg->max_inflight, false);
  {
    std::vector<double> J0(static_cast<size_t>(n) * n, 0.0);
    int rc = pim_create(&s->keeper, n, PIM_J_FP64, J0.data(), nullptr, cfg->scale_c);
    if (rc == PIM_OK)
      rc = pim_set_schedule(s->keeper, cfg->sweeps, cfg->beta, cfg->eta, cfg->xi, PIM_NOISE_GAUSS,
                            PIM_ACT_TANH, 0);
    if (rc == PIM_OK && cfg->device_queue) rc = s->setup_device_queue();
    if (rc != PIM_OK) {
      s->free_device_queue();
      if (s->keeper) pim_destroy(s->keeper);
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      return rc;
    }
  }
  if (s->dq) {
    s->dispatcher = std::thread([s]() { s->run_dq_dispatcher(); });
    s->completer = std::thread([s]() { s->run_dq_completer(); });
  } else {
    s->dispatcher = std::thread([s]() { s->run_dispatcher(); });
    s->completer = std::thread([s]() { s->run_completer(); });
  }
  *out = s;
  return PIM_OK;
}

PIM_API int pim_mimo_server_submit(pim_mimo_server* s, const double* H, const double* y,
                                   double mmse_reg, uint32_t request_id, uint64_t* ticket) {
  if (!s || !H || !y || !ticket || !(mmse_reg > 0.0))
    return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_submit: bad arguments");
  auto r = std::make_shared<Request>();
  r->H.assign(H, H + 2 * static_cast<size_t>(s->cfg.nr) * s->cfg.nt);
  r->y.assign(y, y + 2 * static_cast<size_t>(s->cfg.nr));
  r->reg = mmse_reg;
  r->id = request_id;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return fail_msg(PIM_ERR_STATE, "pim_mimo_server_submit: server stopping");
  r->ticket = s->next_ticket++;
  s->requests[r->ticket] = r;
  s->queue.push_back(r);
  *ticket = r->ticket;
  s->cv_work.notify_all();
  return PIM_OK;
}

PIM_API int pim_mimo_server_poll(pim_mimo_server* s, uint64_t ticket) {
  if (!s) return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_poll: server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_poll: unknown ticket");
  const auto& r = it->second;
  if (r->status == PIM_PENDING || r->t_done == Clock::time_point()) return PIM_PENDING;
  return r->status;
}

PIM_API int pim_mimo_server_result(pim_mimo_server* s, uint64_t ticket, double timeout_s,
                                   double* x_hat, double* best_energy, double* latency_us) {
  if (!s) return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_result: server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_result: unknown ticket");
  auto r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  if (!s->cv_done.wait_until(lk, deadline, [&]() { return r->t_done != Clock::time_point(); }))
    return PIM_PENDING;
  if (r->status != PIM_OK) return fail_msg(r->status, "pim_mimo_server_result: request failed");
  if (x_hat) std::memcpy(x_hat, r->x_hat.data(), r->x_hat.size() * sizeof(double));
  if (best_energy) *best_energy = r->best_E;
  if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
  s->requests.erase(it);
  return PIM_OK;
}

PIM_API int pim_mimo_server_stats(pim_mimo_server* s, uint64_t* completed, double* p50_us,
                                  double* p99_us, double* mean_batch, size_t* peak_bytes) {
  if (!s) return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_stats: server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> l = s->latencies_us;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    const size_t k = std::min(l.size() - 1, static_cast<size_t>(std::ceil(q * l.size())) - (q > 0 ? 1 : 0));
    return l[k];
  };
  if (completed) *completed = s->completed;
  if (p50_us) *p50_us = pct(0.50);
  if (p99_us) *p99_us = pct(0.99);
  if (mean_batch) *mean_batch = s->batches ? static_cast<double>(s->batched) / s->batches : 0.0;
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  return s->error;
}

PIM_API int pim_mimo_server_replay(pim_mimo_server* s, int count, const double* H_all,
                                   const double* y_all, const double* reg_all,
                                   const double* arrival_us, double* x_hat_all,
                                   double* best_energy_all, double* latency_us_all) {
  if (!s || count < 0 || (count && (!H_all || !y_all || !reg_all || !arrival_us)))
    return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_replay: bad arguments");
  const size_t hs = 2 * static_cast<size_t>(s->cfg.nr) * s->cfg.nt, ys = 2 * static_cast<size_t>(s->cfg.nr);
  std::vector<uint64_t> tickets(count);
  const auto t0 = Clock::now();
  for (int k = 0; k < count; ++k) {
    std::this_thread::sleep_until(t0 + std::chrono::duration<double, std::micro>(arrival_us[k]));
    const int rc = pim_mimo_server_submit(s, H_all + k * hs, y_all + k * ys, reg_all[k],
                                          static_cast<uint32_t>(k), &tickets[k]);
    if (rc != PIM_OK) return rc;
  }
  int status = PIM_OK;
  for (int k = 0; k < count; ++k) {
    double lat = 0.0, e = 0.0;
    const int rc = pim_mimo_server_result(s, tickets[k], 600.0,
                                          x_hat_all ? x_hat_all + k * 2 * static_cast<size_t>(s->cfg.nt) : nullptr,
                                          &e, &lat);
    if (rc != PIM_OK) status = rc;
    if (best_energy_all) best_energy_all[k] = e;
    if (latency_us_all) latency_us_all[k] = lat;
  }
  return status;
}

PIM_API int pim_mimo_server_idle_wait(pim_mimo_server* s, double timeout_s) {
  if (!s) return fail_msg(PIM_ERR_INVALID, "pim_mimo_server_idle_wait: server is NULL");
  if (!s->dq) return fail_msg(PIM_ERR_UNSUPPORTED, "pim_mimo_server_idle_wait: no device queue");
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    if (s->in_flight.load() == 0) {
      std::lock_guard<std::mutex> lk(s->kmu);
      if (!s->kernel_launched) break;
      const cudaError_t q = cudaEventQuery(s->kdone);
      if (q == cudaSuccess) {
        int why = 0;
        if (cudaMemcpy(&why, s->d_exit, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
          return fail_msg(PIM_ERR_CUDA, "pim_mimo_server_idle_wait: reading the exit status");
        s->last_exit = why;
        s->kernel_launched = false;
        break;
      }
      if (q != cudaErrorNotReady) return fail_msg(PIM_ERR_CUDA, "pim_mimo_server_idle_wait: cudaEventQuery");
    }
    if (Clock::now() > deadline) return PIM_PENDING;
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  if (s->last_exit == 1)
    return fail_msg(PIM_ERR_TIMEOUT, "pim_mimo_server_idle_wait: the serving kernel's wait for "
                                     "requests ran out (idle limit)");
  return PIM_OK;
}

PIM_API void pim_mimo_server_destroy(pim_mimo_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->dispatcher.joinable()) s->dispatcher.join();
  if (s->dq) {
    // no new requests: the kernel finishes what it claimed and ends once the queue is empty
    __atomic_store_n(s->h_stop, 1u, __ATOMIC_RELEASE);
  }
  if (s->completer.joinable()) s->completer.join();
  s->free_device_queue();
  for (auto& q : s->queue)
    if (q->inst) pim_destroy(q->inst);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  if (s->keeper) pim_destroy(s->keeper);
  delete s;
}

PIM_API int pim_mimo_formulate(int nt, int nr, int qam, const double* H, const double* y,
                               double mmse_reg, double* J, double* h, double* x_mmse) {
  if (nt < 1 || nr < nt || !H || !y || !J || !h || !x_mmse || !(mmse_reg > 0.0) ||
      pim::mimo_spins_per_component(qam) == 0)
    return fail_msg(PIM_ERR_INVALID, "pim_mimo_formulate: bad arguments");
  const int rc = pim::mimo_formulate(nt, nr, qam, H, y, mmse_reg, J, h, x_mmse);
  if (rc != PIM_OK) return fail_msg(rc, "pim_mimo_formulate: MMSE system not positive definite");
  return PIM_OK;
}

PIM_API int pim_mimo_reconstruct(int nt, int qam, const double* x_mmse, const int8_t* spins,
                                 double* x_hat) {
  if (nt < 1 || !x_mmse || !spins || !x_hat || pim::mimo_spins_per_component(qam) == 0)
    return fail_msg(PIM_ERR_INVALID, "pim_mimo_reconstruct: bad arguments");
  pim::mimo_reconstruct(nt, qam, x_mmse, spins, x_hat);
  return PIM_OK;
}

PIM_API int pim_mimo_formulate_depth(int nt, int nr, int qam, int depth, const double* H,
                                     const double* y, double mmse_reg, double* J, double* h,
                                     double* x_mmse) {
  if (nt < 1 || nr < nt || !H || !y || !J || !h || !x_mmse || !(mmse_reg > 0.0) ||
      pim::mimo_depth(qam, depth) == 0)
    return fail_msg(PIM_ERR_INVALID, "pim_mimo_formulate_depth: bad arguments");
  const int rc = pim::mimo_formulate(nt, nr, qam, H, y, mmse_reg, J, h, x_mmse, depth);
  if (rc != PIM_OK)
    return fail_msg(rc, "pim_mimo_formulate_depth: MMSE system not positive definite");
  return PIM_OK;
}

PIM_API int pim_mimo_reconstruct_depth(int nt, int qam, int depth, const double* x_mmse,
                                       const int8_t* spins, double* x_hat) {
  if (nt < 1 || !x_mmse || !spins || !x_hat || pim::mimo_depth(qam, depth) == 0)
    return fail_msg(PIM_ERR_INVALID, "pim_mimo_reconstruct_depth: bad arguments");
  pim::mimo_reconstruct(nt, qam, x_mmse, spins, x_hat, depth);
  return PIM_OK;
}
