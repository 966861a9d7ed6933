// MIMO-detection serving engine (supplementary "Kernel execution" and "Host-side task
// scheduling" subsections, re-designed for one GPU): requests (H, y) are queued on the
// host; a dispatcher thread admits them while a stream slot is free and their device
// memory fits the budget, formulates each (FP64 DI-MIMO), stages it as a BF16 instance and
// launches every admitted request of the moment as one batch on a free stream, so batches
// admitted while others run overlap on the device (continuous batching).  A completion
// thread waits for each batch, selects every request's minimum-energy replica by its FP64
// energy, reconstructs the symbols and records the request's latency (submit -> result).
// The Ising solving runs in the library's sweep kernels through the public entry points.
#include <cuda_runtime.h>

#include <algorithm>
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
    if (rc != PIM_OK) {
      if (s->keeper) pim_destroy(s->keeper);
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      return rc;
    }
  }
  s->dispatcher = std::thread([s]() { s->run_dispatcher(); });
  s->completer = std::thread([s]() { s->run_completer(); });
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

PIM_API void pim_mimo_server_destroy(pim_mimo_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->dispatcher.joinable()) s->dispatcher.join();
  if (s->completer.joinable()) s->completer.join();
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
