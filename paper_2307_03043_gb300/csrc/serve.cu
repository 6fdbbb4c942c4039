// serve.cu -- ch_serve_*: a request loop for Chamfer estimates over resident
// point sets (host C++; the device work is ch_estimate on per-slot streams).
//
//  * Sets are registered once, prepared eagerly (bounding box, |x|^2, finite
//    check; with ch_serve_index also the l2 embedding under the index's hash
//    parameters) and never written again, so every slot may read them at once.
//  * Each request's device footprint is the exact workspace ch_estimate needs
//    for its sizes and parameters; a scheduler thread admits queued requests in
//    arrival order while a slot is free and the admitted footprints stay within
//    the budget (sets excluded).  A request larger than the whole budget is
//    refused at submission (CH_EBUSY).
//  * Each slot owns a context (stream) and a worker thread; an admitted
//    request's workspace comes from the server's stream-ordered pool, so
//    requests of different sizes overlap on the device without reallocations.
//  * Latency is submit -> result on the host; results are a pure function of
//    (sets, parameters), so a request returns the same bits alone or mixed.
//  * Waits are bounded (ch_serve_wait's timeout); host-side fault hooks
//    (CH_SERVE_FAULT=launch|slow|admit) exercise the failure paths without
//    touching the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace chx {
size_t estimate_footprint(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p);
}

using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket = 0;
  uint64_t a = 0, b = 0;
  ch_est_params p{};
  size_t footprint = 0;
  Clock::time_point t_submit, t_done;
  bool done = false;
  ch_status status = CH_EAGAIN;
  double eta = 0.0;
};

enum class Fault { none, launch, slow, admit };

Fault fault_from_env() {
  const char* f = std::getenv("CH_SERVE_FAULT");
  if (!f) return Fault::none;
  if (!std::strcmp(f, "launch")) return Fault::launch;
  if (!std::strcmp(f, "slow")) return Fault::slow;
  if (!std::strcmp(f, "admit")) return Fault::admit;
  return Fault::none;
}

}  // namespace

struct ch_server {
  ch_ctx* main = nullptr;  // registration context (sets live on its device and pool)
  ch_serve_config cfg{};
  Fault fault = Fault::none;
  std::mutex reg_mu;  // serialises use of the registration context
  std::mutex mu;      // everything below
  std::condition_variable cv_sched, cv_slot, cv_done;
  std::unordered_map<uint64_t, ch_set*> sets;
  uint64_t next_set = 1;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<ch_ctx*> slot_ctx;
  std::vector<std::shared_ptr<Request>> slot_req;
  int64_t in_use = 0, peak = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::thread scheduler;
  std::vector<double> lat_us;
  int64_t completed = 0, failed = 0, rejected = 0, launched = 0;
  Clock::time_point t_create;
  bool indexed = false;  // registered sets keep their l2 embedding under index_hp resident
  ch_hash_params index_hp{};
};

namespace {

void scheduler_loop(ch_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_sched.wait(lk, [&] {
      if (s->stop) return true;
      if (s->queue.empty()) return false;
      const bool free_slot = std::any_of(s->slot_req.begin(), s->slot_req.end(), [](auto& r) { return !r; });
      return free_slot && s->in_use + int64_t(s->queue.front()->footprint) <= s->cfg.hbm_budget_bytes;
    });
    if (s->stop) return;
    auto r = s->queue.front();
    s->queue.pop_front();
    for (size_t i = 0; i < s->slot_req.size(); ++i)
      if (!s->slot_req[i]) {
        s->slot_req[i] = r;
        break;
      }
    s->in_use += int64_t(r->footprint);
    s->peak = std::max(s->peak, s->in_use);
    s->cv_slot.notify_all();
  }
}

// one slot: run the request on the slot's context with a pool-backed workspace
ch_status run_request(ch_server* s, ch_ctx* c, Request& r, double* eta) {
  ch_set *A, *B;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    A = s->sets.at(r.a);
    B = s->sets.at(r.b);
  }
  if (s->fault == Fault::launch) return CH_ECUDA;  // injected launch failure
  if (s->fault == Fault::slow) std::this_thread::sleep_for(std::chrono::milliseconds(50));
  void* ws = nullptr;
  if (cudaSetDevice(c->device) != cudaSuccess) return CH_ECUDA;
  if (cudaMallocFromPoolAsync(&ws, r.footprint + 256, s->main->pool, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return CH_ENOMEM;
  }
  c->ws.base = static_cast<char*>(ws);
  c->ws.cap = r.footprint + 256;
  c->ws.used = 0;
  c->ws.borrowed = true;
  const ch_status st = ch_estimate(c, A, B, &r.p, eta, nullptr);
  c->ws.base = nullptr;  // the pool owns it; the context must not free it
  c->ws.cap = 0;
  c->ws.borrowed = false;
  cudaFreeAsync(ws, c->stream);
  return st;
}

void worker_loop(ch_server* s, int slot) {
  ch_ctx* c = s->slot_ctx[slot];
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_slot.wait(lk, [&] { return s->stop || s->slot_req[slot]; });
    if (s->stop) return;
    auto r = s->slot_req[slot];
    lk.unlock();
    double eta = 0.0;
    const ch_status st = run_request(s, c, *r, &eta);
    lk.lock();
    r->status = st;
    r->eta = eta;
    r->done = true;
    r->t_done = Clock::now();
    s->lat_us.push_back(std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
    if (st == CH_OK)
      ++s->completed;
    else
      ++s->failed;
    s->in_use -= int64_t(r->footprint);
    s->slot_req[slot].reset();
    s->cv_sched.notify_all();
    s->cv_done.notify_all();
  }
}

void destroy_server(ch_server* s) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  s->cv_slot.notify_all();
  s->cv_done.notify_all();
  if (s->scheduler.joinable()) s->scheduler.join();
  for (auto& w : s->workers)
    if (w.joinable()) w.join();
  for (auto* c : s->slot_ctx) ch_ctx_destroy(c);
  for (auto& kv : s->sets) ch_set_destroy(kv.second);
  if (s->main) ch_ctx_sync(s->main);
  delete s;
}

}  // namespace

extern "C" {

ch_status ch_serve_create(ch_ctx* ctx, const ch_serve_config* cfg, ch_server** out) {
  if (!ctx || !cfg || !out) return CH_EINVAL;
  if (cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->hbm_budget_bytes <= 0 || cfg->max_queue < 1) {
    ctx->err = "serve config: max_slots in 1..64, positive budget and queue";
    return CH_EINVAL;
  }
  ch_server* s = new (std::nothrow) ch_server();
  if (!s) return CH_ENOMEM;
  s->main = ctx;
  s->cfg = *cfg;
  s->fault = fault_from_env();
  s->t_create = Clock::now();
  for (int i = 0; i < cfg->max_slots; ++i) {
    ch_ctx* c = nullptr;
    const ch_status st = ch_ctx_create(ctx->device, nullptr, &c);
    if (st != CH_OK) {
      ctx->err = "serve: slot context creation failed";
      destroy_server(s);
      return st;
    }
    s->slot_ctx.push_back(c);
    s->slot_req.emplace_back();
  }
  for (int i = 0; i < cfg->max_slots; ++i) s->workers.emplace_back(worker_loop, s, i);
  s->scheduler = std::thread(scheduler_loop, s);
  *out = s;
  return CH_OK;
}

ch_status ch_serve_register(ch_server* s, const void* data, int mode, int64_t n, int32_t d, int32_t dtype,
                            const float* row_scales, uint64_t* set_id) {
  if (!s || !set_id) return CH_EINVAL;
  std::lock_guard<std::mutex> reg(s->reg_mu);
  ch_set* X = nullptr;
  ch_status st = ch_set_create(s->main, data, mode, n, d, dtype, row_scales, &X);
  if (st != CH_OK) return st;
  st = ch_set_prepare(s->main, X);
  if (st == CH_OK && s->indexed) st = ch_set_embed(s->main, X, &s->index_hp);
  if (st != CH_OK) {
    ch_set_destroy(X);
    return st;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *set_id = s->next_set++;
  s->sets[*set_id] = X;
  return CH_OK;
}

ch_status ch_serve_index(ch_server* s, const ch_hash_params* hp) {
  if (!s || !hp) return CH_EINVAL;
  if (hp->metric != CH_L1 && hp->metric != CH_L2) return CH_EINVAL;
  if (hp->proj_dim < 1 || hp->proj_dim > 64) return CH_EINVAL;
  std::lock_guard<std::mutex> reg(s->reg_mu);
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->sets.empty()) return CH_EBUSY;
  s->indexed = true;
  s->index_hp = *hp;
  return CH_OK;
}

ch_status ch_serve_submit(ch_server* s, uint64_t setA, uint64_t setB, const ch_est_params* p, uint64_t* ticket) {
  if (!s || !p || !ticket) return CH_EINVAL;
  auto r = std::make_shared<Request>();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto ia = s->sets.find(setA), ib = s->sets.find(setB);
    if (ia == s->sets.end() || ib == s->sets.end()) return CH_EINVAL;
    const ch_set* A = ia->second;
    const ch_set* B = ib->second;
    if (A->d != B->d || A->dtype != B->dtype || B->n < 1) return CH_EINVAL;
    if (p->T < 0 || (p->T == 0 && !(p->eps > 0.0 && p->eps < 1.0))) return CH_EINVAL;
    r->footprint = chx::estimate_footprint(s->slot_ctx[0], A, B, p);
    if (s->fault == Fault::admit || int64_t(r->footprint) > s->cfg.hbm_budget_bytes) {
      ++s->rejected;
      return CH_EBUSY;
    }
    if (int64_t(s->queue.size()) >= s->cfg.max_queue) return CH_EAGAIN;
    r->ticket = s->next_ticket++;
    r->a = setA;
    r->b = setB;
    r->p = *p;
    r->t_submit = Clock::now();
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_sched.notify_all();
  return CH_OK;
}

ch_status ch_serve_poll(ch_server* s, uint64_t ticket, double* eta, int32_t* req_status) {
  if (!s) return CH_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return CH_EINVAL;
  if (!it->second->done) return CH_EAGAIN;
  if (eta) *eta = it->second->eta;
  if (req_status) *req_status = it->second->status;
  s->reqs.erase(it);
  return CH_OK;
}

ch_status ch_serve_wait(ch_server* s, uint64_t ticket, uint32_t timeout_ms, double* eta, int32_t* req_status) {
  if (!s) return CH_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return CH_EINVAL;
  auto r = it->second;
  if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done || s->stop; }) ||
      !r->done)
    return CH_ETIMEOUT;
  if (eta) *eta = r->eta;
  if (req_status) *req_status = r->status;
  s->reqs.erase(ticket);
  return CH_OK;
}

ch_status ch_serve_stats_get(ch_server* s, ch_serve_stats* out) {
  if (!s || !out) return CH_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  std::vector<double> v = s->lat_us;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      const size_t i = static_cast<size_t>(std::min<double>(v.size() - 1, std::ceil(q * v.size()) - 1));
      return v[i];
    };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    double sum = 0.0;
    for (double x : v) sum += x;
    out->mean_us = sum / v.size();
  }
  const double secs = std::chrono::duration<double>(Clock::now() - s->t_create).count();
  out->throughput_rps = secs > 0 ? s->completed / secs : 0.0;
  out->completed = s->completed;
  out->failed = s->failed;
  out->rejected = s->rejected;
  out->pending = static_cast<int64_t>(s->queue.size());
  for (auto& r : s->slot_req)
    if (r) ++out->pending;
  out->peak_bytes = s->peak;
  return CH_OK;
}

ch_status ch_serve_stats_reset(ch_server* s) {
  if (!s) return CH_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_us.clear();
  s->completed = s->failed = s->rejected = 0;
  s->t_create = Clock::now();
  return CH_OK;
}

void ch_serve_destroy(ch_server* s) {
  if (s) destroy_server(s);
}

}  // extern "C"
