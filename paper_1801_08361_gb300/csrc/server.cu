// server.cu -- the serving runtime: relocalisation attempts submitted one by one by many agents
// (threads), admitted into a fixed pool of request slots and run in batches by a worker thread.
//
// The paper relocalises one attempt at a time in the background (Sec. 3.3.1, Sec. 4.3.1) and
// passes frames between threads through pooled queues whose full pool discards new items
// (Appendix B.1).  Here the pool holds the requests; a request that finds no free slot is
// discarded (RELO_EBUSY).  Batches form from the front of the queue under the HBM budget of one
// batch's workspace and run through relo_relocalise_batch on the worker's own stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/relo.h"

namespace relo {
cudaError_t dev_malloc(void** p, size_t bytes);  // the library's device allocations (api.cu)
void dev_free(void* p);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Slot {
  enum State { kFree, kQueued, kRunning, kDone } state = kFree;
  uint64_t ticket = 0;
  relo_attempt attempt{};
  relo_pose_result result{};
  Clock::time_point t_submit, t_done;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct relo_server {
  relo_server_params p{};
  int device = 0;
  void* ws = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<Slot> slots;
  std::vector<int> free_slots;
  std::deque<int> queue;                        // queued slots, oldest first
  std::unordered_map<uint64_t, int> by_ticket;  // live tickets -> slot
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
  // statistics
  std::vector<double> latencies;
  uint64_t discarded = 0, batches = 0, batched = 0;

  void run();
  void run_batch(const std::vector<int>& pick);
};

// One batch outside the lock: the picked slots are RUNNING, so no other thread touches them.
void relo_server::run_batch(const std::vector<int>& pick) {
  std::vector<relo_attempt> att(pick.size());
  for (size_t k = 0; k < pick.size(); ++k) att[k] = slots[pick[k]].attempt;
  std::vector<relo_pose_result> res(pick.size());
  const relo_status st = relo_relocalise_batch(att.data(), (int32_t)att.size(), &p.ransac, ws,
                                               (size_t)p.workspace_bytes, res.data(), (relo_stream)stream);
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lk(mu);
  for (size_t k = 0; k < pick.size(); ++k) {
    Slot& s = slots[pick[k]];
    s.result = res[k];
    if (st != RELO_OK) {
      s.result = relo_pose_result{};
      s.result.status = st;
    }
    s.state = Slot::kDone;
    s.t_done = now;
    latencies.push_back(ms_between(s.t_submit, now));
  }
  batches += 1;
  batched += pick.size();
  cv_done.notify_all();
}

void relo_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv_work.wait(lk, [&] { return stop || !queue.empty(); });
    if (queue.empty()) break;  // stopping, nothing left to run
    // a partial batch waits for more requests until its oldest has waited max_wait_us
    const Clock::time_point deadline = slots[queue.front()].t_submit + std::chrono::microseconds(p.max_wait_us);
    cv_work.wait_until(lk, deadline, [&] { return stop || (int)queue.size() >= p.max_batch; });
    // admission: take requests from the front while the batch's workspace fits the budget
    std::vector<int> pick;
    std::vector<relo_attempt> cand;
    while (!queue.empty() && (int)pick.size() < p.max_batch) {
      cand.push_back(slots[queue.front()].attempt);
      const size_t need = relo_batch_workspace_size(cand.data(), (int32_t)cand.size(), &p.ransac);
      if (need == 0 || need > p.workspace_bytes) {
        cand.pop_back();
        break;
      }
      pick.push_back(queue.front());
      queue.pop_front();
    }
    if (pick.empty()) {
      // the front request alone exceeds the budget: it completes with RELO_EINVAL
      Slot& s = slots[queue.front()];
      queue.pop_front();
      s.result = relo_pose_result{};
      s.result.status = RELO_EINVAL;
      s.state = Slot::kDone;
      s.t_done = Clock::now();
      cv_done.notify_all();
      continue;
    }
    for (int i : pick) slots[i].state = Slot::kRunning;
    lk.unlock();
    run_batch(pick);
    lk.lock();
  }
}

extern "C" {

relo_status relo_server_create(const relo_server_params* params, relo_server** out) {
  if (!out) return RELO_EINVAL;
  *out = nullptr;
  if (!params || params->max_batch < 1 || params->max_wait_us < 0 || params->slots < 1 ||
      params->workspace_bytes == 0)
    return RELO_EINVAL;
  relo_server* s = new relo_server();
  s->p = *params;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return RELO_ECUDA;
  }
  if (relo::dev_malloc((void**)&s->ws, (size_t)params->workspace_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return RELO_ENOMEM;
  }
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    relo::dev_free(s->ws);
    delete s;
    return RELO_ECUDA;
  }
  s->slots.resize(params->slots);
  for (int i = params->slots - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return RELO_OK;
}

relo_status relo_server_submit(relo_server* s, const relo_attempt* a, uint64_t* ticket) {
  if (!s || !a || !ticket) return RELO_EINVAL;
  if (relo_batch_workspace_size(a, 1, &s->p.ransac) == 0) return RELO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return RELO_EINVAL;
  if (s->free_slots.empty()) {
    s->discarded += 1;  // the pooled queue's discard policy
    return RELO_EBUSY;
  }
  const int i = s->free_slots.back();
  s->free_slots.pop_back();
  Slot& slot = s->slots[i];
  slot.state = Slot::kQueued;
  slot.ticket = s->next_ticket++;
  slot.attempt = *a;
  slot.t_submit = Clock::now();
  s->by_ticket[slot.ticket] = i;
  s->queue.push_back(i);
  *ticket = slot.ticket;
  s->cv_work.notify_one();
  return RELO_OK;
}

relo_status relo_server_wait(relo_server* s, uint64_t ticket, relo_pose_result* result, double* latency_ms) {
  if (!s) return RELO_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return RELO_EINVAL;
  const int i = it->second;
  Slot& slot = s->slots[i];
  s->cv_done.wait(lk, [&] { return slot.state == Slot::kDone; });
  if (result) *result = slot.result;
  if (latency_ms) *latency_ms = ms_between(slot.t_submit, slot.t_done);
  slot.state = Slot::kFree;
  s->by_ticket.erase(it);
  s->free_slots.push_back(i);
  return RELO_OK;
}

relo_status relo_server_stats_get(const relo_server* s, relo_server_stats* out) {
  if (!s || !out) return RELO_EINVAL;
  relo_server* m = const_cast<relo_server*>(s);
  std::lock_guard<std::mutex> lk(m->mu);
  relo_server_stats st{};
  st.completed = m->latencies.size();
  st.discarded = m->discarded;
  st.batches = m->batches;
  st.mean_batch = m->batches ? (double)m->batched / (double)m->batches : 0.0;
  if (!m->latencies.empty()) {
    std::vector<double> v(m->latencies);
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
    st.p50_ms = pct(0.50);
    st.p99_ms = pct(0.99);
    st.max_ms = v.back();
  }
  *out = st;
  return RELO_OK;
}

void relo_server_destroy(relo_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaStreamDestroy(s->stream);
  relo::dev_free(s->ws);
  delete s;
}

}  // extern "C"
