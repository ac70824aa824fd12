// The serving loop in host C++ (continuous batching over one index).
//
// Callers submit searches, inserts and deletes from any thread and get a
// ticket each.  One scheduler thread owns the GPU work:
//   - searches that are waiting when one of `streams` slots is free launch
//     together as one batch on that slot's stream (pinned host staging,
//     device buffers, an event per batch), so batches overlap on the device
//     and requests that arrive meanwhile join the next free slot; a batch
//     is held back while free device memory is below min_free_bytes;
//   - updates wait until update_batch of them are pending or the oldest has
//     waited update_wait_s; then the group goes to the update thread, which
//     applies it on its own stream as its net effect (one delete call, one
//     insert call: an id inserted and deleted inside the group never reaches
//     the index, an id deleted and inserted again is deleted first), in
//     arrival order of the groups.  The scheduler keeps launching batches
//     meanwhile: the index's copy-on-write views let every batch read the
//     version current at its launch;
//   - every maintain_every operations a maintenance pass (Sec. 4) runs.  With
//     concurrent maintenance a worker thread prepares it on its own stream
//     (qk_maintain_prepare) while searches go on, updates wait, and the pass
//     is committed as soon as it is ready; otherwise the scheduler runs it in
//     place.  Neither waits for the batches in flight.  A pass also needs
//     min_window queries since the previous one (its statistics window).
// A request's latency runs from its submission to the moment its result is in
// host memory.  Every GPU step is a call of the index's own C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "index.cuh"

using namespace qk;

namespace {

using Clock = std::chrono::steady_clock;

struct Op {
  int64_t ticket;
  int kind;              // 0 search, 1 insert, 2 delete
  int64_t id;            // inserted / deleted id
  Clock::time_point t;   // submission
};

struct Result {
  std::atomic<int32_t> done{0};
  double latency_s = 0.0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t event = nullptr;
  float* q_host = nullptr;
  int64_t* ids_host = nullptr;
  float* dist_host = nullptr;
  float* q_dev = nullptr;
  int64_t* ids_dev = nullptr;
  float* dist_dev = nullptr;
  std::vector<int64_t> tickets;   // of the batch in flight
  std::vector<Clock::time_point> t0;
  bool busy = false;
  qk_aps_batch* plan = nullptr;   // batched APS workspace of this slot (null: qk_search only)
};

}  // namespace

struct qk_server {
  qk_index* ix = nullptr;
  qk_server_config cfg{};
  std::vector<double> lam_s, lam_us;
  qk_maint_params maint{};
  int d = 0;
  int device = 0;
  // submissions
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Op> searches, updates;
  std::deque<std::vector<float>> search_q; // queries of the waiting searches (same order as `searches`)
  std::unordered_map<int64_t, std::vector<float>> insert_vecs;
  int64_t next_ticket = 0;
  bool stopping = false;
  // results (grown under mu; read without it once done is set)
  std::deque<Result> results;
  std::vector<int64_t> res_ids;            // k per ticket
  std::vector<float> res_dist;
  std::mutex res_mu;
  // scheduler state
  std::vector<Slot> slots;
  std::thread scheduler;
  std::thread preparer;
  std::atomic<int> prep_state{0};          // 0 idle, 1 running, 2 ready, 3 failed
  std::string prep_error;
  cudaStream_t maint_stream = nullptr;
  cudaStream_t update_stream = nullptr;
  // the update thread and its queue of groups (upd_busy: queued or running)
  std::thread updater;
  mutable std::mutex upd_mu;
  std::condition_variable upd_cv;
  std::deque<std::vector<Op>> upd_groups;
  int upd_busy = 0;
  bool upd_stop = false;
  bool hold_updates = false;   // a maintenance pass is due: take no new group until it has started
  // drain handshake: the scheduler acknowledges a request once it has passed
  // its maintenance step with no pass due or being prepared
  std::atomic<int64_t> drain_req{0}, drain_ack{0};
  int64_t ops_seen = 0, passes = 0, searched_since = 0;
  // statistics
  std::atomic<int64_t> n_search{0}, n_insert{0}, n_delete{0}, batches{0}, drains{0};
  double update_s = 0.0, maint_stall_s = 0.0, maint_prepare_s = 0.0;
  // the first failure: error is written under err_mu before failed is set,
  // and read under err_mu by the threads that see failed
  std::atomic<int32_t> failed{0};
  std::mutex err_mu;
  std::string error;
};

namespace {

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

void set_done(qk_server* sv, int64_t ticket, Clock::time_point t0, Clock::time_point now) {
  Result* r;
  {
    std::lock_guard<std::mutex> g(sv->res_mu);
    r = &sv->results[(size_t)ticket];
  }
  r->latency_s = secs(t0, now);
  r->done.store(1, std::memory_order_release);
}

void finish_slot(qk_server* sv, Slot& s) {
  const int k = sv->cfg.k;
  const auto now = Clock::now();
  {
    std::lock_guard<std::mutex> g(sv->res_mu);
    for (size_t j = 0; j < s.tickets.size(); ++j) {
      std::memcpy(&sv->res_ids[(size_t)s.tickets[j] * k], s.ids_host + j * k, sizeof(int64_t) * k);
      std::memcpy(&sv->res_dist[(size_t)s.tickets[j] * k], s.dist_host + j * k, sizeof(float) * k);
    }
  }
  for (size_t j = 0; j < s.tickets.size(); ++j) set_done(sv, s.tickets[j], s.t0[j], now);
  sv->n_search += (int64_t)s.tickets.size();
  s.tickets.clear();
  s.t0.clear();
  s.busy = false;
}

// Stops the server with msg unless an earlier failure did.
void set_failed(qk_server* sv, const std::string& msg) {
  std::lock_guard<std::mutex> g(sv->err_mu);
  if (sv->failed.load()) return;
  sv->error = msg;
  sv->failed.store(1);
}

std::string stopped_error(qk_server* sv) {
  std::lock_guard<std::mutex> g(sv->err_mu);
  return "the server stopped after an error: " + sv->error;
}

bool fail(qk_server* sv, qk_status st, const char* what) {
  if (st == QK_OK) return false;
  set_failed(sv, std::string(what) + ": " + qk_last_error());
  return true;
}

bool free_ok(qk_server* sv) {
  if (sv->cfg.min_free_bytes <= 0) return true;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return true;
  return (int64_t)fr >= sv->cfg.min_free_bytes;
}

// Applies a group of updates as its net effect (see the file comment).
void apply_updates(qk_server* sv, std::vector<Op>& group) {
  const auto c0 = Clock::now();
  struct St {
    bool del = false;
    int64_t ins = -1;   // position in group of the live insert
  };
  std::unordered_map<int64_t, St> state;
  for (size_t j = 0; j < group.size(); ++j) {
    St& s = state[group[j].id];
    if (group[j].kind == 1) s.ins = (int64_t)j;
    else if (s.ins >= 0) s.ins = -1;
    else s.del = true;
  }
  std::vector<int64_t> del_ids, ins_ids;
  std::vector<float> ins_x;
  {
    std::unordered_map<int64_t, bool> seen;
    for (const Op& o : group)
      if (o.kind == 2 && state[o.id].del && !seen[o.id]) {
        seen[o.id] = true;
        del_ids.push_back(o.id);
      }
  }
  std::vector<int64_t> pos;
  for (auto& kv : state)
    if (kv.second.ins >= 0) pos.push_back(kv.second.ins);
  std::sort(pos.begin(), pos.end());
  {
    std::lock_guard<std::mutex> g(sv->mu);
    for (int64_t p : pos) {
      const Op& o = group[(size_t)p];
      auto it = sv->insert_vecs.find(o.ticket);
      ins_ids.push_back(o.id);
      ins_x.insert(ins_x.end(), it->second.begin(), it->second.end());
    }
    for (const Op& o : group)
      if (o.kind == 1) sv->insert_vecs.erase(o.ticket);
  }
  if (!del_ids.empty()) {
    int64_t removed = 0;
    fail(sv, qk_delete(sv->ix, del_ids.data(), (int64_t)del_ids.size(), &removed, sv->update_stream), "delete");
  }
  if (!ins_ids.empty())
    fail(sv, qk_insert(sv->ix, ins_x.data(), ins_ids.data(), (int64_t)ins_ids.size(), sv->update_stream),
         "insert");
  const auto now = Clock::now();
  for (const Op& o : group) {
    set_done(sv, o.ticket, o.t, now);
    if (o.kind == 1) ++sv->n_insert;
    else ++sv->n_delete;
  }
  ++sv->drains;
  std::lock_guard<std::mutex> g(sv->upd_mu);
  sv->update_s += secs(c0, now);
}

// The update thread: applies the queued groups one after the other.
void updater_loop(qk_server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<Op> group;
    {
      std::unique_lock<std::mutex> lk(sv->upd_mu);
      sv->upd_cv.wait(lk, [&] { return sv->upd_stop || !sv->upd_groups.empty(); });
      if (sv->upd_groups.empty()) return;
      group = std::move(sv->upd_groups.front());
      sv->upd_groups.pop_front();
    }
    try {
      apply_updates(sv, group);
    } catch (const std::exception& e) {
      set_error(std::string("update thread: ") + e.what());
      fail(sv, QK_ERR_INTERNAL, "update thread");
    }
    {
      std::lock_guard<std::mutex> lk(sv->upd_mu);
      --sv->upd_busy;
    }
    sv->cv.notify_all();
  }
}

void queue_updates(qk_server* sv, std::vector<Op>&& group) {
  {
    std::lock_guard<std::mutex> lk(sv->upd_mu);
    sv->upd_groups.push_back(std::move(group));
    ++sv->upd_busy;
  }
  sv->upd_cv.notify_one();
}

bool updates_idle(qk_server* sv) {
  std::lock_guard<std::mutex> lk(sv->upd_mu);
  return sv->upd_busy == 0;
}

void run_prepare(qk_server* sv) {
  cudaSetDevice(sv->device);
  const qk_status st = qk_maintain_prepare(sv->ix, &sv->maint, nullptr, 0, nullptr, sv->maint_stream);
  if (st != QK_OK) {
    sv->prep_error = qk_last_error();
    sv->prep_state.store(3);
  } else {
    sv->prep_state.store(2);
  }
}

void scheduler_body(qk_server* sv) {
  cudaSetDevice(sv->device);
  const int d = sv->d;
  const int64_t min_window =
      sv->cfg.maintain_every > 0 ? std::max<int64_t>(1, std::min<int64_t>(1000, sv->cfg.maintain_every / 10)) : 1;
  Clock::time_point prep_t0{};
  for (;;) {
    const int64_t drain_req = sv->drain_req.load();
    // finished batches
    for (Slot& s : sv->slots)
      if (s.busy && cudaEventQuery(s.event) == cudaSuccess) finish_slot(sv, s);
    // a prepared maintenance pass: commit (the batches in flight keep the old structure)
    const int ps = sv->prep_state.load();
    if (ps == 2 || ps == 3) {
      sv->preparer.join();
      const auto c0 = Clock::now();
      if (ps == 2) fail(sv, qk_maintain_commit(sv->ix, sv->maint_stream), "maintain_commit");
      else set_failed(sv, "maintain_prepare: " + sv->prep_error);
      sv->searched_since = 0;
      {
        std::lock_guard<std::mutex> g(sv->upd_mu);   // the statistics read them
        ++sv->passes;
        sv->maint_stall_s += secs(c0, Clock::now());
        sv->maint_prepare_s += secs(prep_t0, c0);
      }
      sv->prep_state.store(0);
    }
    const bool preparing = sv->prep_state.load() == 1;
    // take the due updates (not while a pass is being prepared or is due)
    std::vector<Op> group;
    bool maint_due = false;
    {
      std::unique_lock<std::mutex> g(sv->mu);
      if (!preparing && !sv->hold_updates && !sv->updates.empty()) {
        const double waited = secs(sv->updates.front().t, Clock::now());
        if ((int64_t)sv->updates.size() >= sv->cfg.update_batch || waited >= sv->cfg.update_wait_s ||
            (sv->searches.empty() && sv->stopping)) {
          group.assign(sv->updates.begin(), sv->updates.end());
          sv->updates.clear();
        }
      }
      maint_due = sv->cfg.maintain_every > 0 && sv->prep_state.load() == 0 &&
                  sv->ops_seen / sv->cfg.maintain_every > sv->passes && sv->searched_since >= min_window;
    }
    if (!group.empty()) queue_updates(sv, std::move(group));
    if (maint_due) {
      // the pass plans from the current index: the pending updates go first,
      // and no new group is taken until the update thread is idle
      if (!sv->hold_updates) {
        std::vector<Op> pending;
        {
          std::lock_guard<std::mutex> g(sv->mu);
          pending.assign(sv->updates.begin(), sv->updates.end());
          sv->updates.clear();
          sv->hold_updates = true;
        }
        if (!pending.empty()) queue_updates(sv, std::move(pending));
      }
      if (updates_idle(sv)) {
        {
          std::lock_guard<std::mutex> g(sv->mu);
          sv->hold_updates = false;
        }
        if (sv->cfg.concurrent_maintenance) {
          prep_t0 = Clock::now();
          sv->prep_state.store(1);
          sv->preparer = std::thread(run_prepare, sv);
        } else {
          const auto c0 = Clock::now();
          fail(sv, qk_maintain(sv->ix, &sv->maint, nullptr, 0, nullptr, sv->update_stream), "maintain");
          sv->searched_since = 0;
          std::lock_guard<std::mutex> g(sv->upd_mu);
          ++sv->passes;
          sv->maint_stall_s += secs(c0, Clock::now());
        }
      }
    }
    {
      bool quiet;
      {
        std::lock_guard<std::mutex> g(sv->mu);
        quiet = !sv->hold_updates;
      }
      if (quiet && sv->prep_state.load() == 0 && updates_idle(sv)) sv->drain_ack.store(drain_req);
    }
    // launch batches while a slot is free and memory allows
    bool launched = false;
    for (;;) {
      Slot* slot = nullptr;
      for (Slot& s : sv->slots)
        if (!s.busy) {
          slot = &s;
          break;
        }
      if (!slot) break;
      std::vector<Op> batch;
      {
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->searches.empty()) break;
        if (!free_ok(sv)) break;
        const size_t n = std::min<size_t>(sv->searches.size(), (size_t)sv->cfg.max_batch);
        for (size_t j = 0; j < n; ++j) {
          batch.push_back(sv->searches.front());
          std::memcpy(slot->q_host + j * d, sv->search_q.front().data(), sizeof(float) * d);
          sv->searches.pop_front();
          sv->search_q.pop_front();
        }
      }
      const int64_t n = (int64_t)batch.size();
      for (const Op& o : batch) {
        slot->tickets.push_back(o.ticket);
        slot->t0.push_back(o.t);
      }
      cudaStream_t st = slot->stream;
      const int k = sv->cfg.k;
      cudaMemcpyAsync(slot->q_dev, slot->q_host, sizeof(float) * n * d, cudaMemcpyHostToDevice, st);
      const qk_status ss =
          slot->plan && n >= sv->cfg.batched_from
              ? qk_aps_batch_search(slot->plan, slot->q_dev, n, sv->cfg.recall_target, slot->ids_dev, slot->dist_dev,
                                    nullptr, nullptr, nullptr, 0, st)
              : qk_search(sv->ix, slot->q_dev, n, k, sv->cfg.recall_target, 0, slot->ids_dev, slot->dist_dev, nullptr,
                          nullptr, st);
      if (fail(sv, ss, "search")) {
        slot->tickets.clear();
        slot->t0.clear();
        break;
      }
      cudaMemcpyAsync(slot->ids_host, slot->ids_dev, sizeof(int64_t) * n * k, cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(slot->dist_host, slot->dist_dev, sizeof(float) * n * k, cudaMemcpyDeviceToHost, st);
      cudaEventRecord(slot->event, st);
      slot->busy = true;
      sv->searched_since += n;
      ++sv->batches;
      launched = true;
    }
    // leave when stopping with nothing left; otherwise wait a little for work
    bool any_busy = false;
    for (Slot& s : sv->slots) any_busy |= s.busy;
    if (launched) continue;
    if (any_busy) {   // batches in flight: poll their events soon
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      continue;
    }
    std::unique_lock<std::mutex> g(sv->mu);
    if (sv->stopping && sv->searches.empty() && sv->updates.empty() && sv->prep_state.load() == 0 &&
        !sv->hold_updates && updates_idle(sv))   // a due pass still runs
      return;
    sv->cv.wait_for(g, std::chrono::microseconds(200));
  }
}

// A host exception in the scheduler (a failed allocation) stops the server as
// a failed call does: the error is kept and returned by drain and submissions.
void scheduler_loop(qk_server* sv) {
  try {
    scheduler_body(sv);
  } catch (const std::exception& e) {
    set_error(std::string("scheduler: ") + e.what());
    fail(sv, QK_ERR_INTERNAL, "scheduler");
  }
}

// A request whose latency counts from `at` (its arrival; now for the public
// submit calls).
qk_status submit(qk_server* sv, int kind, const float* x, int64_t id, int64_t* ticket,
                 Clock::time_point at = Clock::time_point{}) {
  if (!sv || !ticket) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  if (sv->failed.load()) {
    set_error(stopped_error(sv));
    return QK_ERR_STATE;
  }
  if (kind != 2) {
    // a vector the kernels would refuse is refused here, so that one bad
    // request cannot stop the server: every element finite, squared norm
    // within FP32
    if (!x) {
      set_error("null vector");
      return QK_ERR_ARG;
    }
    double n2 = 0.0;
    for (int j = 0; j < sv->d; ++j) n2 += (double)x[j] * (double)x[j];
    if (!(n2 < 1e38)) {
      set_error("vector with a NaN or infinite element, or a squared norm beyond FP32");
      return QK_ERR_ARG;
    }
  }
  const int k = sv->cfg.k;
  std::lock_guard<std::mutex> g(sv->mu);
  if (sv->stopping) {
    set_error("the server is stopping");
    return QK_ERR_STATE;
  }
  const int64_t t = sv->next_ticket++;
  {
    std::lock_guard<std::mutex> gr(sv->res_mu);
    sv->results.emplace_back();
    sv->res_ids.resize((size_t)(t + 1) * k, -1);
    sv->res_dist.resize((size_t)(t + 1) * k, INFINITY);
  }
  Op o{t, kind, id, at == Clock::time_point{} ? Clock::now() : at};
  if (kind == 0) {
    sv->searches.push_back(o);
    sv->search_q.emplace_back(x, x + sv->d);
  } else {
    if (kind == 1) sv->insert_vecs.emplace(t, std::vector<float>(x, x + sv->d));
    sv->updates.push_back(o);
  }
  ++sv->ops_seen;
  *ticket = t;
  sv->cv.notify_one();
  return QK_OK;
}

}  // namespace

extern "C" {

void qk_server_config_default(qk_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->k = 10;
  c->recall_target = 0.9f;
  c->max_batch = 2048;
  c->streams = 4;
  c->min_free_bytes = 1LL << 30;
  c->maintain_every = 0;
  c->update_batch = 1024;
  c->update_wait_s = 0.01;
  c->concurrent_maintenance = 1;
  c->maint = nullptr;
  c->batched_from = 0;
}

qk_status qk_server_create(qk_index* ix, const qk_server_config* cfg, qk_server** out) {
  QK_GUARD_BEGIN
  if (!ix || !cfg || !out) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  *out = nullptr;
  if (!ix->ready) {
    set_error("index is empty: build or load it first");
    return QK_ERR_STATE;
  }
  if (cfg->k < 1 || cfg->k > 1024 || cfg->max_batch < 1 || cfg->streams < 1 || cfg->streams > kWorkSlots ||
      cfg->update_batch < 1 || !(cfg->update_wait_s >= 0) || cfg->maintain_every < 0 ||
      (cfg->maintain_every > 0 && !cfg->maint) || cfg->batched_from < 0) {
    set_error("invalid server configuration");
    return QK_ERR_ARG;
  }
  qk_server* sv = new qk_server();
  sv->ix = ix;
  sv->cfg = *cfg;
  sv->d = ix->cfg.d;
  cudaGetDevice(&sv->device);
  if (cfg->maint) {   // the pass parameters are copied, lambda table included
    sv->maint = *cfg->maint;
    sv->lam_s.assign(cfg->maint->lambda_sizes, cfg->maint->lambda_sizes + cfg->maint->lambda_points);
    sv->lam_us.assign(cfg->maint->lambda_us, cfg->maint->lambda_us + cfg->maint->lambda_points);
    sv->maint.lambda_sizes = sv->lam_s.data();
    sv->maint.lambda_us = sv->lam_us.data();
    sv->cfg.maint = &sv->maint;
  }
  const int d = sv->d, k = cfg->k, mb = cfg->max_batch;
  qk_status st = QK_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && st == QK_OK) st = cuda_status(e, "server buffers");
  };
  // stream priorities: updates (short kernels) first, then the search
  // batches, then the maintenance pass prepared beside them (the default,
  // lowest priority), so a pass's long kernels give way to the batches
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  const int prio_search = prio_hi < prio_lo ? prio_hi + 1 : prio_hi;
  sv->slots.resize(cfg->streams);
  for (Slot& s : sv->slots) {
    ck(cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, prio_search));
    ck(cudaEventCreateWithFlags(&s.event, cudaEventDisableTiming));
    ck(cudaMallocHost(&s.q_host, sizeof(float) * mb * d));
    ck(cudaMallocHost(&s.ids_host, sizeof(int64_t) * mb * k));
    ck(cudaMallocHost(&s.dist_host, sizeof(float) * mb * k));
    ck(cudaMalloc(&s.q_dev, sizeof(float) * mb * d));
    ck(cudaMalloc(&s.ids_dev, sizeof(int64_t) * mb * k));
    ck(cudaMalloc(&s.dist_dev, sizeof(float) * mb * k));
  }
  ck(cudaStreamCreateWithFlags(&sv->maint_stream, cudaStreamNonBlocking));
  ck(cudaStreamCreateWithPriority(&sv->update_stream, cudaStreamNonBlocking, prio_hi));
  // a batched APS plan per slot where the index's form allows it; without one
  // every batch runs through qk_search
  if (st == QK_OK && cfg->batched_from > 0 && cfg->batched_from <= mb && ix->cfg.metric == QK_METRIC_L2 &&
      ix->cfg.storage == QK_STORE_F32 && k <= 32) {
    for (Slot& s : sv->slots)
      if (qk_aps_batch_create(ix, mb, k, &s.plan) != QK_OK) s.plan = nullptr;
  }
  if (st != QK_OK) {
    qk_server_destroy(sv);
    return st;
  }
  sv->updater = std::thread(updater_loop, sv);
  sv->scheduler = std::thread(scheduler_loop, sv);
  *out = sv;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_server_submit_search(qk_server* sv, const float* q, int64_t* ticket) {
  QK_GUARD_BEGIN
  if (!q) {
    set_error("null query");
    return QK_ERR_ARG;
  }
  return submit(sv, 0, q, -1, ticket);
  QK_GUARD_END
}

qk_status qk_server_submit_insert(qk_server* sv, const float* x, int64_t id, int64_t* ticket) {
  QK_GUARD_BEGIN
  if (!x) {
    set_error("null vector");
    return QK_ERR_ARG;
  }
  return submit(sv, 1, x, id, ticket);
  QK_GUARD_END
}

qk_status qk_server_submit_delete(qk_server* sv, int64_t id, int64_t* ticket) {
  QK_GUARD_BEGIN
  return submit(sv, 2, nullptr, id, ticket);
  QK_GUARD_END
}

qk_status qk_server_play(qk_server* sv, int64_t n, const int8_t* kind, const int64_t* ref, const float* vec,
                         const double* t_s, double* lag_s) {
  QK_GUARD_BEGIN
  if (!sv || n < 0 || (n > 0 && (!kind || !ref || !t_s))) {
    set_error("invalid arguments");
    return QK_ERR_ARG;
  }
  const Clock::time_point t0 = Clock::now();
  int64_t ticket = 0;
  for (int64_t j = 0; j < n; ++j) {
    const Clock::time_point due =
        t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(t_s[j]));
    Clock::time_point now = Clock::now();
    if (due - now > std::chrono::microseconds(200)) std::this_thread::sleep_for(due - now - std::chrono::microseconds(100));
    while ((now = Clock::now()) < due) {
    }
    if (lag_s) lag_s[j] = secs(due, now);
    const int kd = kind[j];
    if (kd < 0 || kd > 2 || (kd != 2 && !vec)) {
      set_error("operation " + std::to_string(j) + ": invalid kind or missing vector");
      return QK_ERR_ARG;
    }
    QK_TRY(submit(sv, kd, kd == 2 ? nullptr : vec + j * (int64_t)sv->d, kd == 0 ? -1 : ref[j], &ticket, due));
  }
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_server_results(qk_server* sv, int64_t first, int64_t count, int32_t* done, int64_t* ids,
                            float* dist, double* latency_s) {
  QK_GUARD_BEGIN
  if (!sv || count < 0 || first < 0) {
    set_error("invalid arguments");
    return QK_ERR_ARG;
  }
  const int k = sv->cfg.k;
  std::lock_guard<std::mutex> g(sv->res_mu);
  if (first + count > (int64_t)sv->results.size()) {
    set_error("ticket out of range");
    return QK_ERR_ARG;
  }
  for (int64_t j = 0; j < count; ++j) {
    const Result& r = sv->results[(size_t)(first + j)];
    const int32_t dn = r.done.load(std::memory_order_acquire);
    if (done) done[j] = dn;
    if (latency_s) latency_s[j] = dn ? r.latency_s : -1.0;
    if (ids) std::memcpy(ids + j * k, &sv->res_ids[(size_t)(first + j) * k], sizeof(int64_t) * k);
    if (dist) std::memcpy(dist + j * k, &sv->res_dist[(size_t)(first + j) * k], sizeof(float) * k);
  }
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_server_drain(qk_server* sv, double timeout_s) {
  QK_GUARD_BEGIN
  if (!sv) {
    set_error("null server");
    return QK_ERR_ARG;
  }
  const auto t0 = Clock::now();
  for (;;) {
    if (sv->failed.load()) {
      set_error(stopped_error(sv));
      return QK_ERR_STATE;
    }
    int64_t n;
    {
      std::lock_guard<std::mutex> g(sv->res_mu);
      n = (int64_t)sv->results.size();
    }
    bool all = true;
    {
      std::lock_guard<std::mutex> g(sv->res_mu);
      for (int64_t j = n - 1; j >= 0 && all; --j) all = sv->results[(size_t)j].done.load() != 0;
    }
    if (all) {
      // every request is answered; a maintenance pass they made due must also
      // have run: wait for the scheduler to pass its maintenance step once more
      const int64_t req = ++sv->drain_req;
      while (sv->drain_ack.load() < req) {
        if (sv->failed.load()) {
          set_error(stopped_error(sv));
          return QK_ERR_STATE;
        }
        if (timeout_s > 0 && secs(t0, Clock::now()) > timeout_s) {
          set_error("drain timed out");
          return QK_ERR_TIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
      }
      return QK_OK;
    }
    if (timeout_s > 0 && secs(t0, Clock::now()) > timeout_s) {
      set_error("drain timed out");
      return QK_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  QK_GUARD_END
}

qk_status qk_server_get_stats(const qk_server* sv, qk_server_stats* out) {
  QK_GUARD_BEGIN
  if (!sv || !out) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  out->searches = sv->n_search.load();
  out->inserts = sv->n_insert.load();
  out->deletes = sv->n_delete.load();
  out->batches = sv->batches.load();
  out->update_groups = sv->drains.load();
  {
    std::lock_guard<std::mutex> lk(sv->upd_mu);
    out->maintenance_passes = sv->passes;
    out->update_s = sv->update_s;
    out->maintenance_stall_s = sv->maint_stall_s;
    out->maintenance_prepare_s = sv->maint_prepare_s;
  }
  return QK_OK;
  QK_GUARD_END
}

void qk_server_destroy(qk_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    sv->stopping = true;
  }
  sv->cv.notify_all();
  if (sv->scheduler.joinable()) sv->scheduler.join();
  if (sv->preparer.joinable()) sv->preparer.join();
  {
    std::lock_guard<std::mutex> lk(sv->upd_mu);
    sv->upd_stop = true;
  }
  sv->upd_cv.notify_all();
  if (sv->updater.joinable()) sv->updater.join();
  for (Slot& s : sv->slots) {
    if (s.busy && s.event) cudaEventSynchronize(s.event);
    if (s.event) cudaEventDestroy(s.event);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.q_host) cudaFreeHost(s.q_host);
    if (s.ids_host) cudaFreeHost(s.ids_host);
    if (s.dist_host) cudaFreeHost(s.dist_host);
    if (s.q_dev) cudaFree(s.q_dev);
    if (s.ids_dev) cudaFree(s.ids_dev);
    if (s.dist_dev) cudaFree(s.dist_dev);
    if (s.plan) qk_aps_batch_destroy(s.plan);
  }
  if (sv->maint_stream) cudaStreamDestroy(sv->maint_stream);
  if (sv->update_stream) cudaStreamDestroy(sv->update_stream);
  delete sv;
}

}  // extern "C"
