// dpf_server: a request loop that keeps join tables and compressed columns
// resident in the context and runs the queries it is given with continuous
// batching.
//
// Queries are admitted by their device footprint (dpf_plan_footprint): a
// query waits in a FIFO queue until the footprint of the queries on the GPU
// plus its own fits the server's budget.  A dispatcher thread keeps up to
// max_inflight batches on the device, each on its own CUDA stream: whenever a
// slot is free it takes the queued queries that fit (up to max_batch) and
// runs them as ONE persistent fused launch (the batched launch of the
// fused kernel, Sec. 3.2's loop over chunks of every query of the batch).
// Queries that arrive while batches run are launched as soon as a slot and
// memory free up, and their work overlaps on the device with the tail of
// the batches still running.  Each query's records are the same as when it
// runs alone: batching only changes which chunks share a launch.
//
// The server is built on the public C ABI (dpf_prepare / dpf_launch /
// dpf_read_result / dpf_release), so every device step runs in the fused
// kernel.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dpf.h"
#include "host_common.h"

namespace {

using Clock = std::chrono::steady_clock;

// A plan with its arrays owned by the request.
struct OwnedPlan {
  std::vector<dpf_pred> preds;
  std::vector<dpf_join> joins;
  std::vector<dpf_key> keys;
  std::vector<dpf_agg> aggs;
  dpf_plan plan{};
  explicit OwnedPlan(const dpf_plan& p) {
    preds.assign(p.preds, p.preds + (p.preds ? p.n_preds : 0));
    joins.assign(p.joins, p.joins + (p.joins ? p.n_joins : 0));
    keys.assign(p.keys, p.keys + (p.keys ? p.n_keys : 0));
    aggs.assign(p.aggs, p.aggs + (p.aggs ? p.n_aggs : 0));
    plan = p;
    plan.preds = preds.empty() ? nullptr : preds.data();
    plan.joins = joins.empty() ? nullptr : joins.data();
    plan.keys = keys.empty() ? nullptr : keys.data();
    plan.aggs = aggs.empty() ? nullptr : aggs.data();
  }
};

struct Request {
  uint64_t ticket = 0;
  std::unique_ptr<OwnedPlan> plan;
  uint64_t bytes = 0;
  double submit_us = 0, launch_us = 0, done_us = 0;
  uint32_t batch = 0;
  bool done = false;
  dpf_status status = DPF_OK;
  std::string error;
  std::vector<dpf_record> records;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  dpf_prep_id prep = 0;
  std::vector<std::shared_ptr<Request>> reqs;
  uint64_t bytes = 0;
};

}  // namespace

struct dpf_server {
  dpf_ctx* ctx = nullptr;
  dpf_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv;       // dispatcher: work arrived / stop
  std::condition_variable done_cv;  // waiters: a request finished
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> all;  // submitted, not yet collected
  std::vector<Slot> slots;
  uint64_t next_ticket = 1;
  uint64_t in_use = 0;
  bool stop = false;
  std::thread thread;
  Clock::time_point t0;
  dpf_server_stats stats{};

  double now_us() const { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); }
  void run();
  void finish_slot(Slot& s);
};

// Reads the records of every query of a completed slot and publishes them.
void dpf_server::finish_slot(Slot& s) {
  const double t = now_us();
  dpf_status batch_status = DPF_OK;
  std::string batch_error;
  for (size_t i = 0; i < s.reqs.size(); ++i) {
    Request& r = *s.reqs[i];
    uint64_t n = 0;
    std::vector<dpf_record> recs(64);
    dpf_status st = dpf_read_result(ctx, s.prep, int32_t(i), recs.data(), recs.size(), &n, -1);
    if (st == DPF_ETRUNC) {
      recs.resize(n);
      st = dpf_read_result(ctx, s.prep, int32_t(i), recs.data(), recs.size(), &n, -1);
    }
    if (st == DPF_OK) {
      recs.resize(n);
      r.records = std::move(recs);
    } else if (batch_status == DPF_OK) {
      batch_status = st;
      batch_error = dpf_last_error();
    }
    r.status = st;
    if (st) r.error = dpf_last_error();
  }
  dpf_release(ctx, s.prep);
  std::lock_guard<std::mutex> lk(mu);
  for (auto& rp : s.reqs) {
    rp->done_us = t;
    rp->done = true;
  }
  stats.completed += s.reqs.size();
  stats.batches += 1;
  in_use -= s.bytes;
  s.reqs.clear();
  s.bytes = 0;
  s.busy = false;
  done_cv.notify_all();
}

void dpf_server::run() {
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // completions
    bool any_busy = false;
    for (Slot& s : slots) {
      if (!s.busy) continue;
      const cudaError_t e = cudaEventQuery(s.ev);
      if (e == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      lk.unlock();
      finish_slot(s);  // also reports a failed launch through dpf_read_result
      lk.lock();
    }
    // launches: FIFO, while a slot is free and the head of the queue fits
    for (Slot& s : slots) {
      if (s.busy || pending.empty()) continue;
      std::vector<std::shared_ptr<Request>> batch;
      uint64_t bytes = 0;
      while (!pending.empty() && batch.size() < cfg.max_batch) {
        const uint64_t b = pending.front()->bytes;
        if (cfg.mem_budget && in_use + bytes + b > cfg.mem_budget) break;
        bytes += b;
        batch.push_back(pending.front());
        pending.pop_front();
      }
      if (batch.empty()) break;  // the head waits for memory
      s.busy = true;
      s.bytes = bytes;
      in_use += bytes;
      const double t = now_us();
      for (auto& r : batch) {
        r->launch_us = t;
        r->batch = uint32_t(batch.size());
      }
      s.reqs = batch;
      lk.unlock();
      std::vector<dpf_plan> plans;
      plans.reserve(batch.size());
      for (auto& r : batch) plans.push_back(r->plan->plan);
      s.prep = 0;
      dpf_status st = dpf_prepare(ctx, plans.data(), int32_t(plans.size()), &cfg.tuning, &s.prep);
      if (st == DPF_OK) st = dpf_launch(ctx, s.prep, s.stream);
      if (st == DPF_OK && cudaEventRecord(s.ev, s.stream) != cudaSuccess) st = DPF_ECUDA;
      if (st != DPF_OK) {
        const std::string err = dpf_last_error();
        if (s.prep) dpf_release(ctx, s.prep);
        lk.lock();
        for (auto& r : batch) {
          r->status = st;
          r->error = err;
          r->done_us = now_us();
          r->done = true;
        }
        in_use -= bytes;
        s.reqs.clear();
        s.bytes = 0;
        s.busy = false;
        stats.failed += batch.size();
        done_cv.notify_all();
        continue;
      }
      lk.lock();
      stats.launched_batches += 1;
      any_busy = true;
    }
    if (stop && pending.empty() && !any_busy) {
      bool idle = true;
      for (Slot& s : slots) idle &= !s.busy;
      if (idle) break;
    }
    if (any_busy) {
      cv.wait_for(lk, std::chrono::microseconds(20));
    } else {
      cv.wait(lk, [&] { return stop || !pending.empty(); });
    }
  }
}

extern "C" dpf_status dpf_server_create(dpf_ctx* ctx, const dpf_server_config* cfg, dpf_server** out) {
  if (!ctx || !out) return dpf::fail(DPF_EINVAL, "NULL argument");
  *out = nullptr;
  auto s = std::make_unique<dpf_server>();
  s->ctx = ctx;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.max_batch == 0) s->cfg.max_batch = 64;
  if (s->cfg.max_inflight == 0) s->cfg.max_inflight = 2;
  if (s->cfg.max_batch > 4096) return dpf::fail(DPF_EINVAL, "max_batch %u above 4096", s->cfg.max_batch);
  if (s->cfg.max_inflight > 64) return dpf::fail(DPF_EINVAL, "max_inflight %u above 64", s->cfg.max_inflight);
  int32_t device = 0;
  dpf_status st = dpf_context_device(ctx, &device);
  if (st) return st;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  s->slots.resize(s->cfg.max_inflight);
  cudaError_t e = cudaSuccess;
  for (Slot& sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    for (Slot& sl : s->slots) {
      if (sl.ev) cudaEventDestroy(sl.ev);
      if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    return dpf::fail(DPF_ECUDA, "dpf_server_create: %s", cudaGetErrorString(e));
  }
  s->t0 = Clock::now();
  dpf_server* raw = s.get();
  s->thread = std::thread([raw, device] {
    cudaSetDevice(device);
    raw->run();
  });
  *out = s.release();
  return DPF_OK;
}

extern "C" dpf_status dpf_server_submit(dpf_server* s, const dpf_plan* plan, uint64_t* ticket) {
  if (!s || !plan || !ticket) return dpf::fail(DPF_EINVAL, "NULL argument");
  uint64_t bytes = 0;
  dpf_status st = dpf_plan_footprint(s->ctx, plan, &bytes);
  if (st) return st;
  if (s->cfg.mem_budget && bytes > s->cfg.mem_budget)
    return dpf::fail(DPF_EBUSY, "query footprint %llu bytes exceeds the server budget %llu",
                     (unsigned long long)bytes, (unsigned long long)s->cfg.mem_budget);
  auto r = std::make_shared<Request>();
  r->plan = std::make_unique<OwnedPlan>(*plan);
  r->bytes = bytes;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return dpf::fail(DPF_EBUSY, "server is stopping");
    r->ticket = s->next_ticket++;
    r->submit_us = s->now_us();
    s->pending.push_back(r);
    s->all[r->ticket] = r;
    s->stats.submitted += 1;
  }
  s->cv.notify_one();
  *ticket = r->ticket;
  return DPF_OK;
}

extern "C" dpf_status dpf_server_wait(dpf_server* s, uint64_t ticket, dpf_record* buf, uint64_t cap,
                                      uint64_t* n_out, int32_t timeout_ms, dpf_query_times* times) {
  if (!s) return dpf::fail(DPF_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return dpf::fail(DPF_ENOTFOUND, "unknown or already collected ticket %llu",
                                           (unsigned long long)ticket);
  std::shared_ptr<Request> r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) {
    s->done_cv.wait(lk, ready);
  } else if (!s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return dpf::fail(DPF_ETIMEOUT, "ticket %llu not done within %d ms", (unsigned long long)ticket, timeout_ms);
  }
  if (times) {
    times->submit_us = r->submit_us;
    times->launch_us = r->launch_us;
    times->done_us = r->done_us;
    times->batch_size = r->batch;
  }
  if (r->status) {
    s->all.erase(ticket);
    return dpf::fail(r->status, "%s", r->error.c_str());
  }
  if (n_out) *n_out = r->records.size();
  if (cap < r->records.size()) return dpf::fail(DPF_ETRUNC, "need %zu records", r->records.size());
  if (!r->records.empty()) {
    if (!buf) return dpf::fail(DPF_EINVAL, "buf is NULL");
    std::memcpy(buf, r->records.data(), r->records.size() * sizeof(dpf_record));
  }
  s->all.erase(ticket);
  return DPF_OK;
}

extern "C" dpf_status dpf_server_stats_get(dpf_server* s, dpf_server_stats* out) {
  if (!s || !out) return dpf::fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queued = s->pending.size();
  out->in_use_bytes = s->in_use;
  return DPF_OK;
}

extern "C" dpf_status dpf_server_destroy(dpf_server* s) {
  if (!s) return DPF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->thread.joinable()) s->thread.join();
  for (Slot& sl : s->slots) {
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
  return DPF_OK;
}
