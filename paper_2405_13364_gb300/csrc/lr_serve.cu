// lr_serve.cu -- serving loop with continuous batching (lr_server_start, lr_submit,
// lr_poll). Not described by the paper; it serves the single-frame pipeline of Sec. 2.
//
// A host thread owns S slots; each slot is a CUDA stream plus a device workspace
// allocated when the server starts (the admission budget). Requests wait in a FIFO queue.
// Whenever a slot is free, the thread takes requests from the front of the queue while
// the batch still fits the slot's workspace (admission by device memory) and the batch
// has fewer than max_batch_views views, and launches them as one multi-view render
// (one launch per pipeline stage for the whole batch). Up to S batches run on the GPU at
// once, on different streams, so requests that arrive while others are being rendered are
// admitted as soon as a slot frees up. A batch holds requests of one sorter capacity
// (lr_view.sorter_k, e.g. each request's autotuned value); a batch launched while no other
// batch is on the GPU uses programmatic dependent launch, which concurrent batches would
// slow down. Each batch's status word is copied back on its own stream before its
// completion event, so a finished batch needs no further synchronisation; while batches
// run, the thread polls their events in a short spin rather than sleeping (a timed sleep
// of a few microseconds can last tens of microseconds under the kernel's timer slack). A
// batch that exceeds its workspace's reference capacity is split and its requests retried
// alone.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lr_common.cuh"
#include "lr_serve.h"

namespace {

using lr::Ctrl;

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Req {
  lr_view view;
  int status = LR_PENDING;
  bool done = false;
  bool alone = false;        // retry without batching
  uint64_t t_submit = 0, t_launch = 0, t_done = 0;
  int batch_views = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t bytes = 0;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<uint64_t> tickets;
  Ctrl* host_ctrl = nullptr;
};

}  // namespace

struct lr_server {
  lr_ctx* inner = nullptr;         // private context: its error text and last-render state
  lr_server_config cfg;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable wake, done_cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::atomic<bool> submitted{false};   // a request was queued since the loop last looked
  std::thread th;
  lr_server_stats stats;
};

// the sorter capacity a request renders with
static int request_k(const lr_server* s, const lr_view& v) {
  return v.sorter_k ? v.sorter_k : lr_internal_config(s->inner)->sorter_k;
}

static void finish(lr_server* s, uint64_t t, int status) {
  auto it = s->reqs.find(t);
  if (it == s->reqs.end()) return;
  it->second.status = status;
  it->second.done = true;
  it->second.t_done = now_ns();
  s->stats.completed++;
  if (status != LR_OK) s->stats.failed++;
}

static void serve_loop(lr_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  std::vector<lr_view> views;
  for (;;) {
    bool progressed = false;
    // ---- completions ---------------------------------------------------------------
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      // the batch's status word was copied to host memory before its event
      const int status = q == cudaSuccess ? sl.host_ctrl->error : LR_ERR_CUDA;
      if (status == LR_ERR_OVERFLOW && sl.tickets.size() > 1) {
        // too many references for a shared workspace: retry each request alone
        for (auto it = sl.tickets.rbegin(); it != sl.tickets.rend(); ++it) {
          s->reqs[*it].alone = true;
          s->queue.push_front(*it);
        }
        s->stats.split_batches++;
      } else {
        for (uint64_t t : sl.tickets) finish(s, t, status);
      }
      sl.tickets.clear();
      sl.busy = false;
      progressed = true;
    }
    if (progressed) s->done_cv.notify_all();
    // ---- admission -----------------------------------------------------------------
    s->submitted.store(false);
    for (Slot& sl : s->slots) {
      if (sl.busy || s->queue.empty()) continue;
      views.clear();
      std::vector<uint64_t> batch;
      int batch_k = 0;
      while (!s->queue.empty() && (int)batch.size() < s->cfg.max_batch_views) {
        const uint64_t t = s->queue.front();
        Req& r = s->reqs[t];
        if (r.alone && !batch.empty()) break;
        if (!batch.empty() && request_k(s, r.view) != batch_k) break;   // one capacity per batch
        batch_k = request_k(s, r.view);
        views.push_back(r.view);
        size_t need = 0;
        const lr_status st = lr_workspace_size_batch(s->inner, (int32_t)views.size(), views.data(), &need);
        if (st != LR_OK || need > sl.bytes) {
          views.pop_back();
          if (batch.empty()) {   // does not fit even alone
            s->queue.pop_front();
            finish(s, t, st != LR_OK ? st : LR_ERR_OOM);
            progressed = true;
            continue;
          }
          break;
        }
        batch.push_back(t);
        s->queue.pop_front();
        if (r.alone) break;
      }
      if (batch.empty()) continue;
      bool others_busy = false;
      for (const Slot& o : s->slots) others_busy |= o.busy;
      lr_internal_set_pdl(s->inner, others_busy ? 0 : 1);
      const lr_status st = lr_render_batch(s->inner, (int32_t)views.size(), views.data(), sl.ws, sl.bytes,
                                           reinterpret_cast<lr_stream>(sl.stream));
      lr_internal_set_pdl(s->inner, -1);
      const uint64_t t0 = now_ns();
      for (uint64_t t : batch) {
        Req& r = s->reqs[t];
        r.t_launch = t0;
        r.batch_views = (int)batch.size();
      }
      if (st != LR_OK) {
        for (uint64_t t : batch) finish(s, t, st);
        progressed = true;
        continue;
      }
      // the status word travels back on the batch's stream, ahead of its completion event
      if (cudaMemcpyAsync(sl.host_ctrl, sl.ws, sizeof(Ctrl), cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
          cudaEventRecord(sl.done, sl.stream) != cudaSuccess) {
        cudaStreamSynchronize(sl.stream);
        for (uint64_t t : batch) finish(s, t, LR_ERR_CUDA);
        progressed = true;
        continue;
      }
      sl.tickets = batch;
      sl.busy = true;
      s->stats.batches++;
      s->stats.batched_views += (int64_t)batch.size();
      progressed = true;
    }
    if (progressed) s->done_cv.notify_all();
    bool any_busy = false;
    for (const Slot& sl : s->slots) any_busy |= sl.busy;
    if (s->stopping && s->queue.empty() && !any_busy) break;
    if (any_busy) {
      // spin on the running batches' events for up to one poll interval, or until a new
      // request arrives (only this thread changes the slots, so they are read unlocked)
      lk.unlock();
      const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(s->cfg.poll_interval_us);
      for (;;) {
        bool ready = false;
        for (Slot& sl : s->slots) ready |= sl.busy && cudaEventQuery(sl.done) != cudaErrorNotReady;
        if (ready || s->submitted.load() || std::chrono::steady_clock::now() >= until) break;
        std::this_thread::yield();
      }
      lk.lock();
    } else if (s->queue.empty() && !s->stopping) {
      // idle: spin for a while on the submission flag (a new request is then seen within
      // microseconds), then sleep until a submission or stop wakes the thread
      if (s->cfg.idle_spin_us > 0) {
        lk.unlock();
        const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(s->cfg.idle_spin_us);
        while (!s->submitted.load() && std::chrono::steady_clock::now() < until) std::this_thread::yield();
        lk.lock();
      }
      if (s->queue.empty() && !s->stopping) s->wake.wait(lk);
    }
  }
}

static void destroy_server(lr_server* s) {
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.ws) cudaFree(sl.ws);
    if (sl.host_ctrl) cudaFreeHost(sl.host_ctrl);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (s->inner) lr_destroy(s->inner);
  delete s;
}

extern "C" lr_status lr_server_start(lr_ctx* ctx, const lr_server_config* config) {
  if (!ctx) return LR_ERR_INVALID_ARG;
  lr_server** slot = lr_internal_server_slot(ctx);
  if (*slot) return LR_ERR_INVALID_ARG;
  lr_server* s = new (std::nothrow) lr_server();
  if (!s) return LR_ERR_OOM;
  memset(&s->cfg, 0, sizeof(s->cfg));
  if (config) s->cfg = *config;
  if (s->cfg.num_slots <= 0) s->cfg.num_slots = 2;
  if (s->cfg.max_batch_views <= 0) s->cfg.max_batch_views = 16;
  if (s->cfg.slot_workspace_bytes <= 0) s->cfg.slot_workspace_bytes = (int64_t)512 << 20;
  if (s->cfg.poll_interval_us <= 0) s->cfg.poll_interval_us = 20;
  if (s->cfg.idle_spin_us == 0) s->cfg.idle_spin_us = 5000;
  memset(&s->stats, 0, sizeof(s->stats));
  lr_config inner_cfg = *lr_internal_config(ctx);
  inner_cfg.flags &= ~LR_FLAG_TIMING;
  inner_cfg.flags |= LR_FLAG_NO_PDL;   // batches render on several streams at once
  lr_status st = lr_create(&inner_cfg, &s->inner);
  if (st != LR_OK) {
    delete s;
    return st;
  }
  {
    const float* light = lr_internal_light(ctx);   // lit requests use the context's light
    lr_set_lighting(s->inner, light, light[3]);
  }
  s->slots.resize(s->cfg.num_slots);
  for (Slot& sl : s->slots) {
    sl.bytes = (size_t)s->cfg.slot_workspace_bytes;
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&sl.ws, sl.bytes);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&sl.host_ctrl), sizeof(Ctrl));
    if (e != cudaSuccess) {
      destroy_server(s);
      return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : LR_ERR_CUDA;
    }
  }
  s->th = std::thread(serve_loop, s);
  *slot = s;
  return LR_OK;
}

extern "C" lr_status lr_server_stop(lr_ctx* ctx) {
  if (!ctx) return LR_ERR_INVALID_ARG;
  lr_server** slot = lr_internal_server_slot(ctx);
  lr_server* s = *slot;
  if (!s) return LR_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->wake.notify_all();
  s->th.join();
  *slot = nullptr;
  destroy_server(s);
  return LR_OK;
}

extern "C" lr_status lr_submit(lr_ctx* ctx, const lr_view* view, uint64_t* ticket) {
  if (!ctx || !view || !ticket) return LR_ERR_INVALID_ARG;
  lr_server* s = *lr_internal_server_slot(ctx);
  if (!s) return LR_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return LR_ERR_INVALID_ARG;
    // reject a malformed request here, so that it cannot fail the batch it would join
    const lr_status chk = lr_internal_check_view(s->inner, view);
    if (chk != LR_OK) return chk;
    const uint64_t t = s->next_ticket++;
    Req r;
    r.view = *view;
    r.t_submit = now_ns();
    s->reqs.emplace(t, r);
    s->queue.push_back(t);
    s->stats.submitted++;
    *ticket = t;
    s->submitted.store(true);
  }
  s->wake.notify_all();
  return LR_OK;
}

extern "C" lr_status lr_poll_info(lr_ctx* ctx, uint64_t ticket, int32_t timeout_us, lr_status* result,
                                  lr_request_info* info) {
  if (!ctx || !result) return LR_ERR_INVALID_ARG;
  lr_server* s = *lr_internal_server_slot(ctx);
  if (!s) return LR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LR_ERR_INVALID_ARG;
  if (!it->second.done && timeout_us > 0) {
    s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] {
      auto j = s->reqs.find(ticket);
      return j == s->reqs.end() || j->second.done;
    });
    it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LR_ERR_INVALID_ARG;
  }
  if (!it->second.done) {
    *result = LR_PENDING;
    return timeout_us > 0 ? LR_ERR_TIMEOUT : LR_PENDING;
  }
  *result = (lr_status)it->second.status;
  if (info) {
    info->submit_ns = it->second.t_submit;
    info->launch_ns = it->second.t_launch;
    info->done_ns = it->second.t_done;
    info->batch_views = it->second.batch_views;
  }
  s->reqs.erase(it);
  return LR_OK;
}

extern "C" lr_status lr_poll(lr_ctx* ctx, uint64_t ticket, int32_t timeout_us, lr_status* result) {
  return lr_poll_info(ctx, ticket, timeout_us, result, nullptr);
}

extern "C" lr_status lr_server_get_stats(lr_ctx* ctx, lr_server_stats* out) {
  if (!ctx || !out) return LR_ERR_INVALID_ARG;
  lr_server* s = *lr_internal_server_slot(ctx);
  if (!s) return LR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queued = (int64_t)s->queue.size();
  return LR_OK;
}

extern "C" uint64_t lr_now_ns(void) { return now_ns(); }
