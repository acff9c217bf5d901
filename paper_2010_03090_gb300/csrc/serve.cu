// Continuous-batching validation server (host runtime around segments.cu).
//
// Clients submit device-resident buffers from any thread.  A request is
// admitted when the bytes of admitted, unfinished requests stay within the
// memory budget (otherwise it waits, in arrival order, until completions
// free room).  A worker thread groups admitted requests into batches and
// launches each batch as one segments kernel on one of several streams, so
// new batches are formed and launched while earlier ones still run on the
// GPU.  A batch is launched when its oldest request has waited window_min
// and no batch is on the GPU, when it has waited window_max, or when it is
// full (max_batch requests).  The worker polls the batches' events, publishes
// each request's flag and latency (arrival to result) and releases its bytes.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#ifdef __linux__
#include <sys/prctl.h>
#endif

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"
#include "tune.h"
#include "utf8gpu.h"


using namespace utf8gpu;

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket;
  const uint8_t* data;
  uint64_t len;
  int64_t arrival_ns;
};

struct Result {
  uint8_t done = 0;
  uint8_t valid = 0;
  int64_t latency_ns = 0;
};

// A batch slot.  The batch's descriptors (n SegmentDesc, then the n + 1
// entries of the tile prefix) go to the device in one copy; the flags live in
// pinned host memory mapped into the device, set to 1 by the host before the
// launch and cleared by the kernel, so no copy brings them back.
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint8_t* h_desc = nullptr;    // pinned
  uint8_t* d_desc = nullptr;    // device
  uint8_t* h_flags = nullptr;   // pinned, mapped
  uint8_t* dm_flags = nullptr;  // its device address
  std::vector<Request> reqs;
  bool busy = false;
};

size_t desc_bytes(size_t n) { return n * sizeof(SegmentDesc) + (n + 1) * sizeof(int64_t); }

}  // namespace

struct utf8_server {
  utf8_server_config cfg{};
  int device = 0;
  int sm_count = 0;
  LaunchCfg launch;
  std::mutex mu;
  std::condition_variable cv_work;  // new requests / stop
  std::condition_variable cv_done;  // results published
  std::deque<Request> waiting;      // over budget, not yet admitted
  std::deque<Request> pending;      // admitted, not yet launched
  uint64_t admitted_bytes = 0;      // admitted and not finished
  std::vector<Result> results;      // by ticket
  uint64_t next_ticket = 0;
  std::vector<Slot> slots;
  std::thread worker;
  bool stop = false;
  utf8_server_stats stats{};
  int error = UTF8_OK;  // sticky CUDA failure of the worker
};

namespace {

void admit_waiting(utf8_server* s) {  // caller holds mu
  while (!s->waiting.empty() &&
         s->admitted_bytes + s->waiting.front().len <= s->cfg.budget_bytes) {
    s->admitted_bytes += s->waiting.front().len;
    s->pending.push_back(s->waiting.front());
    s->waiting.pop_front();
  }
  if (s->admitted_bytes > s->stats.max_admitted_bytes) s->stats.max_admitted_bytes = s->admitted_bytes;
}

cudaError_t launch_slot(utf8_server* s, Slot& slot) {
  const int64_t n = (int64_t)slot.reqs.size();
  SegmentDesc* h_segs = reinterpret_cast<SegmentDesc*>(slot.h_desc);
  int64_t* h_prefix = reinterpret_cast<int64_t*>(slot.h_desc + n * sizeof(SegmentDesc));
  int64_t tiles = 0;
  for (int64_t k = 0; k < n; ++k) {
    h_segs[k].data = slot.reqs[k].data;
    h_segs[k].len = slot.reqs[k].len;
    h_prefix[k] = tiles;
    tiles += (int64_t)segment_tiles(slot.reqs[k].data, slot.reqs[k].len, s->launch);
    slot.h_flags[k] = 1;
  }
  h_prefix[n] = tiles;
  std::atomic_thread_fence(std::memory_order_release);
  cudaError_t e = cudaMemcpyAsync(slot.d_desc, slot.h_desc, desc_bytes((size_t)n),
                                  cudaMemcpyHostToDevice, slot.stream);
  if (e == cudaSuccess)
    e = launch_segments(reinterpret_cast<const SegmentDesc*>(slot.d_desc),
                        reinterpret_cast<const int64_t*>(slot.d_desc + n * sizeof(SegmentDesc)), n,
                        (uint64_t)tiles, slot.dm_flags, s->launch, s->sm_count, slot.stream);
  if (e == cudaSuccess) e = cudaEventRecord(slot.done, slot.stream);
  return e;
}

void worker_main(utf8_server* s) {
  cudaSetDevice(s->device);
#ifdef __linux__
  // The batching window and the completion polls are microsecond waits; the
  // default timer slack of a thread (50 us) would stretch every one of them.
  prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
  const int64_t wmin = (int64_t)s->cfg.window_min_us * 1000;
  const int64_t wmax = (int64_t)s->cfg.window_max_us * 1000;
  for (;;) {
    bool progress = false;
    // completions
    for (Slot& slot : s->slots) {
      if (!slot.busy) continue;
      const cudaError_t q = cudaEventQuery(slot.done);
      if (q == cudaErrorNotReady) continue;
      const int64_t t = now_ns();
      std::lock_guard<std::mutex> lock(s->mu);
      if (q != cudaSuccess) s->error = UTF8_ERR_CUDA;
      for (size_t k = 0; k < slot.reqs.size(); ++k) {
        const Request& r = slot.reqs[k];
        Result& res = s->results[r.ticket];
        res.valid = q == cudaSuccess ? slot.h_flags[k] : 0;
        res.latency_ns = t - r.arrival_ns;
        res.done = q == cudaSuccess ? 1 : 2;
        s->admitted_bytes -= r.len;
        s->stats.completed += 1;
        s->stats.bytes += r.len;
      }
      slot.reqs.clear();
      slot.busy = false;
      admit_waiting(s);
      s->cv_done.notify_all();
      progress = true;
    }
    // dispatch
    Slot* free_slot = nullptr;
    bool gpu_idle = true;
    for (Slot& slot : s->slots) {
      if (slot.busy) gpu_idle = false;
      else if (!free_slot) free_slot = &slot;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    if (free_slot && !s->pending.empty()) {
      const int64_t age = now_ns() - s->pending.front().arrival_ns;
      const bool go = s->stop || (age >= wmin && gpu_idle) || age >= wmax ||
                      s->pending.size() >= s->cfg.max_batch;
      if (go) {
        while (!s->pending.empty() && free_slot->reqs.size() < s->cfg.max_batch) {
          free_slot->reqs.push_back(s->pending.front());
          s->pending.pop_front();
        }
        s->stats.batches += 1;
        if (free_slot->reqs.size() > s->stats.max_batch_seen)
          s->stats.max_batch_seen = free_slot->reqs.size();
        lock.unlock();
        const cudaError_t e = launch_slot(s, *free_slot);
        if (e == cudaSuccess) {
          free_slot->busy = true;
        } else {  // the batch's requests fail; their bytes are released
          cudaGetLastError();
          std::lock_guard<std::mutex> relock(s->mu);
          s->error = UTF8_ERR_CUDA;
          for (const Request& r : free_slot->reqs) {
            s->results[r.ticket].done = 2;
            s->admitted_bytes -= r.len;
          }
          free_slot->reqs.clear();
          admit_waiting(s);
          s->cv_done.notify_all();
        }
        progress = true;
        lock.lock();
      }
    }
    const bool busy_any = !gpu_idle || progress;
    if (s->stop && s->pending.empty() && s->waiting.empty()) {
      bool any = false;
      for (Slot& slot : s->slots) any = any || slot.busy;
      if (!any) return;
    }
    if (progress) continue;
    if (busy_any) {  // batches on the GPU: poll again shortly
      lock.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(1));
    } else if (s->pending.empty()) {
      s->cv_work.wait_for(lock, std::chrono::milliseconds(5));
    } else {  // wait until the oldest request is old enough
      const int64_t age = now_ns() - s->pending.front().arrival_ns;
      const int64_t left = (age < wmin ? wmin - age : 0) / 1000 + 1;
      s->cv_work.wait_for(lock, std::chrono::microseconds(left));
    }
  }
}

void destroy_slots(utf8_server* s) {
  for (Slot& slot : s->slots) {
    if (slot.done) cudaEventDestroy(slot.done);
    if (slot.stream) cudaStreamDestroy(slot.stream);
    cudaFreeHost(slot.h_desc);
    cudaFreeHost(slot.h_flags);
    cudaFree(slot.d_desc);
  }
  s->slots.clear();
}

}  // namespace

extern "C" {

void utf8_server_default_config(utf8_server_config* cfg) {
  if (!cfg) return;
  cfg->budget_bytes = 8ull << 30;
  cfg->window_min_us = 50;
  cfg->window_max_us = 500;
  cfg->max_batch = 4096;
  cfg->streams = 4;
}

utf8_server* utf8_server_create(const utf8_server_config* cfg) {
  utf8_server_config c;
  utf8_server_default_config(&c);
  if (cfg) c = *cfg;
  if (c.budget_bytes == 0 || c.max_batch == 0 || c.streams == 0 || c.streams > 64 ||
      c.window_max_us < c.window_min_us) {
    set_thread_status(UTF8_ERR_INVALID_ARG);
    return nullptr;
  }
  utf8_server* s = new utf8_server();
  s->cfg = c;
  cudaError_t e = cudaGetDevice(&s->device);
  cudaDeviceProp prop;
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, s->device);
  if (e == cudaSuccess) {
    s->sm_count = prop.multiProcessorCount;
    s->launch = tuned_config(prop.name, prop.multiProcessorCount);
    clamp_to_occupancy(s->launch);
  }
  s->slots.resize(c.streams);
  for (Slot& slot : s->slots) {
    if (e != cudaSuccess) break;
    const size_t n = c.max_batch;
    e = cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc(&slot.h_desc, desc_bytes(n), 0);
    if (e == cudaSuccess) e = cudaMalloc(&slot.d_desc, desc_bytes(n));
    if (e == cudaSuccess) e = cudaHostAlloc(&slot.h_flags, n, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&slot.dm_flags),
                                                       slot.h_flags, 0);
    slot.reqs.reserve(n);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_slots(s);
    delete s;
    set_thread_status(UTF8_ERR_CUDA);
    return nullptr;
  }
  s->worker = std::thread(worker_main, s);
  set_thread_status(UTF8_OK);
  return s;
}

}  // extern "C"

namespace {

// Submits with an explicit arrival time (the clock of now_ns).
int submit_at(utf8_server* s, const uint8_t* data, size_t len, int64_t t, uint64_t* ticket) {
  if (!s || !ticket || (data == nullptr && len > 0)) return set_thread_status(UTF8_ERR_INVALID_ARG);
  if (len > s->cfg.budget_bytes) return set_thread_status(UTF8_ERR_BUDGET);
  if (len > 0 && !is_device_memory(data)) return set_thread_status(UTF8_ERR_INVALID_ARG);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return set_thread_status(UTF8_ERR_INVALID_ARG);
    Request r{s->next_ticket++, data, len, t};
    s->results.emplace_back();
    s->stats.submitted += 1;
    s->waiting.push_back(r);
    admit_waiting(s);
    *ticket = r.ticket;
  }
  s->cv_work.notify_one();
  return set_thread_status(UTF8_OK);
}

}  // namespace

extern "C" {

int utf8_server_submit(utf8_server* s, const uint8_t* data, size_t len, uint64_t* ticket) {
  return submit_at(s, data, len, now_ns(), ticket);
}

int utf8_server_result(utf8_server* s, uint64_t ticket, int64_t timeout_us, int* valid,
                       int64_t* latency_ns) {
  if (!s) return set_thread_status(UTF8_ERR_INVALID_ARG);
  std::unique_lock<std::mutex> lock(s->mu);
  if (ticket >= s->results.size()) return set_thread_status(UTF8_ERR_INVALID_ARG);
  const auto ready = [&] { return s->results[ticket].done != 0; };
  if (timeout_us < 0) {
    s->cv_done.wait(lock, ready);
  } else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready)) {
    return set_thread_status(UTF8_ERR_TIMEOUT);
  }
  const Result& r = s->results[ticket];
  if (r.done == 2) return set_thread_status(UTF8_ERR_CUDA);
  if (valid) *valid = r.valid;
  if (latency_ns) *latency_ns = r.latency_ns;
  return set_thread_status(UTF8_OK);
}

int utf8_server_replay(utf8_server* s, const uint8_t* const* datas, const size_t* lens,
                       const int64_t* arrival_ns, int64_t count, uint8_t* out_valid,
                       int64_t* out_latency_ns) {
  if (!s || count < 0 || (count > 0 && (!datas || !lens || !arrival_ns)))
    return set_thread_status(UTF8_ERR_INVALID_ARG);
  std::vector<uint64_t> tickets((size_t)count);
  const int64_t start = now_ns();
  for (int64_t i = 0; i < count; ++i) {
    const int64_t due = start + arrival_ns[i];
    while (now_ns() < due) {
    }
    // latency counts from the scheduled arrival, so a late submit is not hidden
    const int st = submit_at(s, datas[i], lens[i], due, &tickets[i]);
    if (st != UTF8_OK) return st;
  }
  for (int64_t i = 0; i < count; ++i) {
    int v = 0;
    int64_t lat = 0;
    const int st = utf8_server_result(s, tickets[i], -1, &v, &lat);
    if (st != UTF8_OK) return st;
    if (out_valid) out_valid[i] = (uint8_t)v;
    if (out_latency_ns) out_latency_ns[i] = lat;
  }
  return set_thread_status(UTF8_OK);
}

int utf8_server_stats_get(utf8_server* s, utf8_server_stats* out) {
  if (!s || !out) return set_thread_status(UTF8_ERR_INVALID_ARG);
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  return set_thread_status(s->error);
}

void utf8_server_destroy(utf8_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  destroy_slots(s);
  delete s;
}

}  // extern "C"
