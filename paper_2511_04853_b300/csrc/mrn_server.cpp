// Continuous-batching conversion server.
//
// Clients submit transfer-and-convert requests (at least one side on the
// host); a worker thread admits them in arrival order whenever a slot is
// free and the request's device footprint fits in the remaining HBM budget
// (a request may pass a blocked head of the queue while the head is young),
// runs each admitted request on its slot's own copy/compute streams, so that
// requests overlap on the device, and completes them as their events fire.
// Latency is measured from submission (arrival) to the worker observing
// completion.
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
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mrn_transfer.h"

namespace mrn {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device allocation (offsets, 256-B aligned).
class Arena {
 public:
  int init(uint64_t bytes) {
    bytes_ = bytes;
    if (bytes == 0) return MRN_OK;
    if (cudaMalloc(&base_, bytes) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return MRN_ENOMEM;
    }
    free_[0] = bytes;
    return MRN_OK;
  }
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  // Returns the offset, or ~0 when no free range is large enough.
  uint64_t alloc(uint64_t n) {
    n = align_up(std::max<uint64_t>(n, 1), 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const uint64_t off = it->first, rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        used_ += n;
        return off;
      }
    }
    return ~0ull;
  }
  void release(uint64_t off, uint64_t n) {
    n = align_up(std::max<uint64_t>(n, 1), 256);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* base() const { return static_cast<char*>(base_); }
  uint64_t used() const { return used_; }
  uint64_t bytes() const { return bytes_; }

 private:
  void* base_ = nullptr;
  uint64_t bytes_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

struct Request {
  uint64_t ticket = 0;
  mrn_view src{}, dst{};
  std::vector<void*> cols[4];
  uint64_t footprint = 0, staging = 0;
  uint64_t bytes_in = 0, bytes_out = 0;
  Clock::time_point arrival;
  int status = MRN_EBUSY;
  bool done = false;
  double latency_ms = 0;  // arrival -> completion, set when done
  uint64_t arena_off = ~0ull;
};

struct Slot {
  std::unique_ptr<TransferEngine> engine;
  std::unique_ptr<TransferEngine> engine2;  // second leg of host -> host
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Request* active = nullptr;
  int rc = MRN_OK;
};

bool is_host(const mrn_view& v) { return v.mem == MRN_MEM_HOST || v.mem == MRN_MEM_HOST_PINNED; }

void own(const mrn_view& v, std::vector<void*>* c0, std::vector<void*>* c1, mrn_view* out) {
  *out = v;
  const mrn_schema* s = v.schema;
  if (v.columns) {
    c0->assign(v.columns, v.columns + s->cols.size());
    out->columns = c0->data();
  }
  if (v.child_columns && s->has_jagged) {
    c1->assign(v.child_columns, v.child_columns + s->child->cols.size());
    out->child_columns = c1->data();
  }
}

uint64_t parts_bytes(const mrn_view& v) {
  uint64_t b = 0;
  for (const auto& p : view_parts(v)) b += p.bytes;
  return b;
}

}  // namespace
}  // namespace mrn

using namespace mrn;

struct mrn_server {
  mrn_server_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
  std::vector<Slot> slots;
  Arena arena;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  // statistics
  uint64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, failed = 0;
  uint64_t bytes_in = 0, bytes_out = 0, peak = 0;
  std::vector<double> lat_ms;
  bool have_first = false;
  Clock::time_point first_arrival, last_done;

  uint64_t chunk() const { return opts.chunk_bytes ? opts.chunk_bytes : (4ull << 20); }

  // Device bytes a request holds while admitted: transfer staging, plus the
  // device copy of the destination for a host -> host request.
  uint64_t footprint(const mrn_view& src, const mrn_view& dst, uint64_t* staging) const {
    if (is_host(src) && is_host(dst)) {
      mrn_view dv = dst, tmp;
      dv.mem = MRN_MEM_DEVICE;
      dv.device = device;
      std::vector<void*> a, b;
      const uint64_t inter = staged_view(dv, nullptr, &tmp, a, b);
      *staging = TransferEngine::staging_bytes(src, dv, chunk(), 4);
      return align_up(*staging, 256) + inter;
    }
    *staging = TransferEngine::staging_bytes(src, dst, chunk(), 4);
    return *staging;
  }

  // Enqueues the device work of an admitted request on its slot.
  int start(Slot& sl, Request* r) {
    char* at = r->footprint ? arena.base() + r->arena_off : nullptr;
    int rc;
    if (is_host(r->src) && is_host(r->dst)) {
      mrn_view dv = r->dst, inter;
      dv.mem = MRN_MEM_DEVICE;
      dv.device = device;
      std::vector<void*> a, b;
      staged_view(dv, at + align_up(r->staging, 256), &inter, a, b);
      rc = sl.engine->run(r->src, inter, chunk(), 4, sl.stream, at, r->staging);
      if (!rc) rc = sl.engine2->run(inter, r->dst, chunk(), 4, sl.stream, nullptr, 0);
    } else {
      rc = sl.engine->run(r->src, r->dst, chunk(), 4, sl.stream, at, r->staging);
    }
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess && !rc) rc = MRN_ECUDA;
    return rc;
  }

  void finish(Slot& sl, int rc) {
    Request* r = sl.active;
    sl.active = nullptr;
    if (r->footprint) arena.release(r->arena_off, r->footprint);
    r->status = rc;
    r->done = true;
    const auto now = Clock::now();
    last_done = now;
    if (rc == MRN_OK) {
      completed++;
      bytes_in += r->bytes_in;
      bytes_out += r->bytes_out;
    } else {
      failed++;
    }
    r->latency_ms = std::chrono::duration<double, std::milli>(now - r->arrival).count();
    lat_ms.push_back(r->latency_ms);
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      bool progress = false;
      for (auto& sl : slots) {
        if (!sl.active) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        finish(sl, q == cudaSuccess ? sl.rc : MRN_ECUDA);
        progress = true;
      }
      if (progress) cv_done.notify_all();
      // admissions in arrival order; a later request may pass a blocked head
      // while the head has waited less than 50 ms
      const auto now = Clock::now();
      for (auto it = queue.begin(); it != queue.end();) {
        Slot* free_slot = nullptr;
        for (auto& sl : slots)
          if (!sl.active) {
            free_slot = &sl;
            break;
          }
        if (!free_slot) break;
        Request* r = *it;
        uint64_t off = 0;
        if (r->footprint) off = arena.alloc(r->footprint);
        if (off == ~0ull) {
          if (it == queue.begin() && now - r->arrival > std::chrono::milliseconds(50)) break;
          ++it;
          continue;
        }
        r->arena_off = off;
        it = queue.erase(it);
        admitted++;
        peak = std::max(peak, arena.used());
        free_slot->active = r;
        free_slot->rc = start(*free_slot, r);
        progress = true;
      }
      const bool busy = std::any_of(slots.begin(), slots.end(), [](const Slot& s) { return s.active; });
      if (stop && !busy && queue.empty()) break;
      if (!progress) {
        if (busy || !queue.empty()) {
          lk.unlock();
          std::this_thread::sleep_for(std::chrono::microseconds(10));
          lk.lock();
        } else {
          cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
      }
    }
  }
};

extern "C" {

int mrn_server_create(const mrn_server_opts* opts, mrn_server** out) {
  if (!opts || !out) return MRN_EINVAL;
  *out = nullptr;
  auto* sv = new (std::nothrow) mrn_server();
  if (!sv) return MRN_ENOMEM;
  sv->opts = *opts;
  if (sv->opts.max_slots <= 0) sv->opts.max_slots = 8;
  sv->opts.max_slots = std::min(sv->opts.max_slots, 64);
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return MRN_ECUDA;
  }
  int rc = sv->arena.init(opts->hbm_budget_bytes);
  sv->slots.resize(sv->opts.max_slots);
  for (auto& sl : sv->slots) {
    if (rc) break;
    sl.engine = std::make_unique<TransferEngine>();
    sl.engine2 = std::make_unique<TransferEngine>();
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
      rc = MRN_ECUDA;
  }
  if (rc) {
    for (auto& sl : sv->slots) {
      if (sl.done) cudaEventDestroy(sl.done);
      if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete sv;
    return rc;
  }
  sv->worker = std::thread([sv] { sv->loop(); });
  *out = sv;
  return MRN_OK;
}

int mrn_server_submit(mrn_server* sv, const mrn_view* src, const mrn_view* dst, uint64_t* ticket) {
  if (!sv || !src || !dst || !ticket) return MRN_EINVAL;
  bool jag = false;
  int rc = validate_pair(src, dst, false, &jag);
  if (rc) return rc;
  if (!is_host(*src) && !is_host(*dst)) return MRN_EINVAL;
  if (src->schema->interleaved || is_nested(src->schema)) return MRN_EUNSUPPORTED;  // via the transfer engine
  for (const mrn_view* v : {src, dst})
    if (v->mem == MRN_MEM_DEVICE && v->device != sv->device) return MRN_EINVAL;
  if (jag && dst->layout.kind == MRN_AOS && dst->n_children < src->n_children) return MRN_ESIZE;
  auto r = std::make_unique<Request>();
  r->arrival = Clock::now();
  own(*src, &r->cols[0], &r->cols[1], &r->src);
  own(*dst, &r->cols[2], &r->cols[3], &r->dst);
  r->footprint = sv->footprint(r->src, r->dst, &r->staging);
  r->bytes_in = parts_bytes(r->src);
  r->bytes_out = parts_bytes(r->dst);
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->submitted++;
  if (!sv->have_first) {
    sv->have_first = true;
    sv->first_arrival = r->arrival;
  }
  if (r->footprint > sv->arena.bytes()) {
    sv->rejected++;
    return MRN_ENOMEM;
  }
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  sv->queue.push_back(r.get());
  sv->requests[r->ticket] = std::move(r);
  sv->cv_work.notify_one();
  return MRN_OK;
}

int mrn_server_poll(mrn_server* sv, uint64_t ticket, int* done, int* status) {
  if (!sv || !done || !status) return MRN_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end()) return MRN_ENOTFOUND;
  *done = it->second->done ? 1 : 0;
  *status = it->second->done ? it->second->status : MRN_EBUSY;
  if (it->second->done) sv->requests.erase(it);
  return MRN_OK;
}

int mrn_server_wait(mrn_server* sv, uint64_t ticket, uint64_t timeout_ns, int* status) {
  if (!sv || !status) return MRN_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end()) return MRN_ENOTFOUND;
  Request* r = it->second.get();
  if (!sv->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), [r] { return r->done; }))
    return MRN_ETIMEOUT;
  *status = r->status;
  sv->requests.erase(ticket);
  return MRN_OK;
}

int mrn_server_wait_latency(mrn_server* sv, uint64_t ticket, uint64_t timeout_ns, int* status,
                            double* latency_ms) {
  if (!sv || !status || !latency_ms) return MRN_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end()) return MRN_ENOTFOUND;
  Request* r = it->second.get();
  if (!sv->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), [r] { return r->done; }))
    return MRN_ETIMEOUT;
  *status = r->status;
  *latency_ms = r->latency_ms;
  sv->requests.erase(ticket);
  return MRN_OK;
}

int mrn_server_stats_get(mrn_server* sv, mrn_server_stats* out) {
  if (!sv || !out) return MRN_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = sv->submitted;
  out->admitted = sv->admitted;
  out->completed = sv->completed;
  out->rejected = sv->rejected;
  out->failed = sv->failed;
  out->bytes_in = sv->bytes_in;
  out->bytes_out = sv->bytes_out;
  out->peak_device_bytes = sv->peak;
  if (!sv->lat_ms.empty()) {
    std::vector<double> v = sv->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      const double k = std::ceil(p * (double)v.size()) - 1.0;
      return v[(size_t)std::min<double>((double)v.size() - 1, std::max(0.0, k))];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
    out->busy_s = std::chrono::duration<double>(sv->last_done - sv->first_arrival).count();
  }
  return MRN_OK;
}

void mrn_server_destroy(mrn_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    sl.engine.reset();
    sl.engine2.reset();
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete sv;
}

}  // extern "C"
