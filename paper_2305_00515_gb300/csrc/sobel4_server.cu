// sobel4_server.cu — a continuous-batching request server around the batched
// kernel.  Requests (host images of any size) are admitted first-in
// first-out while a device-memory arena has room for their input (and their
// output, where it must be staged), uploaded on a copy stream, packed into
// one persistent batched launch per scheduling step (at most kMaxInFlight
// batches on the GPU at once, so requests that arrive while a batch runs join
// the next one; a batch of up to three runs as single-image launches).  A result
// buffer in mapped page-locked host memory is the kernel's own output: the
// kernel's stores cross the host link directly, with no device-to-host copy
// (whose rate on a Grace host drops after idle gaps: 4K downloads measured
// 184 us median, up to 2 ms at the 99th percentile with 2.5 ms between
// requests, against 185 / 218 us for the kernel's own stores).  Any other
// result buffer gets an arena block and a download on a third stream.  An
// event after each request's last operation marks it; a completion thread
// waits on those events in order, so a small request never waits for a large
// one's download and no CUDA host function is involved.  Two comparison
// modes: every request its own single-image launch on the same streams
// (plain = 1), or one sobel4_run per request in arrival order on ONE stream,
// upload, kernel and download back to back (plain = 2).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sobel4.h"
#include "sobel4_launch.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxInFlight = 2;
constexpr size_t kSinglesUpTo = 3;  // larger batches take one persistent batched launch
constexpr size_t kAlign = 256;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
size_t elem_bytes(int fmt) {
  return fmt == SOBEL4_OUT_F32 ? 4 : ((fmt == SOBEL4_OUT_U8 || fmt == SOBEL4_OUT_EDGE8) ? 1 : 2);
}

// First-fit allocator over one device buffer; offsets only, no device calls.
class Arena {
 public:
  void reset(size_t bytes) {
    free_.clear();
    free_[0] = bytes;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = round_up(bytes, kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      if (used_ > peak_) peak_ = used_;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(bytes, kAlign);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

enum State { kQueued, kAdmitted, kInFlight, kDone, kFailed };

struct Request {
  const uint8_t *h_src = nullptr;
  size_t sp = 0;
  void *h_dst = nullptr;
  size_t dp = 0;
  int32_t H = 0, W = 0;
  size_t in_bytes = 0, out_bytes = 0, d_sp = 0, d_dp = 0, off = 0;
  bool direct = false;  // the kernel writes h_dst itself (mapped page-locked memory)
  // arena bytes: the input block, then (staged results only) the output
  // block, each 256-byte aligned
  size_t arena_bytes() const {
    return round_up(in_bytes, kAlign) + (direct ? 0 : round_up(out_bytes, kAlign));
  }
  uint8_t *d_in = nullptr, *d_out = nullptr;
  Clock::time_point t_submit, t_done;
  State state = kQueued;
};

struct Batch;

// A request whose last operation has been enqueued: the completion thread
// waits on `ev` (recorded after it) and then retires member `idx` of `b`.
struct Pending {
  cudaEvent_t ev;
  Batch *b;
  size_t idx;
};

}  // namespace

struct sobel4_server_ctx {
  sobel4_handle h = nullptr;
  int device = 0;
  sobel4_server_options opt{};
  uint8_t *arena_mem = nullptr;
  Arena arena;
  cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
  std::thread sched, completer;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_cq;
  bool stop = false;       // no more submissions; the scheduler drains and exits
  bool sched_done = false;  // the scheduler has exited; the completer drains and exits
  bool failed = false;
  std::deque<uint64_t> incoming, admitted;
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<Pending> cq;  // in the order of the GPU work they follow
  int in_flight = 0;
  uint64_t next_ticket = 1;
  std::vector<cudaEvent_t> event_pool;
  sobel4_server_counters stats{};
};

namespace {

// One request of a batch.
struct Member {
  uint64_t ticket;
  cudaEvent_t ev;  // recorded after the request's last operation
};

struct Batch {
  std::vector<Member> members;
  int remaining = 0;  // members not yet retired
  cudaEvent_t done;   // orders upload -> kernel -> downloads across the streams
};

cudaEvent_t take_event(sobel4_server_ctx *s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return e;
}

// With the lock held: a request's result is in host memory.  The batch
// leaves the GPU with its last member; returns the batch to delete, if any.
Batch *retire(sobel4_server_ctx *s, Batch *b, size_t idx) {
  auto it = s->reqs.find(b->members[idx].ticket);
  if (it != s->reqs.end()) {
    Request &r = it->second;
    r.t_done = Clock::now();
    if (r.state != kFailed) {
      r.state = kDone;
      s->stats.completed += 1;
    }
    s->arena.release(r.off, r.arena_bytes());
  }
  s->event_pool.push_back(b->members[idx].ev);
  if (--b->remaining > 0) return nullptr;
  s->in_flight -= 1;
  s->event_pool.push_back(b->done);
  return b;
}

void fail_all(sobel4_server_ctx *s) {
  // called with the lock held
  s->failed = true;
  for (auto &kv : s->reqs)
    if (kv.second.state != kDone) kv.second.state = kFailed;
  s->incoming.clear();
  s->admitted.clear();
  s->cv_done.notify_all();
}

// Waits for each pending request's event in order: every request's last
// operation is on the download stream (the one stream in the one-stream
// mode), whose events complete in the order they were recorded.
void completer(sobel4_server_ctx *s) {
  sobel4::DeviceScope scope(s->device);
  for (;;) {
    Pending p;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_cq.wait(lock, [&] { return !s->cq.empty() || s->sched_done; });
      if (s->cq.empty()) break;
      p = s->cq.front();
    }
    const cudaError_t e = cudaEventSynchronize(p.ev);
    Batch *gone = nullptr;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->cq.pop_front();
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fail_all(s);
      }
      gone = retire(s, p.b, p.idx);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();
    delete gone;
  }
}

// One upload or one batch member, copied out of the request table so that
// CUDA calls run without the lock held.
struct Job {
  uint64_t ticket;
  const uint8_t *h_src;
  size_t sp;
  void *h_dst;
  size_t dp;
  int32_t H, W;
  uint8_t *d_in, *d_out;
  size_t d_sp, d_dp;
  bool direct;
};

Job job_of(uint64_t t, const Request &r) {
  return Job{t, r.h_src, r.sp, r.h_dst, r.dp, r.H, r.W, r.d_in, r.d_out, r.d_sp, r.d_dp,
             r.direct};
}

void scheduler(sobel4_server_ctx *s) {
  sobel4::DeviceScope scope(s->device);
  const int fmt = s->opt.format;
  const size_t planes = fmt == SOBEL4_OUT_S16X4 ? 4 : 1;
  const bool serial = s->opt.plain == 2;
  // the one-stream mode runs everything on the upload stream
  cudaStream_t up = s->up, comp = serial ? s->up : s->comp, down = serial ? s->up : s->down;
  std::vector<Job> uploads, members;
  bool more = false;  // one-stream mode: admitted requests still to issue
  for (;;) {
    uploads.clear();
    members.clear();
    Batch *b = nullptr;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] {
        return more || s->stop || s->failed || !s->incoming.empty() ||
               (!s->admitted.empty() && s->in_flight < kMaxInFlight);
      });
      more = false;
      if (s->failed) break;
      if (s->stop && s->incoming.empty() && s->admitted.empty()) break;
      // 1. Admission, first in first out, while the arena has room.
      while (!s->incoming.empty()) {
        const uint64_t t = s->incoming.front();
        Request &r = s->reqs[t];
        size_t off = 0;
        if (!s->arena.alloc(r.arena_bytes(), &off)) break;
        r.off = off;
        r.d_in = s->arena_mem + off;
        r.d_out = r.direct ? (uint8_t *)r.h_dst : r.d_in + round_up(r.in_bytes, kAlign);
        if (r.direct) r.d_dp = r.dp;
        r.state = kAdmitted;
        uploads.push_back(job_of(t, r));
        s->admitted.push_back(t);
        s->incoming.pop_front();
      }
      // 2. One launch of everything admitted (bounded by max_batch; in the
      //    one-stream mode one request per launch, as many as are admitted).
      if (!s->admitted.empty() && (serial || s->in_flight < kMaxInFlight)) {
        const int32_t cap = serial ? 1 : s->opt.max_batch;
        const size_t n = std::min<size_t>(s->admitted.size(), (size_t)cap);
        b = new (std::nothrow) Batch();
        bool ok = b != nullptr;
        if (ok) b->done = take_event(s);
        ok = ok && b->done;
        for (size_t i = 0; ok && i < n; ++i) {
          cudaEvent_t ev = take_event(s);
          ok = ev != nullptr;
          if (ok) b->members.push_back(Member{0, ev});
        }
        if (!ok) {
          if (b) {
            for (const Member &m : b->members) s->event_pool.push_back(m.ev);
            if (b->done) s->event_pool.push_back(b->done);
          }
          delete b;
          fail_all(s);
          break;
        }
        for (size_t i = 0; i < n; ++i) {
          const uint64_t t = s->admitted.front();
          s->admitted.pop_front();
          Request &r = s->reqs[t];
          r.state = kInFlight;
          b->members[i].ticket = t;
          members.push_back(job_of(t, r));
        }
        b->remaining = (int)n;
        s->in_flight += 1;
        s->stats.batches += 1;
        if ((uint64_t)n > s->stats.max_batch_seen) s->stats.max_batch_seen = n;
      }
      more = serial && !s->admitted.empty();
    }
    // CUDA work, unlocked.  Only this thread issues work on the three streams.
    cudaError_t e = cudaSuccess;
    // One-stream mode: each request's upload goes right before its kernel.
    for (size_t i = 0; i < uploads.size() && !serial; ++i) {
      const Job &j = uploads[i];
      e = cudaMemcpy2DAsync(j.d_in, j.d_sp, j.h_src, j.sp, (size_t)j.W, (size_t)j.H,
                            cudaMemcpyHostToDevice, up);
      if (e != cudaSuccess) break;
    }
    sobel4_status st = SOBEL4_OK;
    if (e == cudaSuccess && b && serial) {
      const Job &j = members[0];
      e = cudaMemcpy2DAsync(j.d_in, j.d_sp, j.h_src, j.sp, (size_t)j.W, (size_t)j.H,
                            cudaMemcpyHostToDevice, up);
      if (e == cudaSuccess)
        st = sobel4_run(s->h, j.d_in, j.d_sp, j.d_out, j.d_dp, j.H, j.W,
                        (sobel4_border)s->opt.border, (sobel4_format)fmt, up);
    } else if (e == cudaSuccess && b) {
      // The upload stream runs in order: its tail covers every upload of this batch.
      e = cudaEventRecord(b->done, up);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(comp, b->done, 0);
      if (e == cudaSuccess) {
        // Batches of up to kSinglesUpTo images run as single-image launches:
        // the batched path adds a descriptor upload and gains nothing there
        // (results into pinned host memory: two 1080p images 111 us batched
        // against 102 us as two launches; four mixed images level).
        if (s->opt.plain || members.size() <= kSinglesUpTo) {
          for (const Job &j : members) {
            st = sobel4_run(s->h, j.d_in, j.d_sp, j.d_out, j.d_dp, j.H, j.W,
                            (sobel4_border)s->opt.border, (sobel4_format)fmt, comp);
            if (st != SOBEL4_OK) break;
          }
        } else {
          std::vector<sobel4_image> imgs;
          imgs.reserve(members.size());
          for (const Job &j : members)
            imgs.push_back(sobel4_image{j.d_in, j.d_sp, j.d_out, j.d_dp, j.H, j.W});
          st = sobel4_run_batched(s->h, imgs.data(), (int32_t)imgs.size(),
                                  (sobel4_border)s->opt.border, (sobel4_format)fmt, comp);
          // The batched launch refuses results that overlap (two pending
          // requests sharing one result buffer, written in place): those run
          // one launch each rather than failing the server.
          if (st == SOBEL4_ERR_INVALID_ARG) {
            st = SOBEL4_OK;
            for (size_t i = 0; i < members.size() && st == SOBEL4_OK; ++i) {
              const Job &j = members[i];
              st = sobel4_run(s->h, j.d_in, j.d_sp, j.d_out, j.d_dp, j.H, j.W,
                              (sobel4_border)s->opt.border, (sobel4_format)fmt, comp);
            }
          }
        }
      }
      if (e == cudaSuccess && st == SOBEL4_OK) e = cudaEventRecord(b->done, comp);
      if (e == cudaSuccess && st == SOBEL4_OK) e = cudaStreamWaitEvent(down, b->done, 0);
    }
    // Each member's download (results the kernel did not write in place),
    // then its event, then its place in the completion queue.
    size_t enqueued = 0;
    for (size_t i = 0; b && i < members.size() && e == cudaSuccess && st == SOBEL4_OK; ++i) {
      const Job &j = members[i];
      if (!j.direct)
        e = cudaMemcpy2DAsync(j.h_dst, j.dp, j.d_out, j.d_dp, (size_t)j.W * elem_bytes(fmt),
                              (size_t)j.H * planes, cudaMemcpyDeviceToHost, down);
      if (e == cudaSuccess) e = cudaEventRecord(b->members[i].ev, down);
      if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->cq.push_back(Pending{b->members[i].ev, b, i});
        ++enqueued;
      }
      s->cv_cq.notify_one();
    }
    if (e != cudaSuccess || st != SOBEL4_OK) {
      if (e != cudaSuccess) (void)cudaGetLastError();
      Batch *gone = nullptr;
      {
        std::lock_guard<std::mutex> lock(s->mu);
        fail_all(s);
        // members that never reached the completion queue are retired here;
        // the batch goes with the last of its members
        for (size_t i = enqueued; b && i < members.size(); ++i) {
          Batch *g = retire(s, b, i);
          if (g) gone = g;
        }
      }
      delete gone;
      break;
    }
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->sched_done = true;
  }
  s->cv_cq.notify_all();
}

}  // namespace

extern "C" sobel4_status sobel4_server_create(sobel4_handle h, const sobel4_server_options *opt,
                                              sobel4_server *out) {
  if (!out) return SOBEL4_ERR_INVALID_ARG;
  *out = nullptr;
  if (!h || !opt || opt->border < SOBEL4_BORDER_VALID || opt->border > SOBEL4_BORDER_CONSTANT0 ||
      opt->format < SOBEL4_OUT_F32 || opt->format > SOBEL4_OUT_EDGE8 || opt->max_batch < 0 ||
      opt->memory_budget < 0 || opt->plain < 0 || opt->plain > 2)
    return SOBEL4_ERR_INVALID_ARG;
  sobel4_server_ctx *s = new (std::nothrow) sobel4_server_ctx();
  if (!s) return SOBEL4_ERR_OOM;
  s->h = h;
  s->device = sobel4::handle_info(h).device;
  s->opt = *opt;
  if (s->opt.memory_budget == 0) s->opt.memory_budget = 8ll << 30;
  if (s->opt.max_batch == 0) s->opt.max_batch = 256;
  sobel4::DeviceScope scope(s->device);
  cudaError_t e = cudaMalloc((void **)&s->arena_mem, (size_t)s->opt.memory_budget);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->down, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();  // the failure is reported here, not by a later call
    sobel4_server_destroy(s);
    return e == cudaErrorMemoryAllocation ? SOBEL4_ERR_OOM : SOBEL4_ERR_CUDA;
  }
  s->arena.reset((size_t)s->opt.memory_budget);
  s->sched = std::thread(scheduler, s);
  s->completer = std::thread(completer, s);
  *out = s;
  return SOBEL4_OK;
}

extern "C" sobel4_status sobel4_server_submit(sobel4_server s, const uint8_t *h_src,
                                              size_t src_pitch, void *h_dst, size_t dst_pitch,
                                              int32_t height, int32_t width, uint64_t *ticket) {
  if (!s || !h_src || !h_dst || !ticket || height < 1 || width < 1 ||
      src_pitch < (size_t)width || dst_pitch < (size_t)width * elem_bytes(s->opt.format) ||
      (s->opt.border == SOBEL4_BORDER_REFLECT101 && (height < 3 || width < 3)))
    return SOBEL4_ERR_INVALID_ARG;
  Request r;
  r.h_src = h_src;
  r.sp = src_pitch;
  r.h_dst = h_dst;
  r.dp = dst_pitch;
  r.H = height;
  r.W = width;
  r.d_sp = round_up((size_t)width, 16);
  r.d_dp = round_up((size_t)width * elem_bytes(s->opt.format), 16);
  r.in_bytes = r.d_sp * (size_t)height;
  const size_t planes = s->opt.format == SOBEL4_OUT_S16X4 ? 4 : 1;
  r.out_bytes = r.d_dp * (size_t)height * planes;
  {
    sobel4::DeviceScope scope(s->device);
    r.direct = sobel4::host_kernel_writable(h_dst, dst_pitch, (size_t)height * planes,
                                            (size_t)width * elem_bytes(s->opt.format),
                                            elem_bytes(s->opt.format));
  }
  if (r.arena_bytes() > (size_t)s->opt.memory_budget)
    return SOBEL4_ERR_UNSUPPORTED;  // could never be admitted
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->failed) return SOBEL4_ERR_CUDA;
    if (s->stop) return SOBEL4_ERR_INVALID_ARG;
    const uint64_t t = s->next_ticket++;
    s->reqs.emplace(t, r);
    s->incoming.push_back(t);
    s->stats.submitted += 1;
    *ticket = t;
  }
  s->cv_work.notify_one();
  return SOBEL4_OK;
}

extern "C" sobel4_status sobel4_server_wait(sobel4_server s, uint64_t ticket, int64_t timeout_us,
                                            double *latency_us) {
  if (!s) return SOBEL4_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SOBEL4_ERR_INVALID_ARG;
  auto finished = [&] {
    const State st = s->reqs[ticket].state;
    return st == kDone || st == kFailed;
  };
  if (timeout_us < 0) {
    s->cv_done.wait(lock, finished);
  } else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), finished)) {
    return SOBEL4_ERR_TIMEOUT;  // still pending; wait again later
  }
  Request r = s->reqs[ticket];
  s->reqs.erase(ticket);
  if (r.state == kFailed) return SOBEL4_ERR_CUDA;
  if (latency_us)
    *latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
  return SOBEL4_OK;
}

extern "C" sobel4_status sobel4_server_stats(sobel4_server s, sobel4_server_counters *out) {
  if (!s || !out) return SOBEL4_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  out->device_bytes_in_use = (int64_t)s->arena.used();
  out->device_bytes_peak = (int64_t)s->arena.peak();
  return SOBEL4_OK;
}

extern "C" sobel4_status sobel4_server_destroy(sobel4_server s) {
  if (!s) return SOBEL4_OK;
  if (s->sched.joinable()) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->sched.join();
  }
  // the scheduler has exited (or never started): the completer retires what
  // is still on the GPU, then exits
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->sched_done = true;
  }
  s->cv_cq.notify_all();
  if (s->completer.joinable()) s->completer.join();
  sobel4::DeviceScope scope(s->device);
  for (cudaStream_t st : {s->up, s->comp, s->down})
    if (st) cudaStreamSynchronize(st);
  for (cudaStream_t st : {s->up, s->comp, s->down})
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  if (s->arena_mem) cudaFree(s->arena_mem);
  delete s;
  return SOBEL4_OK;
}
