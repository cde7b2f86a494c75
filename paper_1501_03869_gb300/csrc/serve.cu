// serve.cu -- request loop of the on-line reconstruction (include/pat_bp.h,
// serving).  Sec. III separates the off-line table build from the on-line
// frame reconstruction; this layer serves the on-line step to a stream of
// single-frame requests for several subjects (speed maps):
//   * admission: a subject's table (and working buffers) must be resident to
//     run; tables live within an HBM budget, the least recently used idle
//     subject is evicted to its pinned host copy when room is needed (its
//     device buffers handed straight to the incoming subject when their sizes
//     match, so the reload is only the upload);
//   * batching: the pending frames of one subject (same dtype, arrival order,
//     up to max_batch_frames) go in one reconstruction;
//   * continuous batching: batches of different subjects run concurrently on
//     separate streams; requests arriving meanwhile are queued and admitted
//     as streams and memory free up.
// A frame's result does not depend on its batch (fixed summation order).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handle.h"

using namespace patbp;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int subject = 0;
  const void* sig = nullptr;
  pat_dtype dtype = PAT_F32;
  const float* scales = nullptr;
  float* out = nullptr;
  double t_submit = 0.0;
  double latency = 0.0;
  pat_status status = PAT_PENDING;
};

struct Subject {
  pat_bp_t h = nullptr;
  uint64_t last_use = 0;
  bool busy = false;
};

// A result whose host buffer is pageable: the device copies it into the
// slot's page-locked staging buffer, and the scheduler copies it on to the
// caller's buffer once the batch is done (outside the server lock).
struct HostCopy {
  void* dst;
  const void* src;
  size_t bytes;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  int subject = -1;
  std::vector<uint64_t> tickets;
  std::vector<HostCopy> out_copies;
  void* d_sig = nullptr;
  size_t sig_cap = 0;
  float* d_sc = nullptr;
  size_t sc_cap = 0;
  float* d_out = nullptr;
  size_t out_cap = 0;
  void* h_sig = nullptr;   // page-locked staging of pageable signals and scales
  size_t h_sig_cap = 0;
  void* h_out = nullptr;   // page-locked staging of results for pageable buffers
  size_t h_out_cap = 0;
};

pat_status grow_dev(void** p, size_t* cap, size_t need) {
  if (need <= *cap) return PAT_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need) != cudaSuccess) return fail(PAT_ERR_OOM, "serving staging buffer");
  *cap = need;
  return PAT_OK;
}

pat_status grow_pinned(void** p, size_t* cap, size_t need) {
  if (need <= *cap) return PAT_OK;
  cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost(p, need) != cudaSuccess) return fail(PAT_ERR_OOM, "serving host staging buffer");
  *cap = need;
  return PAT_OK;
}

// True for page-locked host memory, which copy engines read and write
// asynchronously (a copy to or from pageable memory can block the host).
bool page_locked(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

}  // namespace

struct pat_srv_s {
  int device = 0;
  size_t budget = 0;
  pat_srv_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<Subject> subjects;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Slot> slots;
  uint64_t next_ticket = 1, tick = 0;
  uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, uploads = 0, evictions = 0;
  uint64_t batched_frames = 0;
  std::vector<double> latencies;
  bool stop = false;
  std::thread th;
};

namespace {

size_t resident_total(pat_srv_t s) {
  size_t t = 0;
  for (const Subject& sub : s->subjects) t += resident_bytes(sub.h);
  return t;
}

// Bytes a subject needs on the device to run a batch of max_batch_frames.
size_t subject_need(pat_srv_t s, pat_bp_t h) {
  const size_t frames = size_t(s->cfg.max_batch_frames);
  size_t work = (frames * h->ns * h->nt_pad + 16 * 8) * 4 + frames * h->ns_pad * 4;
  work += std::max(frames, size_t(h->SW)) * h->n_tiles * h->n_seg * h->P * 4 + frames * h->n_tiles * 4;
  return table_device_bytes(h) + work;
}

void finish(pat_srv_t s, uint64_t t, pat_status st) {
  auto it = s->reqs.find(t);
  if (it == s->reqs.end()) return;
  it->second.status = st;
  it->second.latency = now_s() - it->second.t_submit;
  if (st == PAT_OK) {
    ++s->completed;
    s->latencies.push_back(it->second.latency);
  } else {
    ++s->failed;
  }
}

void reap(pat_srv_t s, std::unique_lock<std::mutex>& lk) {
  bool any = false;
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    cudaError_t e = cudaEventQuery(sl.ev);
    if (e == cudaErrorNotReady) continue;
    pat_status st = e == cudaSuccess ? PAT_OK : cuda_fail(e, "serving batch");
    if (st == PAT_OK && !sl.out_copies.empty()) {
      // results of pageable buffers: the slot stays busy (nobody else touches
      // it or its requests' buffers) while the lock is released for the copies
      lk.unlock();
      for (const HostCopy& c : sl.out_copies) std::memcpy(c.dst, c.src, c.bytes);
      lk.lock();
    }
    sl.out_copies.clear();
    if (st == PAT_OK) {
      int flag = 0;
      pat_bp_t h = s->subjects[sl.subject].h;
      if (cudaMemcpy(&flag, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && flag) {
        cudaMemset(h->d_status, 0, sizeof(int));
        if (h->d_counter) cudaMemset(h->d_counter, 0, h->counter_cap);
        cudaMemset(h->d_sched, 0, 4 * sizeof(unsigned));
        st = fail(PAT_ERR_TIMEOUT, "a device wait ran out of time");
      }
    }
    for (uint64_t t : sl.tickets) finish(s, t, st);
    sl.tickets.clear();
    s->subjects[sl.subject].busy = false;
    sl.busy = false;
    any = true;
  }
  if (any) s->cv_done.notify_all();
}

// Working buffers for the largest batch, allocated while the subject becomes
// resident: a batch never grows them later, because the cudaFree of a growth
// would synchronise the device and stall every batch in flight.  They cover
// every smaller batch too (n frames in groups of FB take at most as much).
pat_status reserve_batch_buffers(pat_srv_t s, pat_bp_t h) {
  const int F = s->cfg.max_batch_frames;
  return ensure_buffers_fb(h, F, frames_per_group(F));
}

// Make subject k resident within the budget, evicting least recently used idle
// subjects.  PAT_ERR_BUSY: not now (others busy); PAT_ERR_OOM: never fits.
pat_status admit(pat_srv_t s, int k, cudaStream_t st) {
  pat_bp_t h = s->subjects[k].h;
  if (!h->evicted) return PAT_OK;
  const size_t need = subject_need(s, h);
  if (need > s->budget) return fail(PAT_ERR_OOM, "subject does not fit in the HBM budget");
  while (resident_total(s) + need > s->budget) {
    int victim = -1;
    for (int i = 0; i < int(s->subjects.size()); ++i) {
      const Subject& c = s->subjects[i];
      if (i == k || c.busy || c.h->evicted) continue;
      if (victim < 0 || c.last_use < s->subjects[victim].last_use) victim = i;
    }
    if (victim < 0) return PAT_ERR_BUSY;
    // an idle victim of the same sizes hands its buffers over (no device
    // synchronisation, free or allocation); any other is evicted normally
    if (!donate_buffers_locked(s->subjects[victim].h, h)) {
      pat_status e = evict_locked(s->subjects[victim].h);
      if (e != PAT_OK) return e;
    }
    ++s->evictions;
  }
  pat_status e = restore_locked(h, st);
  if (e != PAT_OK) return e;
  ++s->uploads;
  return reserve_batch_buffers(s, h);
}

// Launch one batch of subject k's pending requests (same dtype) on slot sl.
pat_status launch_batch(pat_srv_t s, Slot& sl, int k, const std::vector<uint64_t>& ts) {
  pat_bp_t h = s->subjects[k].h;
  const Request& r0 = s->reqs[ts[0]];
  const size_t F = ts.size();
  const size_t esz = r0.dtype == PAT_F32 ? 4 : 2;
  const size_t row = size_t(h->ns) * h->nt * esz;
  const size_t out_row = size_t(h->out_stride) * 4;
  pat_status st;
  if ((st = grow_dev(&sl.d_sig, &sl.sig_cap, F * row)) != PAT_OK) return st;
  if ((st = grow_dev(reinterpret_cast<void**>(&sl.d_out), &sl.out_cap, F * out_row)) != PAT_OK) return st;
  const bool lowp = r0.dtype != PAT_F32;
  if (lowp && (st = grow_dev(reinterpret_cast<void**>(&sl.d_sc), &sl.sc_cap, F * h->ns * 4)) != PAT_OK)
    return st;
  // Inputs: page-locked buffers are copied as they are; pageable ones are first
  // packed into the slot's page-locked staging buffer (frames, then scales).
  const size_t sc_row = size_t(h->ns) * 4;
  size_t staged = 0;
  for (size_t f = 0; f < F; ++f) {
    const Request& r = s->reqs[ts[f]];
    if (!page_locked(r.sig)) staged += row;
    if (lowp && !page_locked(r.scales)) staged += sc_row;
  }
  if (staged && (st = grow_pinned(&sl.h_sig, &sl.h_sig_cap, staged)) != PAT_OK) return st;
  size_t at = 0;
  auto copy_in = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (page_locked(src)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, sl.st);
    char* stage = static_cast<char*>(sl.h_sig) + at;
    std::memcpy(stage, src, bytes);
    at += bytes;
    return cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyHostToDevice, sl.st);
  };
  for (size_t f = 0; f < F; ++f) {
    const Request& r = s->reqs[ts[f]];
    PAT_CUDA(copy_in(static_cast<char*>(sl.d_sig) + f * row, r.sig, row));
    if (lowp) PAT_CUDA(copy_in(sl.d_sc + f * h->ns, r.scales, sc_row));
  }
  if ((st = reconstruct_locked(h, sl.d_sig, r0.dtype, lowp ? sl.d_sc : nullptr, int(F), sl.d_out,
                               sl.st)) != PAT_OK)
    return st;
  // Results: straight into page-locked buffers, else into the staging buffer
  // (copied on to the caller's buffer when the batch is reaped).
  size_t n_pageable = 0;
  for (size_t f = 0; f < F; ++f) n_pageable += page_locked(s->reqs[ts[f]].out) ? 0 : 1;
  if (n_pageable && (st = grow_pinned(&sl.h_out, &sl.h_out_cap, n_pageable * out_row)) != PAT_OK)
    return st;
  sl.out_copies.clear();
  size_t n_staged = 0;
  for (size_t f = 0; f < F; ++f) {
    float* dst = s->reqs[ts[f]].out;
    const char* src = reinterpret_cast<const char*>(sl.d_out) + f * out_row;
    if (page_locked(dst)) {
      PAT_CUDA(cudaMemcpyAsync(dst, src, out_row, cudaMemcpyDeviceToHost, sl.st));
    } else {
      char* stage = static_cast<char*>(sl.h_out) + n_staged++ * out_row;
      PAT_CUDA(cudaMemcpyAsync(stage, src, out_row, cudaMemcpyDeviceToHost, sl.st));
      sl.out_copies.push_back(HostCopy{dst, stage, out_row});
    }
  }
  PAT_CUDA(cudaEventRecord(sl.ev, sl.st));
  return PAT_OK;
}

// Admit and launch as many batches as free streams, memory and the queue allow.
void schedule(pat_srv_t s) {
  std::vector<bool> tried(s->subjects.size(), false);
  for (;;) {
    Slot* free_slot = nullptr;
    for (Slot& sl : s->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (!free_slot) return;
    // the subject of the oldest pending request that can run now
    int k = -1;
    pat_dtype dt = PAT_F32;
    for (uint64_t t : s->pending) {
      const Request& r = s->reqs[t];
      if (!s->subjects[r.subject].busy && !tried[r.subject]) {
        k = r.subject;
        dt = r.dtype;
        break;
      }
    }
    if (k < 0) return;
    tried[k] = true;
    pat_status st = admit(s, k, free_slot->st);
    if (st == PAT_ERR_BUSY) continue;  // wait for running batches to free memory
    std::vector<uint64_t> batch;
    for (auto it = s->pending.begin(); it != s->pending.end();) {
      const Request& r = s->reqs[*it];
      if (r.subject == k && r.dtype == dt && int(batch.size()) < s->cfg.max_batch_frames) {
        batch.push_back(*it);
        it = s->pending.erase(it);
      } else {
        ++it;
      }
    }
    if (st == PAT_OK) st = launch_batch(s, *free_slot, k, batch);
    if (st != PAT_OK) {
      for (uint64_t t : batch) finish(s, t, st);
      s->cv_done.notify_all();
      continue;
    }
    free_slot->busy = true;
    free_slot->subject = k;
    free_slot->tickets = batch;
    s->subjects[k].busy = true;
    s->subjects[k].last_use = ++s->tick;
    ++s->batches;
    s->batched_frames += batch.size();
  }
}

void scheduler_main(pat_srv_t s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (s->cfg.stall_us > 0) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(s->cfg.stall_us));
      lk.lock();
    }
    reap(s, lk);
    schedule(s);
    bool busy = false;
    for (const Slot& sl : s->slots) busy = busy || sl.busy;
    if (s->stop && !busy && s->pending.empty()) break;
    if (busy)
      s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    else
      s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
  }
}

}  // namespace

extern "C" pat_status pat_srv_create(size_t hbm_budget, const pat_srv_cfg* cfg, pat_srv_t* out) {
  if (!out) return fail(PAT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (hbm_budget == 0) return fail(PAT_ERR_INVALID, "hbm_budget must be > 0");
  pat_srv_t s = new (std::nothrow) pat_srv_s();
  if (!s) return fail(PAT_ERR_OOM, "server");
  s->budget = hbm_budget;
  s->cfg.n_streams = 4;
  s->cfg.max_batch_frames = 16;
  s->cfg.max_queue = 4096;
  s->cfg.stall_us = 0;
  if (cfg) {
    if (cfg->n_streams > 0) s->cfg.n_streams = std::min(cfg->n_streams, 32);
    if (cfg->max_batch_frames > 0) s->cfg.max_batch_frames = std::min(cfg->max_batch_frames, 1024);
    if (cfg->max_queue > 0) s->cfg.max_queue = cfg->max_queue;
    s->cfg.stall_us = std::max(0, cfg->stall_us);
  }
  cudaGetDevice(&s->device);
  s->slots.resize(size_t(s->cfg.n_streams));
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      delete s;
      return fail(PAT_ERR_CUDA, "server streams");
    }
  }
  s->th = std::thread(scheduler_main, s);
  *out = s;
  return PAT_OK;
}

extern "C" pat_status pat_srv_register(pat_srv_t s, const float* speed_host, const pat_grid* grid,
                                       const double* sensors_host, int n_sensors,
                                       const uint8_t* mask_host, const float* weights_host,
                                       double dt, int n_samples, unsigned flags, int* subject_id) {
  if (!s || !subject_id) return fail(PAT_ERR_INVALID, "NULL argument");
  cudaSetDevice(s->device);
  pat_bp_t h = nullptr;
  pat_status st = pat_bp_create(speed_host, grid, sensors_host, n_sensors, mask_host, weights_host, dt,
                                n_samples, flags | PAT_FLAG_HOST_MIRROR, &h);
  if (st != PAT_OK) return st;
  std::lock_guard<std::mutex> lk(s->mu);
  // every slot's staging for a full batch of this subject (FP32 signals, the
  // largest), so no batch grows them later: a growth's cudaFree would
  // synchronise the device and stall the batches in flight
  {
    const size_t F = size_t(s->cfg.max_batch_frames);
    for (Slot& sl : s->slots) {
      if ((st = grow_dev(&sl.d_sig, &sl.sig_cap, F * h->ns * h->nt * 4)) != PAT_OK ||
          (st = grow_dev(reinterpret_cast<void**>(&sl.d_sc), &sl.sc_cap, F * h->ns * 4)) != PAT_OK ||
          (st = grow_dev(reinterpret_cast<void**>(&sl.d_out), &sl.out_cap, F * size_t(h->out_stride) * 4)) != PAT_OK) {
        pat_bp_destroy(h);
        return st;
      }
    }
  }
  // resident until the scheduler needs the room: account it now
  if (resident_total(s) + subject_need(s, h) > s->budget) {
    evict_locked(h);
  } else if ((st = reserve_batch_buffers(s, h)) != PAT_OK) {
    pat_bp_destroy(h);
    return st;
  }
  s->subjects.push_back(Subject{h, 0, false});
  *subject_id = int(s->subjects.size()) - 1;
  return PAT_OK;
}

extern "C" pat_status pat_srv_submit(pat_srv_t s, int subject, const void* signals_host,
                                     pat_dtype dtype, const float* scales_host, float* out_host,
                                     uint64_t* ticket) {
  if (!s || !ticket) return fail(PAT_ERR_INVALID, "NULL argument");
  if (!signals_host || !out_host) return fail(PAT_ERR_INVALID, "signals/out NULL");
  if (dtype != PAT_F32 && dtype != PAT_BF16 && dtype != PAT_F16) return fail(PAT_ERR_INVALID, "dtype");
  if (dtype != PAT_F32 && !scales_host) return fail(PAT_ERR_INVALID, "16-bit signals need scales");
  std::lock_guard<std::mutex> lk(s->mu);
  if (subject < 0 || subject >= int(s->subjects.size())) return fail(PAT_ERR_NOT_FOUND, "unknown subject");
  if (int(s->pending.size()) >= s->cfg.max_queue) return fail(PAT_ERR_BUSY, "request queue full");
  Request r;
  r.subject = subject;
  r.sig = signals_host;
  r.dtype = dtype;
  r.scales = scales_host;
  r.out = out_host;
  r.t_submit = now_s();
  const uint64_t t = s->next_ticket++;
  s->reqs.emplace(t, r);
  s->pending.push_back(t);
  ++s->submitted;
  *ticket = t;
  s->cv_work.notify_one();
  return PAT_OK;
}

extern "C" pat_status pat_srv_poll(pat_srv_t s, uint64_t ticket, int timeout_us, double* latency_s) {
  if (!s) return fail(PAT_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(PAT_ERR_NOT_FOUND, "unknown ticket");
  if (it->second.status == PAT_PENDING && timeout_us > 0) {
    s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] {
      auto j = s->reqs.find(ticket);
      return j == s->reqs.end() || j->second.status != PAT_PENDING;
    });
    it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(PAT_ERR_NOT_FOUND, "unknown ticket");
  }
  const pat_status st = it->second.status;
  if (st == PAT_PENDING) return PAT_PENDING;
  if (latency_s) *latency_s = it->second.latency;
  s->reqs.erase(it);
  return st;
}

extern "C" pat_status pat_srv_stats(pat_srv_t s, pat_srv_stats_t* out) {
  if (!s || !out) return fail(PAT_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->batches = s->batches;
  out->uploads = s->uploads;
  out->evictions = s->evictions;
  out->mean_batch_frames = s->batches ? double(s->batched_frames) / double(s->batches) : 0.0;
  out->resident_bytes = resident_total(s);
  out->budget_bytes = s->budget;
  if (!s->latencies.empty()) {
    std::vector<double> v(s->latencies);
    std::sort(v.begin(), v.end());
    auto q = [&](double p) { return v[std::min(v.size() - 1, size_t(p * double(v.size() - 1) + 0.5))]; };
    out->p50_ms = q(0.50) * 1e3;
    out->p99_ms = q(0.99) * 1e3;
  }
  return PAT_OK;
}

extern "C" pat_status pat_srv_set_budget(pat_srv_t s, size_t hbm_budget) {
  if (!s) return fail(PAT_ERR_INVALID, "NULL server");
  if (hbm_budget == 0) return fail(PAT_ERR_INVALID, "hbm_budget must be > 0");
  std::lock_guard<std::mutex> lk(s->mu);
  cudaSetDevice(s->device);
  s->budget = hbm_budget;
  // idle subjects leave, least recently used first, until the rest fit; busy
  // ones stay until their batches are done (admissions then respect the budget)
  while (resident_total(s) > s->budget) {
    int victim = -1;
    for (int i = 0; i < int(s->subjects.size()); ++i) {
      const Subject& c = s->subjects[i];
      if (c.busy || c.h->evicted) continue;
      if (victim < 0 || c.last_use < s->subjects[victim].last_use) victim = i;
    }
    if (victim < 0) break;
    pat_status e = evict_locked(s->subjects[victim].h);
    if (e != PAT_OK) return e;
    ++s->evictions;
  }
  return PAT_OK;
}

extern "C" pat_status pat_srv_destroy(pat_srv_t s) {
  if (!s) return PAT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  for (Slot& sl : s->slots) {
    cudaFree(sl.d_sig);
    cudaFree(sl.d_sc);
    cudaFree(sl.d_out);
    cudaFreeHost(sl.h_sig);
    cudaFreeHost(sl.h_out);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  for (Subject& sub : s->subjects) pat_bp_destroy(sub.h);
  delete s;
  return PAT_OK;
}
