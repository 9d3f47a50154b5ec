// mg_serve.cu -- serving loop: continuous batching of matrix-element requests on one GPU.
//
// A request is (process, seed, nevt): the events 0..nevt-1 of the seed's Philox stream are turned
// into momenta and matrix elements (the paper's workflow, Sec. 1 / Fig. 1) and returned to the host.
// Requests of different processes and sizes arrive at any time; a scheduler thread admits them as
// slots and device memory free up:
//   * a slot = one CUDA stream, one pre-reserved context per process and device/pinned buffers for
//     max_nevt events, all created up front, so serving allocates nothing and never synchronises
//     the device;
//   * admission: a free slot and (sum of in-flight device footprints + this request's) <=
//     hbm_cap_bytes; otherwise the request waits in FIFO order;
//   * the slots' streams run concurrently, so small requests overlap with each other and with large
//     ones on the GPU; completion is detected with events and the results staged through pinned
//     memory;
//   * half of the slots own high-priority streams and take the "small" requests (estimated work,
//     events x flops per event of the process, below one full 65,536-event g g -> t tbar g batch),
//     so their thread blocks are dispatched ahead of a large request's pending blocks; large
//     requests use the low-priority slots; a small request may pass a large one that waits for a
//     slot.
// Helicity masks are resident: one per process, computed when the server is created from the first
// params.hel_warmup events of Philox seed MG_SERVE_MASK_SEED and copied into every slot's context, so no
// request runs the filter.  A request's result depends only on (process, seed, nevt) and that mask, and
// every kernel sums in a fixed order, so a request gives the same bits alone and in any mix.  Requests
// larger than max_nevt run as consecutive chunks on one slot.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mg_alloc.h"
#include "mg_ctx.h"
#include "mg_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  bool small = true;
  uint64_t ticket;
  mg_process proc;
  uint64_t seed;
  int64_t nevt;
  Clock::time_point t_submit, t_done;
  std::vector<double> me;
  int64_t next = 0;          // first event of the next chunk
  int64_t computed = 0;      // events of the chunks that finished
  bool cancel = false;       // mg_serve_cancel while in flight: launch no further chunk
  bool done = false;
  mg_status status = MG_OK;
  int64_t footprint = 0;
};

struct Slot {
  bool high = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  mg_ctx* ctx[4] = {nullptr, nullptr, nullptr, nullptr};
  double* mom = nullptr;
  double* me = nullptr;
  double* host = nullptr;                 // pinned staging of one chunk's MEs
  unsigned long long* host_nbad = nullptr;
  Request* req = nullptr;
  int64_t chunk_e0 = 0, chunk_n = 0;
};

}  // namespace

struct mg_server {
  mg_serve_cfg cfg;
  int device = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  int64_t inflight_bytes = 0, peak_bytes = 0, completed = 0, events = 0;
  int inflight = 0, peak_inflight = 0;
  mg_status fatal = MG_OK;
};

namespace {

int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Enqueue the next chunk of s.req on the slot's stream.
mg_status launch_chunk(mg_server* srv, Slot& s) {
  Request* r = s.req;
  const int64_t n = min64(srv->cfg.max_nevt, r->nevt - r->next);
  s.chunk_e0 = r->next;
  s.chunk_n = n;
  mg_ctx* ctx = s.ctx[r->proc];
  mg_status st = mg_rambo_range(ctx, r->seed, r->next, n, srv->cfg.sqrts, s.mom, nullptr, s.stream);
  if (st == MG_OK) st = mg_sigmakin(ctx, s.mom, n, srv->cfg.precision, s.me, s.stream);
  if (st != MG_OK) return st;
  if (cudaMemcpyAsync(s.host, s.me, n * sizeof(double), cudaMemcpyDeviceToHost, s.stream) != cudaSuccess ||
      cudaMemcpyAsync(s.host_nbad, ctx->d_nbad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s.stream) !=
          cudaSuccess ||
      cudaMemsetAsync(ctx->d_nbad, 0, sizeof(unsigned long long), s.stream) != cudaSuccess ||
      cudaEventRecord(s.ev, s.stream) != cudaSuccess)
    return MG_ECUDA;
  r->next += n;
  return MG_OK;
}

void worker_loop(mg_server* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    bool progressed = false;
    // completions
    for (Slot& s : srv->slots) {
      if (!s.req) continue;
      const cudaError_t q = cudaEventQuery(s.ev);
      if (q == cudaErrorNotReady) continue;
      Request* r = s.req;
      progressed = true;
      if (q != cudaSuccess) {
        cudaGetLastError();
        r->status = MG_ECUDA;
        r->next = r->nevt;
      } else {
        std::memcpy(r->me.data() + s.chunk_e0, s.host, s.chunk_n * sizeof(double));
        r->computed += s.chunk_n;
        if (*s.host_nbad && r->status == MG_OK) r->status = MG_ENOCONV;
      }
      if (r->cancel && r->next < r->nevt && r->status != MG_ECUDA) {
        r->status = MG_ECANCELED;
        r->next = r->nevt;
      }
      if (r->next < r->nevt && r->status != MG_ECUDA) {
        const mg_status st = launch_chunk(srv, s);
        if (st != MG_OK) { r->status = st; r->next = r->nevt; }
        else continue;
      }
      r->done = true;
      r->t_done = Clock::now();
      s.req = nullptr;
      srv->inflight--;
      srv->inflight_bytes -= r->footprint;
      srv->completed++;
      srv->events += r->computed;
      srv->cv_done.notify_all();
    }
    // admission: FIFO within each class; small requests take high-priority slots first and may
    // pass a large request that is waiting for a low-priority slot
    for (auto it = srv->queue.begin(); it != srv->queue.end();) {
      Request* r = *it;
      Slot* free_slot = nullptr;
      for (Slot& s : srv->slots)
        if (!s.req && s.high == r->small) { free_slot = &s; break; }
      if (!free_slot && r->small)
        for (Slot& s : srv->slots)
          if (!s.req) { free_slot = &s; break; }
      if (!free_slot) { ++it; continue; }
      if (srv->inflight > 0 && srv->inflight_bytes + r->footprint > srv->cfg.hbm_cap_bytes) break;
      it = srv->queue.erase(it);
      free_slot->req = r;
      srv->inflight++;
      srv->inflight_bytes += r->footprint;
      if (srv->inflight > srv->peak_inflight) srv->peak_inflight = srv->inflight;
      if (srv->inflight_bytes > srv->peak_bytes) srv->peak_bytes = srv->inflight_bytes;
      const mg_status st = launch_chunk(srv, *free_slot);
      progressed = true;
      if (st != MG_OK) {
        r->status = st;
        r->done = true;
        r->t_done = Clock::now();
        free_slot->req = nullptr;
        srv->inflight--;
        srv->inflight_bytes -= r->footprint;
        srv->cv_done.notify_all();
      }
    }
    if (srv->stop && srv->inflight == 0 && srv->queue.empty()) break;
    if (!progressed) {
      if (srv->inflight == 0 && srv->queue.empty() && !srv->stop)
        srv->cv_work.wait(lk);
      else
        srv->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

void destroy_slots(mg_server* srv) {
  for (Slot& s : srv->slots) {
    for (mg_ctx*& c : s.ctx)
      if (c) { mg_destroy(c); c = nullptr; }
    if (s.mom) mg::dev_free(s.mom);
    if (s.me) mg::dev_free(s.me);
    if (s.host) mg::host_free(s.host);
    if (s.host_nbad) mg::host_free(s.host_nbad);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  srv->slots.clear();
}

}  // namespace

extern "C" {

void mg_serve_default_cfg(mg_serve_cfg* c) {
  if (!c) return;
  c->slots = 8;
  c->max_nevt = 65536;
  c->hbm_cap_bytes = int64_t(64) << 30;
  c->precision = MG_FP64;
  c->sqrts = 1500.0;
  mg_default_params(&c->params);
}

int64_t mg_serve_footprint(mg_process proc, int64_t nevt, mg_precision precision) {
  if (proc < MG_GG_TT || proc > MG_GG_TTGGG || nevt < 0) return -1;
  return mg::footprint_bytes(proc, nevt, precision);
}

mg_status mg_serve_create(const mg_serve_cfg* cfg_in, mg_server** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  mg_serve_cfg cfg;
  mg_serve_default_cfg(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.slots < 1 || cfg.slots > 64 || cfg.max_nevt < 32 || cfg.hbm_cap_bytes < 1 ||
      !(cfg.sqrts > 2.0 * cfg.params.mt) || cfg.precision < MG_FP64 || cfg.precision > MG_MIXED)
    return MG_EINVAL;
  mg_server* srv = new (std::nothrow) mg_server;
  if (!srv) return MG_ENOMEM;
  srv->cfg = cfg;
  srv->cfg.max_nevt = (cfg.max_nevt + 31) / 32 * 32;
  if (cudaGetDevice(&srv->device) != cudaSuccess) { cudaGetLastError(); delete srv; return MG_ECUDA; }
  srv->slots.resize(cfg.slots);
  mg_status st = MG_OK;
  const int64_t nmax = srv->cfg.max_nevt;
  int prio_low = 0, prio_high = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) { cudaGetLastError(); prio_low = prio_high = 0; }
  for (size_t i = 0; i < srv->slots.size(); ++i) {
    Slot& s = srv->slots[i];
    s.high = cfg.slots > 1 && i < srv->slots.size() / 2;
    if (cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, s.high ? prio_high : prio_low) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
        mg::dev_alloc(&s.mom, static_cast<size_t>(mg_mom_count(MG_GG_TTGGG, nmax)) * sizeof(double)) != cudaSuccess ||
        mg::dev_alloc(&s.me, nmax * sizeof(double)) != cudaSuccess ||
        mg::host_alloc(&s.host, nmax * sizeof(double)) != cudaSuccess ||
        mg::host_alloc(&s.host_nbad, sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      st = MG_ENOMEM;
      break;
    }
    for (int p = 0; p < 4 && st == MG_OK; ++p) {
      st = mg_create(static_cast<mg_process>(p), &cfg.params, &s.ctx[p]);
      if (st == MG_OK) st = mg::ctx_reserve(s.ctx[p], nmax, cfg.precision);
    }
    if (st != MG_OK) break;
  }
  // resident helicity masks: computed once per process on slot 0's context from the fixed warm-up sample,
  // copied to the other slots' contexts
  for (int p = 0; p < 4 && st == MG_OK; ++p) {
    Slot& s0 = srv->slots[0];
    const int64_t nw = cfg.params.hel_warmup < nmax ? cfg.params.hel_warmup : nmax;
    st = mg_rambo(s0.ctx[p], MG_SERVE_MASK_SEED, nw, cfg.sqrts, s0.mom, nullptr, s0.stream);
    if (st == MG_OK) st = mg_hel_filter(s0.ctx[p], s0.mom, nw, s0.stream);
    for (size_t i = 1; i < srv->slots.size() && st == MG_OK; ++i) st = mg::ctx_copy_mask(srv->slots[i].ctx[p], s0.ctx[p], s0.stream);
    if (st == MG_OK && cudaStreamSynchronize(s0.stream) != cudaSuccess) { cudaGetLastError(); st = MG_ECUDA; }
    if (st == MG_OK && mg_check(s0.ctx[p], s0.stream, nullptr) != MG_OK) st = MG_ENOCONV;
  }
  if (st == MG_OK && cudaDeviceSynchronize() != cudaSuccess) { cudaGetLastError(); st = MG_ECUDA; }
  if (st != MG_OK) {
    destroy_slots(srv);
    delete srv;
    return st;
  }
  srv->worker = std::thread(worker_loop, srv);
  *out = srv;
  return MG_OK;
}

mg_status mg_serve_submit(mg_server* srv, mg_process proc, uint64_t seed, int64_t nevt, uint64_t* ticket) {
  if (!srv || !ticket || proc < MG_GG_TT || proc > MG_GG_TTGGG || nevt < 1) return MG_EINVAL;
  Request* r = new (std::nothrow) Request;
  if (!r) return MG_ENOMEM;
  try {
    r->me.assign(nevt, 0.0);
  } catch (...) {
    delete r;
    return MG_ENOMEM;
  }
  r->proc = proc;
  r->seed = seed;
  r->nevt = nevt;
  r->footprint = mg::footprint_bytes(proc, min64(nevt, srv->cfg.max_nevt), srv->cfg.precision);
  // estimated work: events x FP64 flops per event of the process (mg_flops_per_event, all helicities)
  static const double kFlopsPerEvent[4] = {8.6e3, 7.56e4, 9.58e5, 1.67e7};
  r->small = srv->cfg.slots == 1 || static_cast<double>(nevt) * kFlopsPerEvent[proc] <= 65536.0 * kFlopsPerEvent[1];
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(srv->mu);
    if (srv->stop) { delete r; return MG_EINVAL; }
    r->ticket = srv->next_ticket++;
    srv->reqs[r->ticket] = r;
    srv->queue.push_back(r);
  }
  srv->cv_work.notify_one();
  *ticket = r->ticket;
  return MG_OK;
}

static mg_status take_result(mg_server* srv, Request* r, double* me_out, double* latency_ms) {
  if (me_out) std::memcpy(me_out, r->me.data(), r->nevt * sizeof(double));
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const mg_status st = r->status;
  srv->reqs.erase(r->ticket);
  delete r;
  return st;
}

mg_status mg_serve_poll(mg_server* srv, uint64_t ticket, double* me_out_host, int* done, double* latency_ms) {
  if (!srv || !done) return MG_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return MG_EINVAL;
  Request* r = it->second;
  if (!r->done) { *done = 0; return MG_OK; }
  *done = 1;
  return take_result(srv, r, me_out_host, latency_ms);
}

mg_status mg_serve_wait(mg_server* srv, uint64_t ticket, double* me_out_host, int64_t timeout_ms, double* latency_ms) {
  if (!srv || timeout_ms < 0) return MG_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return MG_EINVAL;
  Request* r = it->second;
  if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [r] { return r->done; }))
    return MG_ETIMEOUT;
  return take_result(srv, r, me_out_host, latency_ms);
}

mg_status mg_serve_cancel(mg_server* srv, uint64_t ticket) {
  if (!srv) return MG_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return MG_EINVAL;
  Request* r = it->second;
  if (r->done) return MG_OK;
  for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q) {
    if (*q != r) continue;
    srv->queue.erase(q);   // not admitted yet: nothing of it ran
    r->status = MG_ECANCELED;
    r->done = true;
    r->t_done = Clock::now();
    srv->completed++;
    srv->cv_done.notify_all();
    return MG_OK;
  }
  r->cancel = true;        // in flight: the worker stops it at its next chunk boundary
  return MG_OK;
}

mg_status mg_serve_stats(mg_server* srv, int64_t* completed, int64_t* events, int64_t* peak_bytes, int* peak_inflight) {
  if (!srv) return MG_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  if (completed) *completed = srv->completed;
  if (events) *events = srv->events;
  if (peak_bytes) *peak_bytes = srv->peak_bytes;
  if (peak_inflight) *peak_inflight = srv->peak_inflight;
  return MG_OK;
}

void mg_serve_destroy(mg_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  cudaDeviceSynchronize();
  destroy_slots(srv);
  for (auto& kv : srv->reqs) delete kv.second;
  delete srv;
}

}  // extern "C"
