// Serving loop: continuous batching of cube-synthesis requests.
//
// Each slot owns two CUDA streams, of the highest and the lowest priority, and a status
// word.  A scheduler thread admits a queued request as soon as a slot is free and the
// request's workspace fits in the part of the HBM budget that running requests have not
// reserved: the oldest that fits (first fit), or the one with the least estimated device
// time among those that fit (shortest first).  A request can be passed over only until
// it has waited the age limit; after that it is next, whether or not it fits yet, so no
// request starves.  Express slots, beyond the general ones, take only short requests
// (estimated device time under 2 ms), so these never wait in the queue behind long
// requests that hold every general slot.  A request whose estimated device time is short runs on the
// high-priority stream: when long requests' kernels hold the SMs, the block scheduler
// starts its blocks as soon as any resources free up instead of after the long kernels'
// remaining blocks.  (Measured on the mixed serving workload: p50 and p99 both lower than
// with one priority; a third, middle level lowered p50 further but raised p99.)  The
// workspace comes from the stream-ordered allocator on the slot's stream and goes
// back to it when the request completes, so memory frees up in launch order.  Work
// of different slots overlaps on the device.  Completion is reported by a host
// function enqueued after the request's kernels, which stamps the latency and
// wakes the scheduler and any waiter.
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "rsim_ctx.h"

namespace rsim {
namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2 };

struct Slot;
struct Server;

struct Req {
  uint64_t ticket = 0;
  rsim_request r{};
  Consts k{};
  rsim_plan plan{};
  size_t bytes = 0;
  int state = kQueued;
  rsim_status result = RSIM_OK;
  Clock::time_point t_submit, t_admit, t_done;
  double est_ms = 0.0;  // estimated device time: path-samples at the tier's nominal rate
  int slot = -1;
  int prio = 0;  // index into the slot's streams: 0 high priority, 1 low
  void* ws = nullptr;
};

constexpr int kPrios = 2;

struct Slot {
  cudaStream_t st[kPrios] = {};         // highest priority first
  unsigned* status = nullptr;           // device status word of this slot
  unsigned long long* pv_host = nullptr;  // pinned: P_valid of the request in flight
  uint64_t ticket = 0;
  bool busy = false;
  Server* srv = nullptr;
  int index = 0;
};

}  // namespace
}  // namespace rsim

struct rsim_server {
  rsim_ctx* ctx = nullptr;
  rsim_server_opts opts{};
  std::vector<rsim::Slot> slots;
  std::deque<uint64_t> queue;
  std::map<uint64_t, rsim::Req> reqs;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::thread sched;
  bool stop = false;
  uint64_t next_ticket = 1;
  size_t reserved = 0;
  // statistics
  rsim_server_stats stats{};
  std::vector<double> lat_ms, queue_ms;
  std::chrono::milliseconds age_limit{100};  // overtaking allowed until a request waited this long
  bool have_first = false;
  rsim::Clock::time_point t_first, t_last;
  int in_flight = 0;
  // Slots whose host function fired, to be retired.  Guarded by cb_mu alone, which is
  // never held across a CUDA call: the host function runs on CUDA's callback thread, and
  // a CUDA call made while holding a lock it needs (the scheduler launches work holding
  // `mu`; a launch that first loads a kernel module can wait for device work, including
  // that host function) would never return.
  std::mutex cb_mu;
  std::vector<int> completed_slots;
};

namespace rsim {
namespace {

struct HostFnArg {
  rsim_server* s;
  int slot;
};

// Runs on a CUDA-owned host thread after the slot's kernels: no CUDA calls here.
void CUDART_CB on_complete(void* p) {
  HostFnArg* a = (HostFnArg*)p;
  rsim_server* s = a->s;
  {
    std::lock_guard<std::mutex> g(s->cb_mu);
    s->completed_slots.push_back(a->slot);
  }
  s->cv_sched.notify_all();  // a missed wake-up costs at most the scheduler's 50 ms poll
  delete a;
}

// Retire a finished slot: read its status, free the workspace, record latency.
void retire(rsim_server* s, int si) {
  Slot& sl = s->slots[si];
  auto it = s->reqs.find(sl.ticket);
  unsigned w = 0;
  cudaMemcpy(&w, sl.status, 4, cudaMemcpyDeviceToHost);
  if (w) cudaMemset(sl.status, 0, 4);
  cudaError_t e = cudaGetLastError();
  if (it != s->reqs.end()) {
    Req& r = it->second;
    r.t_done = Clock::now();
    if (r.ws) cudaFreeAsync(r.ws, sl.st[r.prio]);
    r.ws = nullptr;
    s->reserved -= r.bytes;
    if (e != cudaSuccess) r.result = RSIM_ERR_CUDA;
    else if (w & kStatusTimeout) r.result = RSIM_ERR_TIMEOUT;
    else if (w & kStatusNonfinite) r.result = RSIM_ERR_NONFINITE;
    r.state = kDone;
    const double ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
    if (r.result == RSIM_OK) {
      s->stats.completed++;
      s->lat_ms.push_back(ms);
      s->queue_ms.push_back(std::chrono::duration<double, std::milli>(r.t_admit - r.t_submit).count());
      s->stats.path_samples += (double)(*sl.pv_host) * r.k.V * r.k.Ns * r.k.L;
    } else {
      s->stats.failed++;
    }
    s->t_last = r.t_done;
  }
  sl.busy = false;
  sl.ticket = 0;
  s->in_flight--;
}

// Position in the queue of the request to admit next, or -1 when none may start now.
// The queue is in submission order, so its head is the oldest request: once the head has
// waited the age limit (or the limit is negative: strict FIFO) only the head may start on
// a general slot.  For an express slot (short_only) only short requests qualify; an aged
// long head keeps its claim on the budget (an express request must leave room for it),
// and an aged short head goes first.
long pick_next(rsim_server* s, Clock::time_point now, bool short_only) {
  const size_t budget = s->opts.hbm_budget_bytes;
  const Req& head = s->reqs[s->queue.front()];
  const bool head_aged = s->opts.age_limit_ms < 0 || now - head.t_submit >= s->age_limit;
  const size_t keep = (short_only && head_aged && head.prio != 0) ? head.bytes : 0;
  auto fits = [&](const Req& r) { return !budget || s->reserved + r.bytes + keep <= budget; };
  if (head_aged && (!short_only || head.prio == 0)) return fits(head) ? 0 : -1;
  long best = -1;
  for (size_t i = 0; i < s->queue.size(); ++i) {
    const Req& r = s->reqs[s->queue[i]];
    if (short_only && r.prio != 0) continue;
    if (!fits(r)) continue;
    if (s->opts.policy == RSIM_SERVE_FIRST_FIT) return (long)i;
    if (best < 0 || r.est_ms < s->reqs[s->queue[best]].est_ms) best = (long)i;
  }
  return best;
}

// Try to start one queued request on a free slot.  Called with the lock held.  Slots
// [0, slots) are general; the express slots after them take short requests only, and a
// short request picked for a general slot goes to a free express slot instead, keeping
// the general slots for long requests.
bool admit_one(rsim_server* s) {
  if (s->queue.empty()) return false;
  const int n_general = s->opts.slots;
  int gen = -1, exp = -1;
  for (int i = 0; i < (int)s->slots.size(); ++i) {
    if (s->slots[i].busy) continue;
    if (i < n_general && gen < 0) gen = i;
    if (i >= n_general && exp < 0) exp = i;
  }
  if (gen < 0 && exp < 0) return false;
  const Clock::time_point now = Clock::now();
  long qi = -1;
  int free_slot = -1;
  if (gen >= 0) {
    qi = pick_next(s, now, false);
    if (qi >= 0) free_slot = (s->reqs[s->queue[qi]].prio == 0 && exp >= 0) ? exp : gen;
  }
  if (qi < 0 && exp >= 0) {
    qi = pick_next(s, now, true);
    free_slot = exp;
  }
  if (qi < 0) return false;
  Req& r = s->reqs[s->queue[qi]];
  if (qi > 0) s->stats.overtakes++;
  s->queue.erase(s->queue.begin() + qi);
  r.t_admit = now;
  Slot& sl = s->slots[free_slot];
  cudaStream_t rs = sl.st[r.prio];
  cudaError_t e = cudaMallocAsync(&r.ws, r.bytes, rs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    r.result = RSIM_ERR_OOM;
    r.state = kDone;
    r.t_done = Clock::now();
    s->stats.failed++;
    s->cv_done.notify_all();
    return true;
  }
  s->reserved += r.bytes;
  s->stats.peak_reserved_bytes = std::max(s->stats.peak_reserved_bytes, s->reserved);
  r.state = kRunning;
  r.slot = free_slot;
  sl.busy = true;
  sl.ticket = r.ticket;
  s->in_flight++;
  s->stats.peak_in_flight = std::max(s->stats.peak_in_flight, s->in_flight);
  void* cubes[1] = {r.r.cube};
  char what[64];
  snprintf(what, sizeof what, "request %llu", (unsigned long long)r.ticket);
  NvtxRange request_range(what);
  rsim_status st = run_frames(s->ctx, (char*)r.ws, r.bytes, r.k, &r.r.pixels, 1, cubes, r.r.tier,
                              r.r.out_dtype, r.plan, sl.status, rs);
  // P_valid of this request, read by retire() once the stream reaches it
  size_t o = ((sizeof(FrameIO) + 255) / 256) * 256;
  cudaMemcpyAsync(sl.pv_host, (char*)r.ws + o, 8, cudaMemcpyDeviceToHost, rs);
  r.result = st;
  HostFnArg* a = new HostFnArg{s, free_slot};
  e = cudaLaunchHostFunc(rs, on_complete, a);
  if (e != cudaSuccess) {
    delete a;
    cudaGetLastError();
    r.result = RSIM_ERR_CUDA;
    cudaStreamSynchronize(rs);
    retire(s, free_slot);
    s->cv_done.notify_all();
  }
  return true;
}

void scheduler(rsim_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progressed = false;
    std::vector<int> done;
    {
      std::lock_guard<std::mutex> g(s->cb_mu);
      done.swap(s->completed_slots);
    }
    for (int si : done) {
      retire(s, si);
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    while (!s->stop && admit_one(s)) {
    }
    if (s->stop && s->in_flight == 0) {
      std::lock_guard<std::mutex> g(s->cb_mu);
      if (s->completed_slots.empty()) break;
    }
    s->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  size_t i = (size_t)std::ceil(q * v.size());  // nearest rank
  if (i < 1) i = 1;
  if (i > v.size()) i = v.size();
  return v[i - 1];
}

}  // namespace
}  // namespace rsim

using namespace rsim;

extern "C" {

rsim_status rsim_server_create(rsim_ctx* ctx, const rsim_server_opts* opts, rsim_server** out) {
  if (!ctx || !opts || !out) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  if (opts->slots < 1 || opts->slots > 64) return fail(RSIM_ERR_INVALID_ARG, "slots must be in 1..64");
  if (opts->express_slots < 0 || opts->express_slots > 64)
    return fail(RSIM_ERR_INVALID_ARG, "express_slots must be in 0..64");
  if (opts->max_queue < 1) return fail(RSIM_ERR_INVALID_ARG, "max_queue must be >= 1");
  if (opts->policy != RSIM_SERVE_FIRST_FIT && opts->policy != RSIM_SERVE_SHORTEST_FIRST)
    return fail(RSIM_ERR_INVALID_ARG, "unknown admission policy");
  cudaSetDevice(ctx->device);
  rsim_server* s = new rsim_server();
  s->ctx = ctx;
  s->opts = *opts;
  if (opts->age_limit_ms > 0) s->age_limit = std::chrono::milliseconds(opts->age_limit_ms);
  const int n_slots = opts->slots + opts->express_slots;
  s->slots.resize(n_slots);
  for (int i = 0; i < n_slots; ++i) {
    Slot& sl = s->slots[i];
    sl.index = i;
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int q = 0; q < kPrios && e == cudaSuccess; ++q) {
      // greatest (numerically lowest) first, least last
      const int pr = greatest + (least - greatest) * q / (kPrios - 1);
      e = cudaStreamCreateWithPriority(&sl.st[q], cudaStreamNonBlocking, pr);
    }
    if (e == cudaSuccess) e = cudaMalloc(&sl.status, 256);
    if (e == cudaSuccess) e = cudaMemset(sl.status, 0, 256);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.pv_host, 64);
    if (e != cudaSuccess) {
      rsim_server_destroy(s);
      return cuda_fail(e, "server slot set-up");
    }
  }
  s->sched = std::thread(scheduler, s);
  *out = s;
  return RSIM_OK;
}

rsim_status rsim_server_submit(rsim_server* s, const rsim_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  Req r;
  r.r = *req;
  rsim_status st = check_params(&req->params, &r.k);
  if (st != RSIM_OK) return st;
  st = check_pixels(&req->pixels);
  if (st != RSIM_OK) return st;
  if (!tier_ok(req->tier)) return fail(RSIM_ERR_INVALID_ARG, "unknown tier");
  if (req->out_dtype != RSIM_C64 && req->out_dtype != RSIM_C128)
    return fail(RSIM_ERR_INVALID_ARG, "out_dtype must be RSIM_C64 or RSIM_C128");
  if (!req->cube) return fail(RSIM_ERR_INVALID_ARG, "cube is NULL");
  if (tensor_tier(req->tier) && !(s->ctx->cc_major == 10 && s->ctx->cc_minor == 3))
    return fail(RSIM_ERR_UNSUPPORTED, "tensor-core tiers need an sm_103 device");
  r.plan = choose_plan(s->ctx, req->tier, r.k, req->pixels.P);
  int64_t P = req->pixels.P;
  r.bytes = batch_bytes(r.k, &P, 1, r.plan, req->tier);
  // estimated device time from the path-samples at the tier's nominal rate (CUDA cores
  // about 6e12/s, tensor cores and the NUFFT about 6e13/s): high priority under 2 ms
  const double work = (double)req->pixels.P * r.k.V * r.k.Ns * r.k.L;
  r.est_ms = work / (req->tier == RSIM_TIER_FP32 ? 6e12 : 6e13) * 1e3;
  r.prio = r.est_ms < 2.0 ? 0 : 1;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->opts.hbm_budget_bytes && r.bytes > s->opts.hbm_budget_bytes)
    return fail(RSIM_ERR_BUDGET, "request workspace exceeds the server HBM budget");
  if ((int)s->queue.size() >= s->opts.max_queue) return fail(RSIM_ERR_BUDGET, "server queue is full");
  r.ticket = s->next_ticket++;
  r.t_submit = Clock::now();
  if (!s->have_first) {
    s->have_first = true;
    s->t_first = r.t_submit;
  }
  s->stats.submitted++;
  *ticket = r.ticket;
  s->reqs[r.ticket] = r;
  s->queue.push_back(r.ticket);
  s->cv_sched.notify_all();
  return RSIM_OK;
}

rsim_status rsim_server_wait(rsim_server* s, uint64_t ticket, int32_t timeout_ms) {
  if (!s) return fail(RSIM_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto done = [&] {
    auto it = s->reqs.find(ticket);
    return it == s->reqs.end() || it->second.state == kDone;
  };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    return fail(RSIM_ERR_TIMEOUT, "request has not finished");
  }
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(RSIM_ERR_NOT_FOUND, "unknown or already collected ticket");
  rsim_status r = it->second.result;
  s->reqs.erase(it);
  if (r == RSIM_ERR_NONFINITE) return fail(r, "a valid pixel has a non-finite field or R <= 0");
  if (r == RSIM_ERR_CANCELLED) return fail(r, "request was cancelled");
  if (r != RSIM_OK) return fail(r, "request failed");
  return RSIM_OK;
}

rsim_status rsim_server_cancel(rsim_server* s, uint64_t ticket) {
  if (!s) return fail(RSIM_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(RSIM_ERR_NOT_FOUND, "unknown ticket");
  if (it->second.state != kQueued) return fail(RSIM_ERR_INVALID_ARG, "request already admitted");
  s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), ticket), s->queue.end());
  it->second.state = kDone;
  it->second.result = RSIM_ERR_CANCELLED;
  s->stats.cancelled++;
  s->cv_done.notify_all();
  return RSIM_OK;
}

rsim_status rsim_server_stats_get(rsim_server* s, rsim_server_stats* out) {
  if (!s || !out) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->stats;
  out->p50_ms = percentile(s->lat_ms, 0.50);
  out->p99_ms = percentile(s->lat_ms, 0.99);
  double sum = 0, mx = 0;
  for (double x : s->lat_ms) {
    sum += x;
    mx = std::max(mx, x);
  }
  out->mean_ms = s->lat_ms.empty() ? 0 : sum / s->lat_ms.size();
  out->max_ms = mx;
  out->p99_queue_ms = percentile(s->queue_ms, 0.99);
  out->max_queue_ms = s->queue_ms.empty() ? 0.0 : *std::max_element(s->queue_ms.begin(), s->queue_ms.end());
  out->busy_s = s->have_first ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
  return RSIM_OK;
}

rsim_status rsim_server_stats_reset(rsim_server* s) {
  if (!s) return fail(RSIM_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  s->stats = rsim_server_stats{};
  s->stats.peak_reserved_bytes = s->reserved;
  s->stats.peak_in_flight = s->in_flight;
  s->lat_ms.clear();
  s->queue_ms.clear();
  s->have_first = false;
  return RSIM_OK;
}

rsim_status rsim_server_destroy(rsim_server* s) {
  if (!s) return RSIM_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    for (uint64_t t : s->queue) {
      s->reqs[t].state = kDone;
      s->reqs[t].result = RSIM_ERR_CANCELLED;
    }
    s->queue.clear();
  }
  s->cv_sched.notify_all();
  if (s->sched.joinable()) s->sched.join();
  cudaSetDevice(s->ctx->device);
  for (Slot& sl : s->slots) {
    for (int q = 0; q < kPrios; ++q) {
      if (!sl.st[q]) continue;
      cudaStreamSynchronize(sl.st[q]);
      cudaStreamDestroy(sl.st[q]);
    }
    if (sl.status) cudaFree(sl.status);
    if (sl.pv_host) cudaFreeHost(sl.pv_host);
  }
  delete s;
  return RSIM_OK;
}

}  // extern "C"
