// Serving loop: continuous batching of projection requests from an ensemble of independent droplet runs.
//
// Requests of any grid size arrive at any time (vofp_server_submit returns at once with a ticket).  A worker
// thread admits them as in-flight slots and device memory free up.  Plans stay resident: each plan (tables,
// factor tables and workspace, one block of the server's arena -- one cudaMalloc at creation, a first-fit
// free list being the memory-based admission) is kept after its request completes and is reused by the
// next request with the same grid, boundary conditions and options; a request that finds no idle plan of
// its shape gets a new one (host tables built without holding the lock, uploaded asynchronously), evicting
// the least recently used idle plans when the arena is full.  Each request runs on its slot's own stream,
// so the work of requests admitted while others are on the GPU overlaps on the device.  An event recorded
// after each request's kernels is polled by the worker (every 50 us while work is in flight), which then
// stamps the completion and frees the slot and the plan: there is no cudaMalloc, cudaFree, host callback
// or device synchronisation on the serving path.  Latency is measured from the request's arrival (a time on
// the server's clock the caller gives, else the submission) to that completion stamp, so any wait before
// the caller could submit counts; the waits before submission and in the server's queue are kept apart.  Each request runs exactly the kernels it would run alone (its plan depends only on its own grid),
// so its result does not depend on what else is in flight.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <string>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "solve_internal.h"

using namespace vofp;
using Clock = std::chrono::steady_clock;

namespace {

// A resident plan: placed in the arena, reused by every request of its shape while idle.
struct CachedPlan {
  std::string key;
  PlanPrep prep;  // prep.p is the bound plan
  size_t block_off, block_bytes;
  bool busy;
  bool bound;
  Clock::time_point last;
};

struct Req {
  unsigned long long id;
  vofp_request r;
  std::vector<double> dz;
  std::string key;    // grid, spacing, boundary conditions: requests with equal keys share plans
  CachedPlan* plan;   // while admitted
  Clock::time_point t_arrive;  // arrival (given by the caller on the server clock, else the submission)
  Clock::time_point t_submit;
  Clock::time_point t_launch;  // enqueued on its slot's stream
  Clock::time_point t_done;
  int status;
  bool done;
  bool prepared;  // plan->prep holds tables built for this request
  int slot;
};

struct Slot {
  cudaStream_t st;
  cudaEvent_t done;  // recorded after the request's last kernel; polled by the worker
  unsigned char* stage;
  size_t stage_bytes;
  bool busy;
  Req* req;
};

}  // namespace

struct vofp_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<unsigned long long, Req*> all;
  std::vector<Slot> slots;
  unsigned char* arena;
  size_t arena_bytes;
  std::map<size_t, size_t> free_list;  // offset -> bytes
  size_t in_use;
  vofp_opts opts;
  unsigned long long next_id;
  bool stop;
  std::thread worker;
  int device;
  Clock::time_point origin;  // zero of the server clock (vofp_server_clock)
  // statistics
  std::vector<double> lat;       // arrival -> completion
  std::vector<double> wait_sub;  // arrival -> submission
  std::vector<double> wait_q;    // submission -> enqueued
  unsigned long long completed, rejected, admitted;
  long long queued;  // submitted, not yet admitted or rejected
  double t_prepare, t_launch;  // worker seconds spent building plans and enqueuing work
  unsigned long long loops;
  double cells_done;
  Clock::time_point t0;
  // resident plans
  std::list<CachedPlan*> plans;  // least recently used first
  unsigned long long plan_hits, plan_misses, plan_evictions;
};

namespace {

// Requests beyond the free slots that the worker prepares and tries to admit per iteration (the oldest
// first; a request that cannot be placed does not block the ones behind it inside this window).
constexpr int kLookahead = 16;

bool arena_alloc(vofp_server* s, size_t bytes, size_t* off) {
  bytes = (bytes + 255) & ~(size_t)255;
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t roff = it->first + bytes;
      s->free_list.erase(it);
      if (rest) s->free_list[roff] = rest;
      s->in_use += bytes;
      return true;
    }
  }
  return false;
}

void arena_free(vofp_server* s, size_t off, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  s->in_use -= bytes;
  auto it = s->free_list.emplace(off, bytes).first;
  // merge with the next and the previous block
  auto nx = std::next(it);
  if (nx != s->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_list.erase(nx);
  }
  if (it != s->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_list.erase(it);
    }
  }
}

// Completion of the request on slot `k` (lock held): stamp it, free its slot and plan (which stays resident).
void complete(vofp_server* s, int k, Clock::time_point t) {
  Slot& sl = s->slots[k];
  Req* q = sl.req;
  q->t_done = t;
  q->done = true;
  sl.busy = false;
  sl.req = nullptr;
  CachedPlan* cp = q->plan;
  cp->busy = false;
  cp->last = t;
  s->plans.remove(cp);
  s->plans.push_back(cp);  // most recently used last
  q->plan = nullptr;
  s->completed++;
  s->cells_done += (double)q->r.n[0] * q->r.n[1] * q->r.n[2];
  s->lat.push_back(std::chrono::duration<double>(q->t_done - q->t_arrive).count());
  s->wait_sub.push_back(std::chrono::duration<double>(q->t_submit - q->t_arrive).count());
  s->wait_q.push_back(std::chrono::duration<double>(q->t_launch - q->t_submit).count());
}

// An idle resident plan for `key` (lock held), or NULL.
CachedPlan* find_idle(vofp_server* s, const std::string& key) {
  for (CachedPlan* cp : s->plans)
    if (!cp->busy && cp->bound && cp->key == key) return cp;
  return nullptr;
}

// Arena block for a new plan (lock held), evicting least recently used idle plans as needed.
bool alloc_plan_block(vofp_server* s, size_t bytes, size_t* off) {
  while (!arena_alloc(s, bytes, off)) {
    CachedPlan* victim = nullptr;
    for (CachedPlan* cp : s->plans)
      if (!cp->busy) {
        victim = cp;
        break;
      }
    if (!victim) return false;
    s->plans.remove(victim);
    arena_free(s, victim->block_off, victim->block_bytes);
    plan_free_host(victim->prep.p);
    delete victim;
    s->plan_evictions++;
  }
  return true;
}

// Host part of admission (no lock): build a new plan's tables into a resident-plan record for q.
// Returns a status; < 0 rejects the request.
int prepare_request(vofp_server* s, Req* q) {
  CachedPlan* cp = new CachedPlan();
  cp->key = q->key;
  cp->busy = false;
  cp->bound = false;
  const int st = plan_prepare(q->r.n[0], q->r.n[1], q->r.n[2], q->r.dx, q->r.dy, q->dz.data(), q->r.bc, &s->opts,
                              &cp->prep);
  if (st) {
    delete cp;
    return st;
  }
  cp->block_bytes = plan_prep_device_bytes(&cp->prep);
  q->plan = cp;
  q->prepared = true;
  if (cp->block_bytes > s->arena_bytes) return VOFP_ERR_BUSY;                            // can never fit
  if (plan_prep_stage_bytes(&cp->prep) > (size_t)(4 << 20)) return VOFP_ERR_UNSUPPORTED;  // staging size
  return VOFP_OK;
}

// Finish a request that will not run (lock held).
void reject(vofp_server* s, Req* q, int status) {
  q->status = status;
  q->done = true;
  q->t_done = Clock::now();
  if (q->plan && !q->plan->bound) {  // a prepared plan that never got a block
    plan_free_host(q->plan->prep.p);
    delete q->plan;
  }
  q->plan = nullptr;
  s->rejected++;
  s->queued--;
}

// Reserve a slot and a plan for q (lock held): an idle resident plan of q's shape, else the plan prepared
// for q placed in a new arena block.  False: not now (no slot, no memory, or q still needs its tables).
bool reserve(vofp_server* s, Req* q) {
  int slot = -1;
  for (size_t i = 0; i < s->slots.size(); ++i)
    if (!s->slots[i].busy) {
      slot = (int)i;
      break;
    }
  if (slot < 0) return false;
  CachedPlan* cp = find_idle(s, q->key);
  if (cp) {
    if (q->plan && !q->plan->bound) {  // tables built speculatively, not needed
      plan_free_host(q->plan->prep.p);
      delete q->plan;
    }
    s->plan_hits++;
  } else {
    if (!q->prepared) return false;
    cp = q->plan;
    if (!alloc_plan_block(s, cp->block_bytes, &cp->block_off)) return false;
    s->plans.push_back(cp);
    s->plan_misses++;
  }
  cp->busy = true;
  q->plan = cp;
  s->slots[slot].busy = true;
  q->slot = slot;
  s->admitted++;
  s->queued--;
  return true;
}

// Place a new plan (tables uploaded asynchronously), enqueue the projection and record the slot's completion
// event (no lock).
void launch_request(vofp_server* s, Req* q) {
  Slot& sl = s->slots[q->slot];
  CachedPlan* cp = q->plan;
  int st = VOFP_OK;
  q->t_launch = Clock::now();
  if (!cp->bound) {
    st = plan_bind(&cp->prep, s->arena + cp->block_off, sl.st, sl.stage);
    cp->bound = true;  // the stage buffer is free again once this stream passes the upload
  }
  if (!st) st = vofp_project(cp->prep.p, q->r.u, q->r.v, q->r.w, q->r.src, q->r.dt_over_rho0, q->r.p, sl.st, nullptr);
  if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) {
    cudaStreamSynchronize(sl.st);  // the worker's next poll then finds the event complete or in error
    st = VOFP_ERR_CUDA;
  }
  q->status = st;
}

// The worker takes submitted requests into its own queue, builds their plans without holding the lock,
// admits them oldest first as slots and arena memory allow (a large request does not block smaller ones),
// launches each outside the lock, and retires finished ones by polling their slots' events -- no host
// callbacks in the streams, which would stall the hardware queues the streams share.
void worker_loop(vofp_server* s) {
  cudaSetDevice(s->device);
  std::deque<Req*> local;
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->loops++;
    int inflight = 0;
    for (const Slot& sl : s->slots) inflight += sl.busy;
    if (local.empty() && inflight == 0) {
      s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
      if (s->stop && s->pending.empty()) break;
    }
    // retire finished requests
    bool retired = false;
    const Clock::time_point now = Clock::now();
    for (size_t k = 0; k < s->slots.size(); ++k) {
      if (!s->slots[k].busy || !s->slots[k].req) continue;
      const cudaError_t e = cudaEventQuery(s->slots[k].done);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) s->slots[k].req->status = VOFP_ERR_CUDA;
      complete(s, (int)k, now);
      retired = true;
    }
    if (retired) s->cv_done.notify_all();
    while (!s->pending.empty()) {
      local.push_back(s->pending.front());
      s->pending.pop_front();
    }
    int free_slots = 0;
    for (const Slot& sl : s->slots) free_slots += !sl.busy;
    // host tables for the requests next in line whose shape has no idle resident plan -- only as many as
    // could be admitted now, plus a short look-ahead: under overload thousands wait, and building (or even
    // matching) tables for all of them every iteration would starve the admissions
    std::vector<std::pair<Req*, int>> built;
    {
      int window = free_slots + kLookahead;
      for (Req* q : local) {
        if (window-- <= 0) break;
        if (!q->prepared && !q->done && !find_idle(s, q->key)) built.emplace_back(q, 0);
      }
    }
    if (!built.empty()) {
      lk.unlock();
      const Clock::time_point a = Clock::now();
      for (auto& b : built) b.second = prepare_request(s, b.first);
      const double dt = std::chrono::duration<double>(Clock::now() - a).count();
      lk.lock();
      s->t_prepare += dt;
      for (auto& b : built)
        if (b.second) {
          reject(s, b.first, b.second);
          s->cv_done.notify_all();
        }
    }
    bool progress = retired;
    int window = free_slots + kLookahead;
    for (auto it = local.begin(); it != local.end();) {
      Req* q = *it;
      if (q->done) {  // rejected above
        it = local.erase(it);
        progress = true;
        continue;
      }
      // nothing more can start without a free slot; past the look-ahead window no tables are ready
      if (free_slots == 0 || window-- <= 0) break;
      if (!reserve(s, q)) {
        ++it;
        continue;
      }
      s->slots[q->slot].req = q;
      --free_slots;
      it = local.erase(it);
      lk.unlock();
      const Clock::time_point a = Clock::now();
      launch_request(s, q);
      const double dt = std::chrono::duration<double>(Clock::now() - a).count();
      lk.lock();
      s->t_launch += dt;
      progress = true;
    }
    if (s->stop && s->pending.empty() && local.empty()) {
      bool any = false;
      for (const Slot& sl : s->slots) any |= sl.busy;
      if (!any) break;
    }
    // poll again shortly while work is on the GPU; a submission wakes the worker at once
    if (!progress) s->cv_work.wait_for(lk, std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" int vofp_server_create(size_t mem_budget_bytes, int max_inflight, const vofp_opts* opt,
                                  vofp_server** out) {
  if (!out || max_inflight < 1 || max_inflight > 256) return VOFP_ERR_INVALID_ARG;
  *out = nullptr;
  vofp_server* s = new vofp_server();
  if (opt)
    s->opts = *opt;
  else
    vofp_opts_default(&s->opts);
  s->opts.tune = 0;
  cudaGetDevice(&s->device);
  if (mem_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    mem_budget_bytes = fr / 2;
  }
  s->arena_bytes = mem_budget_bytes & ~(size_t)255;
  if (device_alloc((void**)&s->arena, s->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return VOFP_ERR_OOM;
  }
  s->free_list[0] = s->arena_bytes;
  s->in_use = 0;
  s->slots.resize(max_inflight);
  bool staged = true;
  for (auto& sl : s->slots) {
    cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    sl.req = nullptr;
    sl.stage_bytes = 4 << 20;
    if (!staged || pinned_alloc((void**)&sl.stage, sl.stage_bytes) != cudaSuccess) {
      cudaGetLastError();
      sl.stage = nullptr;
      sl.stage_bytes = 0;
      staged = false;
    }
    sl.busy = false;
  }
  if (!staged) {  // every slot needs its pinned staging buffer for the plan uploads: give everything back
    for (auto& sl : s->slots) {
      cudaStreamDestroy(sl.st);
      cudaEventDestroy(sl.done);
      if (sl.stage) cudaFreeHost(sl.stage);
    }
    cudaFree(s->arena);
    delete s;
    return VOFP_ERR_OOM;
  }
  s->next_id = 1;
  s->stop = false;
  s->completed = s->rejected = s->admitted = 0;
  s->queued = 0;
  s->plan_hits = s->plan_misses = s->plan_evictions = 0;
  s->t_prepare = s->t_launch = 0;
  s->loops = 0;
  s->cells_done = 0;
  s->t0 = Clock::now();
  s->origin = s->t0;
  init_kernel_attributes_fp64();
  init_kernel_attributes_mixed();
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return VOFP_OK;
}

extern "C" int vofp_server_submit(vofp_server* s, const vofp_request* r, unsigned long long* ticket) {
  if (!s || !r || !ticket || !r->u || !r->v || !r->w || !r->dz) return VOFP_ERR_INVALID_ARG;
  if (r->n[0] < 1 || r->n[1] < 1 || r->n[2] < 1 || !(r->dt_over_rho0 > 0)) return VOFP_ERR_INVALID_ARG;
  Req* q = new Req();
  q->r = *r;
  q->dz.assign(r->dz, r->dz + r->n[2]);
  q->r.dz = nullptr;
  {
    // plan key: grid, spacings and boundary conditions (bit patterns; the options are the server's)
    std::string k((const char*)r->n, sizeof(r->n));
    k.append((const char*)&r->dx, sizeof(double));
    k.append((const char*)&r->dy, sizeof(double));
    k.append((const char*)r->bc, sizeof(r->bc));
    k.append((const char*)q->dz.data(), sizeof(double) * q->dz.size());
    q->key = std::move(k);
  }
  q->plan = nullptr;
  q->t_submit = Clock::now();
  q->t_arrive = q->t_submit;
  if (r->arrival_s > 0) {
    const Clock::time_point a =
        s->origin + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(r->arrival_s));
    if (a < q->t_submit) q->t_arrive = a;  // an arrival in the future is taken as the submission
  }
  q->t_launch = q->t_submit;
  q->status = VOFP_OK;
  q->done = false;
  q->prepared = false;
  q->slot = -1;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->id = s->next_id++;
    s->all[q->id] = q;
    s->pending.push_back(q);
    s->queued++;
    *ticket = q->id;
  }
  s->cv_work.notify_one();
  return VOFP_OK;
}

static int finish_ticket(vofp_server* s, Req* q, vofp_info* info, double* latency_s) {
  const int st = q->status;
  if (latency_s) *latency_s = std::chrono::duration<double>(q->t_done - q->t_arrive).count();
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = st;
  }
  s->all.erase(q->id);
  delete q;
  return st < 0 ? st : VOFP_OK;
}

extern "C" int vofp_server_poll(vofp_server* s, unsigned long long ticket, vofp_info* info, double* latency_s) {
  if (!s) return VOFP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return VOFP_ERR_INVALID_ARG;
  if (!it->second->done) return 1;
  return finish_ticket(s, it->second, info, latency_s);
}

extern "C" int vofp_server_wait(vofp_server* s, unsigned long long ticket, double timeout_s, vofp_info* info,
                                double* latency_s) {
  if (!s) return VOFP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return VOFP_ERR_INVALID_ARG;
  Req* q = it->second;
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  if (!s->cv_done.wait_until(lk, until, [&] { return q->done; })) return VOFP_ERR_TIMEOUT;
  return finish_ticket(s, q, info, latency_s);
}

// out[0] completed, [1] admitted, [2] rejected, [3] queued, [4] arena bytes in use, [5] arena bytes,
// [6] p50 latency s, [7] p99 latency s, [8] cells solved (sum), [9] seconds since creation or reset,
// [10] worker seconds building plans, [11] worker seconds enqueuing work, [12] worker loop iterations,
// [13] requests served by a resident plan, [14] requests that needed a new plan, [15] plans evicted,
// [16] resident plans, [17] p99 arrival -> submission (s), [18] p99 submission -> enqueued (s).
static double percentile(std::vector<double> l, double q) {
  if (l.empty()) return 0.0;
  std::sort(l.begin(), l.end());
  size_t i = (size_t)(q * (l.size() - 1) + 0.5);
  return l[std::min(i, l.size() - 1)];
}

extern "C" int vofp_server_stats(vofp_server* s, double* out, int n, int reset) {
  if (!s || !out || n < 1) return VOFP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  double v[VOFP_SERVER_STATS] = {
      (double)s->completed, (double)s->admitted, (double)s->rejected, (double)s->queued, (double)s->in_use,
      (double)s->arena_bytes, percentile(s->lat, 0.50), percentile(s->lat, 0.99), s->cells_done,
      std::chrono::duration<double>(Clock::now() - s->t0).count(), s->t_prepare, s->t_launch, (double)s->loops,
      (double)s->plan_hits, (double)s->plan_misses, (double)s->plan_evictions, (double)s->plans.size(),
      percentile(s->wait_sub, 0.99), percentile(s->wait_q, 0.99)};
  for (int i = 0; i < n && i < VOFP_SERVER_STATS; ++i) out[i] = v[i];
  if (reset) {
    s->lat.clear();
    s->wait_sub.clear();
    s->wait_q.clear();
    s->completed = s->admitted = s->rejected = 0;
    s->cells_done = 0;
    s->t_prepare = s->t_launch = 0;
    s->loops = 0;
    s->plan_hits = s->plan_misses = s->plan_evictions = 0;
    s->t0 = Clock::now();
  }
  return VOFP_OK;
}

extern "C" int vofp_server_clock(vofp_server* s, double* seconds) {
  if (!s || !seconds) return VOFP_ERR_INVALID_ARG;
  *seconds = std::chrono::duration<double>(Clock::now() - s->origin).count();
  return VOFP_OK;
}

extern "C" void vofp_server_destroy(vofp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->worker.join();
  for (auto& sl : s->slots) cudaStreamSynchronize(sl.st);
  for (auto& kv : s->all) {
    Req* q = kv.second;
    if (q->plan && !q->plan->bound) {
      plan_free_host(q->plan->prep.p);
      delete q->plan;
    }
    delete q;
  }
  for (CachedPlan* cp : s->plans) {
    plan_free_host(cp->prep.p);
    delete cp;
  }
  for (auto& sl : s->slots) {
    cudaStreamDestroy(sl.st);
    cudaEventDestroy(sl.done);
    if (sl.stage) cudaFreeHost(sl.stage);
  }
  cudaFree(s->arena);
  delete s;
}
