// Serving loop: continuous batching of projection requests from an ensemble of independent droplet runs.
//
// Requests of any grid size arrive at any time (vofp_server_submit returns at once with a ticket).  A worker
// thread admits them as in-flight slots and device memory free up: each admitted request gets a plan built
// on the host (tables), placed in a block of the server's arena (one cudaMalloc at creation; the arena's
// free list is the memory-based admission), uploaded and solved asynchronously on the slot's own stream,
// so the work of requests admitted while others are on the GPU overlaps on the device.  A host callback
// enqueued after each request's kernels stamps its completion, returns its arena block and slot and wakes
// the worker: there is no cudaMalloc, cudaFree or device synchronisation on the serving path.  Latency is
// measured from submission to that completion stamp.  Each request runs exactly the kernels it would run
// alone (its plan depends only on its own grid), so its result does not depend on what else is in flight.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "solve_internal.h"

using namespace vofp;
using Clock = std::chrono::steady_clock;

namespace {

struct Req {
  unsigned long long id;
  vofp_request r;
  std::vector<double> dz;
  Clock::time_point t_submit;
  Clock::time_point t_done;
  int status;
  bool done;
  // in flight
  PlanPrep prep;
  bool prepared;
  size_t block_off, block_bytes;
  int slot;
};

struct Slot {
  cudaStream_t st;
  unsigned char* stage;
  size_t stage_bytes;
  bool busy;
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
  // statistics
  std::vector<double> lat;
  unsigned long long completed, rejected, admitted;
  double cells_done;
  Clock::time_point t0;
};

namespace {

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

struct DoneCtx {
  vofp_server* s;
  Req* q;
};

void CUDART_CB on_done(void* arg) {
  DoneCtx* c = (DoneCtx*)arg;
  vofp_server* s = c->s;
  Req* q = c->q;
  delete c;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->t_done = Clock::now();
    q->done = true;
    arena_free(s, q->block_off, q->block_bytes);
    s->slots[q->slot].busy = false;
    plan_free_host(q->prep.p);
    q->prep.p = nullptr;
    q->prep.host.clear();
    q->prep.host.shrink_to_fit();
    s->completed++;
    s->cells_done += (double)q->r.n[0] * q->r.n[1] * q->r.n[2];
    s->lat.push_back(std::chrono::duration<double>(q->t_done - q->t_submit).count());
  }
  s->cv_work.notify_one();
  s->cv_done.notify_all();
}

// Try to admit request q (lock held).  Returns true if it was launched or rejected (removed from pending).
bool try_admit(vofp_server* s, Req* q) {
  if (!q->prepared) {
    const int st = plan_prepare(q->r.n[0], q->r.n[1], q->r.n[2], q->r.dx, q->r.dy, q->dz.data(), q->r.bc, &s->opts,
                                &q->prep);
    if (st) {
      q->status = st;
      q->done = true;
      q->t_done = Clock::now();
      s->rejected++;
      return true;
    }
    q->prepared = true;
    q->block_bytes = plan_prep_device_bytes(&q->prep);
    if (q->block_bytes > s->arena_bytes) {
      q->status = VOFP_ERR_BUSY;
      q->done = true;
      q->t_done = Clock::now();
      plan_free_host(q->prep.p);
      q->prep.p = nullptr;
      s->rejected++;
      return true;
    }
  }
  int slot = -1;
  for (size_t i = 0; i < s->slots.size(); ++i)
    if (!s->slots[i].busy) {
      slot = (int)i;
      break;
    }
  if (slot < 0) return false;
  size_t off;
  if (!arena_alloc(s, q->block_bytes, &off)) return false;
  Slot& sl = s->slots[slot];
  if (plan_prep_stage_bytes(&q->prep) > sl.stage_bytes) {
    // (the staging buffers are sized at creation for axes up to 4096 cells; no pinned allocation here,
    // which could wait on the device while the lock is held)
    arena_free(s, off, q->block_bytes);
    q->status = VOFP_ERR_UNSUPPORTED;
    q->done = true;
    q->t_done = Clock::now();
    plan_free_host(q->prep.p);
    q->prep.p = nullptr;
    s->rejected++;
    return true;
  }
  sl.busy = true;
  q->slot = slot;
  q->block_off = off;
  int st = plan_bind(&q->prep, s->arena + off, sl.st, sl.stage);
  if (!st) {
    st = vofp_project(q->prep.p, q->r.u, q->r.v, q->r.w, q->r.src, q->r.dt_over_rho0, q->r.p, sl.st, nullptr);
  }
  q->status = st;
  s->admitted++;
  DoneCtx* c = new DoneCtx{s, q};
  if (cudaLaunchHostFunc(sl.st, on_done, c) != cudaSuccess) {
    // could not enqueue the completion: finish synchronously
    delete c;
    cudaStreamSynchronize(sl.st);
    q->t_done = Clock::now();
    q->done = true;
    arena_free(s, off, q->block_bytes);
    sl.busy = false;
    q->status = VOFP_ERR_CUDA;
  }
  return true;
}

void worker_loop(vofp_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
    if (s->stop && s->pending.empty()) break;
    // admit every pending request that fits now, oldest first (a large request does not block smaller ones)
    bool progress = false;
    int scanned = 0;
    for (auto it = s->pending.begin(); it != s->pending.end() && scanned < 256; ++scanned) {
      Req* q = *it;
      if (try_admit(s, q)) {
        it = s->pending.erase(it);
        progress = true;
        if (q->done) s->cv_done.notify_all();
      } else {
        ++it;
      }
    }
    if (!progress && !s->pending.empty()) {
      // nothing fits: wait for a completion (on_done notifies cv_work)
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
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
  if (cudaMalloc((void**)&s->arena, s->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return VOFP_ERR_OOM;
  }
  s->free_list[0] = s->arena_bytes;
  s->in_use = 0;
  s->slots.resize(max_inflight);
  for (auto& sl : s->slots) {
    cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    sl.stage_bytes = 4 << 20;
    if (cudaMallocHost((void**)&sl.stage, sl.stage_bytes) != cudaSuccess) {
      cudaGetLastError();
      sl.stage = nullptr;
      sl.stage_bytes = 0;
    }
    sl.busy = false;
  }
  s->next_id = 1;
  s->stop = false;
  s->completed = s->rejected = s->admitted = 0;
  s->cells_done = 0;
  s->t0 = Clock::now();
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
  q->t_submit = Clock::now();
  q->status = VOFP_OK;
  q->done = false;
  q->prepared = false;
  q->prep.p = nullptr;
  q->slot = -1;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->id = s->next_id++;
    s->all[q->id] = q;
    s->pending.push_back(q);
    *ticket = q->id;
  }
  s->cv_work.notify_one();
  return VOFP_OK;
}

static int finish_ticket(vofp_server* s, Req* q, vofp_info* info, double* latency_s) {
  const int st = q->status;
  if (latency_s) *latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
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

// out[0] completed, [1] admitted, [2] rejected, [3] pending, [4] arena bytes in use, [5] arena bytes,
// [6] p50 latency s, [7] p99 latency s, [8] cells solved (sum), [9] seconds since creation or reset.
extern "C" int vofp_server_stats(vofp_server* s, double* out, int n, int reset) {
  if (!s || !out || n < 1) return VOFP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> l = s->lat;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    size_t i = (size_t)(q * (l.size() - 1) + 0.5);
    return l[std::min(i, l.size() - 1)];
  };
  double v[10] = {(double)s->completed, (double)s->admitted, (double)s->rejected, (double)s->pending.size(),
                  (double)s->in_use,    (double)s->arena_bytes, pct(0.50), pct(0.99), s->cells_done,
                  std::chrono::duration<double>(Clock::now() - s->t0).count()};
  for (int i = 0; i < n && i < 10; ++i) out[i] = v[i];
  if (reset) {
    s->lat.clear();
    s->completed = s->admitted = s->rejected = 0;
    s->cells_done = 0;
    s->t0 = Clock::now();
  }
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
    if (kv.second->prep.p) plan_free_host(kv.second->prep.p);
    delete kv.second;
  }
  for (auto& sl : s->slots) {
    cudaStreamDestroy(sl.st);
    if (sl.stage) cudaFreeHost(sl.stage);
  }
  cudaFree(s->arena);
  delete s;
}
