// Kernel tracing: when enabled, every launch of the library is bracketed by a pair of CUDA events recorded
// on the launching stream; vofp_trace_collect() waits for them and returns the summed device time and the
// launch count per kernel class.  Disabled by default (one relaxed atomic load per launch).
#include <atomic>
#include <mutex>
#include <vector>

#include "solve_internal.h"

namespace vofp {

static const char* kNames[KID_COUNT] = {
    "x_forward",   "x_forward_div",   "x_forward_stefan", "x_forward_div_stefan", "y_forward",
    "z_tridiag",   "y_inverse",       "x_inverse",        "grad_update",          "extend_epilogue",
    "stefan_source", "residual_update", "batched",        "noalloc_tables",
    "z_low_modes", "gauge_shift",     "vd_predict",
    "vof_update"};

struct TraceRec {
  int kid;
  cudaEvent_t a, b;
};

static std::atomic<int> g_on{0};
static std::mutex g_mu;
static std::vector<TraceRec> g_recs;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void trace_begin(int kid, cudaStream_t st, TraceTok* tok) {
  tok->active = 0;
  if (!g_on.load(std::memory_order_relaxed) || capturing()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  tok->active = 1;
  tok->kid = kid;
  tok->a = get_event();
  tok->b = get_event();
  cudaEventRecord(tok->a, st);
}

void trace_end(TraceTok* tok, cudaStream_t st) {
  if (!tok->active) return;
  cudaEventRecord(tok->b, st);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({tok->kid, tok->a, tok->b});
}

// Allocation-failure injection (tests of the out-of-memory paths without exhausting a GPU): while
// g_fail_after = k >= 0, the next k allocations succeed and the one after fails, once.
static std::atomic<long long> g_fail_after{-1};

static bool inject_failure() {
  long long v = g_fail_after.load();
  while (v >= 0)
    if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}

cudaError_t device_alloc(void** p, size_t bytes) {
  if (inject_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t pinned_alloc(void** p, size_t bytes) {
  if (inject_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

// Readers of the bounds-checked build's device words, one per translation unit (registered during the
// library's static initialisation; the plain build registers none).
typedef int (*ChkReader)(long long*, int);
static std::vector<ChkReader>& chk_readers() {
  static std::vector<ChkReader> r;
  return r;
}
int chk_register(int (*read)(long long* out, int reset)) {
  chk_readers().push_back(read);
  return (int)chk_readers().size();
}

// One index test that fails by construction and touches no memory.
static __global__ void k_check_selftest(int idx, int ext) { (void)VOFP_IN(idx, ext, CHK_SELFTEST); }

}  // namespace vofp

using namespace vofp;

extern "C" int vofp_debug_fail_alloc(long long after) {
  g_fail_after.store(after < 0 ? -1 : after);
  return VOFP_OK;
}

extern "C" int vofp_debug_check_word(long long* out, int reset) {
  if (!out) return VOFP_ERR_INVALID_ARG;
  for (int q = 0; q < 4; ++q) out[q] = 0;
  if (chk_readers().empty()) return 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return VOFP_ERR_CUDA;
  for (ChkReader rd : chk_readers()) {
    long long w[4];
    if (rd(w, reset) != 0) return VOFP_ERR_CUDA;
    if (w[0] > 0 && out[0] == 0) {
      out[1] = w[1];
      out[2] = w[2];
      out[3] = w[3];
    }
    out[0] += w[0];
  }
  return 1;
}

extern "C" int vofp_debug_check_selftest(void* stream) {
  k_check_selftest<<<1, 1, 0, (cudaStream_t)stream>>>(5, 4);
  return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

extern "C" int vofp_trace_enable(int on) {
  const int prev = g_on.exchange(on ? 1 : 0);
  return prev;
}

extern "C" int vofp_trace_collect(double* ms, unsigned long long* count, int n) {
  if (!ms || !count || n <= 0) return VOFP_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    ms[i] = 0;
    count[i] = 0;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  int status = VOFP_OK;
  for (const TraceRec& r : g_recs) {
    float t = 0;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
      status = VOFP_ERR_CUDA;
    if (r.kid >= 0 && r.kid < n) {
      ms[r.kid] += t;
      count[r.kid] += 1;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  return status;
}

extern "C" const char* vofp_trace_name(int id) { return (id >= 0 && id < KID_COUNT) ? kNames[id] : "unknown"; }

extern "C" int vofp_trace_kernel_classes(void) { return KID_COUNT; }
