// Launch-shape autotuner.
//
// For one plan it times whole Poisson solves (CUDA events on a private stream, after a warm-up) while
// walking each knob in turn -- line pairs per block of the x passes, columns per block of the y passes, the
// z kernel (segmented tiles, shared-memory staged chains, or streamed chains with their systems per block),
// and the order of the FFT radix stages on x and on y (the plan's factorisation or its reverse) -- and keeps
// the fastest value of each (coordinate descent over the candidates that fit in shared memory).  Results are cached per process and, when the environment
// variable VOFP_TUNE_CACHE names a file, in that file (one line per grid/precision/GPU key), so a serving
// process or a batch pays the search once per shape.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "solve_internal.h"
#include "zsolve.cuh"

namespace {

struct Shape {
  int xpb, ytx, zti, ord;
};

std::mutex g_mu;
std::map<std::string, Shape> g_cache;
std::string g_loaded_path;  // the cache file last read (read again when VOFP_TUNE_CACHE names another)

std::string key_of(const vofp_plan* p) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, p->device);
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|%d|%d|%d|%d|%d|%d|%d", prop.name, p->n[0], p->n[1], p->n[2], p->bc[0], p->bc[1],
           p->bc[2], p->opts.prec);
  for (char* c = buf; *c; ++c)
    if (*c == ' ') *c = '_';
  return buf;
}

void load_file() {
  const char* path = getenv("VOFP_TUNE_CACHE");
  if (!path || g_loaded_path == path) return;
  g_loaded_path = path;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512], k[256];
  while (fgets(line, sizeof(line), f)) {
    Shape s{0, 0, 0, 0};
    if (sscanf(line, "%255s %d %d %d %d", k, &s.xpb, &s.ytx, &s.zti, &s.ord) >= 4) g_cache[k] = s;
  }
  fclose(f);
}

void save_entry(const std::string& k, const Shape& s) {
  const char* path = getenv("VOFP_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d\n", k.c_str(), s.xpb, s.ytx, s.zti, s.ord);
  fclose(f);
}

// the reduced-precision (refinement) paths keep their shapes in ytx32 / zti32
bool mixed(const vofp_plan* p) { return p->opts.prec != VOFP_FP64; }

// Reverse the radix sequence of an axis (any order of the stages gives the same transform, up to rounding).
void reverse_stages(vofp::FftDesc& fd) {
  for (int a = 0, b = fd.nst - 1; a < b; ++a, --b) {
    const int t = fd.radix[a];
    fd.radix[a] = fd.radix[b];
    fd.radix[b] = t;
  }
}

void apply(vofp_plan* p, const Shape& s) {
  for (int a = 0; a < 2; ++a)
    if (((s.ord ^ p->radix_order) >> a) & 1) reverse_stages(p->ax[a].fd);
  p->radix_order = s.ord;
  p->xpb = s.xpb;
  if (mixed(p)) {
    p->ytx32 = s.ytx;
    p->zti32 = s.zti;
  } else {
    p->ytx = s.ytx;
    p->zti = s.zti;
  }
}

Shape current(const vofp_plan* p) {
  return Shape{p->xpb, mixed(p) ? p->ytx32 : p->ytx, mixed(p) ? p->zti32 : p->zti, p->radix_order};
}

bool fits(const vofp_plan* p, const Shape& s) {
  const bool f32 = p->opts.prec == VOFP_MIXED;
  const size_t c = f32 ? sizeof(float2) : sizeof(double2);
  const size_t r = f32 ? sizeof(float) : sizeof(double);
  const size_t lim = 160 * 1024;
  const int sx = vofp::fft_span(p->ax[0].fd, p->ax[0].blu64), sy = vofp::fft_span(p->ax[1].fd, p->ax[1].blu64);
  if (s.xpb < 1 || s.xpb > vofp::kMaxPB) return false;  // the x passes keep per-line tables of 2 kMaxPB
  if (2 * (size_t)s.xpb * sx * c > lim) return false;
  if (2 * (size_t)(s.ytx / 2) * vofp::y_ld(sy) * c > lim) return false;
  if (s.zti > 128) return false;  // at most 128 systems per block
  if (!p->ztab && s.zti < 1) return false;
  if (p->ztab) {  // factor-table kernels: -1 = segmented tiles, 0 = staged (if the tile fits), else whole
                  // warps of one system each
    const size_t e = f32 ? sizeof(float) : sizeof(double);
    if (s.zti == -1 || s.zti == -2) return vofp::ztab_seg_smem(p->n[2], e, s.zti == -2) <= 200 * 1024;
    return s.zti == 0 ? vofp::ztab_staged_smem(p->n[2], e) <= 200 * 1024 : s.zti >= 32;
  }
  return (size_t)3 * s.zti * p->n[2] * r <= lim;
}

// Average milliseconds of a Poisson solve of the plan's scratch potential (in place).
float time_solve(vofp_plan* p, cudaStream_t st) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int reps = 4;
  vofp_poisson_solve(p, p->P, p->P, st, nullptr);
  cudaEventRecord(a, st);
  for (int r = 0; r < reps; ++r) vofp_poisson_solve(p, p->P, p->P, st, nullptr);
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

}  // namespace

extern "C" int vofp_plan_tune(vofp_plan* p) {
  if (!p) return VOFP_ERR_INVALID_ARG;
  const std::string k = key_of(p);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file();
    auto it = g_cache.find(k);
    if (it != g_cache.end()) {
      if (fits(p, it->second)) apply(p, it->second);
      return VOFP_OK;
    }
  }
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return VOFP_ERR_CUDA;
  // a bounded, deterministic right-hand side: zeros (the kernels' cost does not depend on the values)
  cudaMemsetAsync(p->P, 0, sizeof(double) * (size_t)p->n[0] * p->n[1] * p->n[2], st);
  Shape best = current(p);
  float tbest = time_solve(p, st);
  const int xs[] = {1, 2, 4, 8, 16, 32};
  const int ys[] = {2, 4, 8, 16, 32};
  const int zs[] = {-1, -2, 0, 8, 16, 32, 64, 128};
  const int os[] = {0, 1, 2, 3};
  for (int knob = 0; knob < 4; ++knob) {
    const int* cand = knob == 0 ? xs : (knob == 1 ? ys : (knob == 2 ? zs : os));
    const int nc = knob == 0 ? 6 : (knob == 1 ? 5 : (knob == 2 ? 8 : 4));
    for (int c = 0; c < nc; ++c) {
      Shape s = best;
      if (knob == 0) s.xpb = cand[c];
      if (knob == 1) s.ytx = cand[c];
      if (knob == 2) s.zti = cand[c];
      if (knob == 3) s.ord = cand[c];
      if (!fits(p, s)) continue;
      apply(p, s);
      const float t = time_solve(p, st);
      if (t < tbest) {
        tbest = t;
        best = s;
      }
    }
    apply(p, best);
  }
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (cudaGetLastError() != cudaSuccess) return VOFP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[k] = best;
  save_entry(k, best);
  return VOFP_OK;
}
