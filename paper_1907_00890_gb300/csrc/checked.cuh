// Bounds-checked build.
//
// Compiled with -DVOFP_CHECKED (the library libvofp_checked.so), each kernel tests the indices it derives from
// its launch coordinates -- the cell, face, line, column or table entry it is about to touch -- against the
// extent of that array before the access.  An index out of range skips the access (a load reads zero) and is
// recorded in a device word of its translation unit: the number of failed tests and the site, index and extent
// of the first.  Offsets along an axis inside a kernel run over that axis' loop bounds from a checked base.
// Nothing traps and nothing waits: a failed test leaves the kernel running to its normal end.  The host reads
// (and clears) the words of every translation unit through vofp_debug_check_word.  Without the flag every test
// is the constant true and the kernels compile to the same code as before.
//
// This stands in for a device memory checker: run the GPU parity tests against the checked library and
// require, besides the oracle's values, a zero count.
#pragma once

#include <cuda_runtime.h>

namespace vofp {

enum ChkSite {
  CHK_NONE = 0,
  CHK_CELL_LOAD = 1,    // cell-field loads of the stencils (right-hand side, residual, gradient of C)
  CHK_FACE_LOAD = 2,    // face-field loads of the divergence stencil
  CHK_XFWD_STORE = 3,   // x forward pass: spectrum and saved right-hand side
  CHK_Y_PASS = 4,       // y pass: spectrum loads and stores
  CHK_XINV = 5,         // x inverse pass: spectrum loads, potential stores
  CHK_Z_COLUMN = 6,     // z passes: (x, y) spectral column of a system
  CHK_Z_TABLE = 7,      // z passes: factor-table entry
  CHK_FACE_STORE = 8,   // face epilogues: face offset
  CHK_FACE_LINE = 9,    // face epilogues: the cell line a face gradient or face mean reads
  CHK_CELL_STORE = 10,  // per-cell outputs (interface geometry, VoF update)
  CHK_VOF_LOAD = 11,    // VoF update: face-velocity and cell loads
  CHK_Y_TMA = 12,       // TMA y pass: spectrum stores
  CHK_X_TMA = 13,       // TMA x inverse pass: potential stores
  CHK_XTC = 14,         // tensor-core x passes: spectrum / potential
  CHK_BATCH = 15,       // batched launches: block -> instance mapping
  CHK_SELFTEST = 99,    // vofp_debug_check_selftest
};

#ifdef VOFP_CHECKED

struct ChkWord {
  unsigned long long count;
  long long site, index, extent;
};
static __device__ ChkWord g_chk;

__device__ __noinline__ static bool chk_fail(int site, long long index, long long extent) {
  if (atomicAdd(&g_chk.count, 1ull) == 0ull) {
    g_chk.site = site;
    g_chk.index = index;
    g_chk.extent = extent;
  }
  return false;
}

// true when 0 <= idx < ext; otherwise records the failure and returns false
#define VOFP_IN(idx, ext, site)                                                        \
  (((unsigned long long)(long long)(idx) < (unsigned long long)(long long)(ext)) || \
   ::vofp::chk_fail((site), (long long)(idx), (long long)(ext)))

template <typename T>
__device__ __forceinline__ T ldg_in(const T* p, size_t i, size_t ext, int site) {
  return VOFP_IN(i, ext, site) ? __ldg(p + i) : T(0);
}

// host side: every translation unit registers a reader of its own word (trace.cu keeps the list)
int chk_register(int (*read)(long long* out, int reset));
static int chk_read_tu(long long* out, int reset) {
  ChkWord w;
  if (cudaMemcpyFromSymbol(&w, g_chk, sizeof(w)) != cudaSuccess) return -1;
  out[0] = (long long)w.count;
  out[1] = w.site;
  out[2] = w.index;
  out[3] = w.extent;
  if (reset) {
    const ChkWord z = {0ull, 0, 0, 0};
    if (cudaMemcpyToSymbol(g_chk, &z, sizeof(z)) != cudaSuccess) return -1;
  }
  return 0;
}
[[maybe_unused]] static const int g_chk_registered = chk_register(&chk_read_tu);

#else

#define VOFP_IN(idx, ext, site) true

template <typename T>
__device__ __forceinline__ T ldg_in(const T* p, size_t i, size_t, int) {
  return __ldg(p + i);
}

#endif

}  // namespace vofp
