// Host-side internal entry points shared between the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "vofp_internal.cuh"

namespace vofp {

// Kernel classes for tracing.
enum KernelId {
  KID_XFWD = 0,       // x pass, right-hand side given
  KID_XFWD_DIV,       // x pass fused with the divergence (+ optional source array)
  KID_XFWD_STEFAN,    // x pass fused with the Stefan source
  KID_XFWD_DIVSTEF,   // x pass fused with divergence and Stefan source
  KID_YFWD,
  KID_ZSOLVE,
  KID_YINV,
  KID_XINV,
  KID_GRAD,
  KID_EXTEND_EPI,
  KID_STEFAN,
  KID_RESID,
  KID_FUSED_YZY,
  KID_BATCHED,
  KID_NOALLOC_TABLES,
  KID_COUNT
};

struct TraceTok {
  int active;
  int kid;
  cudaEvent_t a, b;
};
void trace_begin(int kid, cudaStream_t st, TraceTok* tok);
void trace_end(TraceTok* tok, cudaStream_t st);

// Count `n` kernel launches (read by vofp_launch_count).
void note_launches(int n);

// Launch a kernel with launch counting and optional tracing: VOFP_LAUNCH(kid, stream, kernel<<<...>>>(...)).
#define VOFP_LAUNCH(kid, st, ...)         \
  do {                                    \
    ::vofp::TraceTok _tk;                 \
    ::vofp::trace_begin((kid), (st), &_tk); \
    __VA_ARGS__;                          \
    ::vofp::trace_end(&_tk, (st));        \
    ::vofp::note_launches(1);             \
  } while (0)

struct XArgs;
struct GridDev;
GridDev grid_dev(const vofp_plan* pl);
int grid_blocks(size_t total, int threads);
void init_kernel_attributes_fp64();
void init_kernel_attributes_mixed();
int fp64_solve(vofp_plan* pl, int mode, XArgs xa, double* pout, cudaStream_t st, bool stats);
// Mixed-precision solve: FP32 transforms with FP64 defect correction.  `xa` carries the right-hand-side
// inputs for RHS_DIV / RHS_STEFAN (NULL for RHS_F, which reads `f`).  Fills `info` (if non-NULL) and
// synchronises the stream in that case.
int mixed_solve(vofp_plan* pl, int mode, const XArgs* xa, const double* f, double* pout, cudaStream_t st,
                vofp_info* info);
int begin_info(vofp_plan* pl, cudaStream_t st, vofp_info* info);
int finish_info(vofp_plan* pl, cudaStream_t st, vofp_info* info, int status);
}  // namespace vofp
