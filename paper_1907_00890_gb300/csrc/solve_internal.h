// Host-side internal entry points shared between the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <vector>

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
  KID_BATCHED,
  KID_NOALLOC_TABLES,
  KID_ZLOW,     // refinement plans: the low-eigenvalue z systems in FP64
  KID_GAUGE,    // gauge restoration of p
  KID_VD,       // variable-density splitting: u* -= dt (1/rho_f - 1/rho0) G p_hat
  KID_VOF,      // volume-of-fluid update with the interface velocity
  KID_COUNT
};

struct TraceTok {
  int active;
  int kid;
  cudaEvent_t a, b;
};
void trace_begin(int kid, cudaStream_t st, TraceTok* tok);
void trace_end(TraceTok* tok, cudaStream_t st);

// Every device (and pinned host) block the library allocates goes through these: cudaMalloc /
// cudaMallocHost, or an injected failure (vofp_debug_fail_alloc).
cudaError_t device_alloc(void** p, size_t bytes);
cudaError_t pinned_alloc(void** p, size_t bytes);

// Count `n` kernel launches (read by vofp_launch_count).
void note_launches(int n);
// Graph capture on this thread: launches are counted apart and not traced; capture_end returns their number.
bool capturing();
void capture_begin();
unsigned long long capture_end();

// Launch a kernel with launch counting and optional tracing: VOFP_LAUNCH(kid, stream, kernel<<<...>>>(...)).
#define VOFP_LAUNCH(kid, st, ...)         \
  do {                                    \
    ::vofp::TraceTok _tk;                 \
    ::vofp::trace_begin((kid), (st), &_tk); \
    __VA_ARGS__;                          \
    ::vofp::trace_end(&_tk, (st));        \
    ::vofp::note_launches(1);             \
  } while (0)

// ---- plan construction in two phases (see plan.cu) ----
struct PlanLayout {
  size_t lam[2], tw[2], q[2], tw32[2], q32[2], twff[2], qff[2], blu64[2], blu32[2], bluff[2];
  size_t za, zb, zc, dz, hz, rdz, rhz, rzc, conv, info, low, za32, zaff, lowcut, kz, volf, dzff;
  size_t table_bytes;  // host-built part, uploaded as one copy
  size_t P, S, T, S32, F, lowscr, lowtab, xtc;
  size_t total;
};
struct PlanPrep {
  vofp_plan* p;
  std::vector<unsigned char> host;
  PlanLayout L;
};
int plan_prepare(int nx, int ny, int nz, double dx, double dy, const double* dz, const int bc[3],
                 const vofp_opts* opt, PlanPrep* pp);
int plan_bind(PlanPrep* pp, void* block, cudaStream_t st, unsigned char* stage);
size_t plan_prep_device_bytes(const PlanPrep* pp);
size_t plan_prep_stage_bytes(const PlanPrep* pp);
void plan_free_host(vofp_plan* p);
// Allocate the interface-geometry workspace (s, n) on first use.
int ensure_geometry(vofp_plan* p);
// Release the host-buffer step's device fields, streams and events (plan destruction).
void free_host_step(vofp_plan* p);

struct XArgs;
struct XInvArgs;
struct GridDev;
struct ZArgs;
GridDev grid_dev(const vofp_plan* pl);
ZArgs z_args(const vofp_plan* pl, bool stats);
struct ZTabArgs;
ZTabArgs ztab_args(const vofp_plan* pl);
int grid_blocks(size_t total, int threads);
void init_kernel_attributes_fp64();
void init_kernel_attributes_mixed();
// True the first time it is called for the current device (each kernel's shared-memory attribute is set
// once per device and process, not on every plan).
bool first_use_on_device(int which);
int fp64_solve(vofp_plan* pl, int mode, XArgs xa, double* pout, cudaStream_t st, bool stats);
// The FP64 plans' y pass on TMA-staged tiles when applicable (power-of-two ny; mixed.cu); false: not run.
struct YArgs;
bool ypass_tma_f64(vofp_plan* pl, const YArgs& ya, bool inv, cudaStream_t st);
// The plan's FP64 x transform (forward, or inverse) of nlines lines `in` -> `out` (see solve.cu).
int fp64_x_lines(vofp_plan* pl, bool inverse, const double* in, double* out, int nlines, cudaStream_t st);
// Tensor-core x passes of FP32 refinement plans (xtc.cu): table sizes at plan preparation, the tables' build
// at plan placement, and the passes themselves (false: not applicable, the caller runs the FFT pass).
size_t xtc_table_bytes(int nx, long nlines, int prec);
int xtc_build(vofp_plan* pl, void* tables, cudaStream_t st);
bool xtc_xfwd(vofp_plan* pl, int mode, const XArgs& xa, cudaStream_t st);
bool xtc_xinv(vofp_plan* pl, const XInvArgs& xi, cudaStream_t st);
// Mixed-precision solve: FP32 transforms with FP64 defect correction.  `xa` carries the right-hand-side
// inputs for RHS_DIV / RHS_DIV_STEFAN (NULL for RHS_F, which reads `f`).  Fills `info` (if non-NULL) and
// synchronises the stream in that case.
int mixed_solve(vofp_plan* pl, int mode, const XArgs* xa, const double* f, double* pout, cudaStream_t st,
                vofp_info* info);
int begin_info(vofp_plan* pl, cudaStream_t st, vofp_info* info);
// Thomas factor tables for a bounded z axis (in the plan's arithmetic type), built on `st`; `sync` waits.
int build_z_factors(vofp_plan* pl, cudaStream_t st, bool sync);
// The same for the low-eigenvalue systems of a mixed plan.
int build_low_factors(vofp_plan* pl, cudaStream_t st, bool sync);
int finish_info(vofp_plan* pl, cudaStream_t st, vofp_info* info, int status);
}  // namespace vofp

extern "C" int vofp_plan_tune(vofp_plan* plan);
