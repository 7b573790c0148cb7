/*
 * vofp.h -- C ABI of the GB300 FFT-based Poisson projection library.
 *
 * The library implements the pressure-projection and liquid-velocity-extension solves of the two-fluid
 * evaporating-flow VoF method of Scapin, Costa & Brandt (arXiv 1907.00890):
 *
 *   - the constant-coefficient Poisson equation of the pressure-splitting projection (§3.2, Eq. lap_p,
 *     constant-density part) and the velocity correction that follows it;
 *   - the Stefan-flow potential lap(phi) = mdot (1/rho2 - 1/rho1) |grad C| (§3.6, Eq. ext_div), the
 *     divergence-free liquid extension u1e = u - grad(phi) (Eq. jump_subtr) and the interface velocity
 *     uG = u1e - (mdot/rho1) n (Eq. int_vel);
 *   - the full variable-density pressure step of Eq. lap_p (the pressure-splitting term with the
 *     extrapolated pressure, vofp_project_vd) and the boiling variant of the interface velocity (Appendix A,
 *     vofp_extend_vapour_velocity);
 *   - the volume-fraction update that the interface velocity drives (§3.1, Eqs. fluxes and final_corr_2,
 *     vofp_vof_update).
 *
 * Both Poisson equations are solved exactly (direct solver, §3.2) on a uniform-in-x,y MAC grid: real-to-real
 * transforms in x and y (periodic: DFT; Neumann: DCT-II; Dirichlet: DST-II; mixed: DCT-IV / DST-IV), one
 * tridiagonal system in z per (x, y) wavenumber pair, inverse transforms, gradient correction.  All kernels
 * are hand-written CUDA for sm_103a.
 *
 * GRID AND LAYOUT (all arrays C-ordered [z][y][x], x fastest, FP64):
 *   cell arrays (p, f, src, C, mdot, phi): nz * ny * nx values.
 *   face arrays: index i along the face's own axis is the LOW face of cell i.  A periodic axis stores n
 *   faces, a bounded axis n + 1 (both boundary faces):
 *     u: nz * ny * (nx + (bc[0] != VOFP_BC_P)),  v: nz * (ny + (bc[1] != VOFP_BC_P)) * nx,
 *     w: (nz + (bc[2] != VOFP_BC_P)) * ny * nx.
 *   Boundary conditions are homogeneous, per axis (§3.2: several combinations of homogeneous pressure
 *   boundary conditions; §3.6: phi takes the pressure's).  N = zero normal gradient at the boundary face
 *   (the face velocity there is an input the projection leaves unchanged); D = zero value at the boundary
 *   face (ghost value -p).  ND / DN (N at the low end, D at the high end, and the reverse) are accepted on
 *   every axis: on x and y they make the transform a DCT-IV / DST-IV.
 *   When no axis has a D end the operator is singular: the volume-weighted mean of the right-hand side is
 *   removed (reported as compat_defect) and the returned potential has zero volume-weighted mean.
 *
 * OWNERSHIP AND STREAMS: the caller owns every field pointer (device memory).  The plan owns its tables
 * and workspace; vofp_plan_destroy frees them.  Calls are asynchronous on the given stream (a
 * cudaStream_t passed as void*, NULL = legacy default stream) unless `info` is non-NULL, in which case the
 * call synchronises that stream to fill it.  One plan may be used by one stream at a time (its workspace is
 * shared by its calls).
 *
 * ERRORS: every int-returning call returns 0 on success, > 0 for a warning, < 0 for an error; nothing is
 * launched when an argument check fails.  vofp_error_string() gives the message.
 */
#ifndef VOFP_H
#define VOFP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define VOFP_OK 0
#define VOFP_WARN_INCOMPATIBLE_RHS 1 /* singular operator and |mean(f)| > 1e-12 * mean(|f|)            */
#define VOFP_WARN_NOT_CONVERGED 2    /* mixed precision: refinement stopped at max_refine              */
#define VOFP_ERR_INVALID_ARG -1
#define VOFP_ERR_UNSUPPORTED -2
#define VOFP_ERR_OOM -3
#define VOFP_ERR_CUDA -4
#define VOFP_ERR_TIMEOUT -5
#define VOFP_ERR_BUSY -6
#define VOFP_ERR_NONFINITE -7

/* boundary condition per axis (first letter = low end, second = high end) */
typedef enum { VOFP_BC_P = 0, VOFP_BC_NN = 1, VOFP_BC_DD = 2, VOFP_BC_ND = 3, VOFP_BC_DN = 4 } vofp_bc;

/* arithmetic of the solve */
typedef enum {
  VOFP_FP64 = 0,  /* every step in FP64                                                              */
  VOFP_MIXED = 1, /* FP32 transforms, FP64 low modes / reductions / residual, defect-correction refinement */
  VOFP_FF = 2     /* as VOFP_MIXED, but the transforms and z recurrences in FP32-pair (float-float)
                     arithmetic (~1e-14 relative) on the FP32 pipe: the first solve is already within
                     ~1e-13 and one correction confirms it; max_refine = 0 skips the confirmation        */
} vofp_prec;

typedef struct {
  int prec;       /* vofp_prec                                                                  */
  double tol;     /* mixed: stop when ||f - L p|| / ||f|| <= tol (default 1e-10)                   */
  int max_refine; /* mixed: maximum defect-correction iterations (default 3)                       */
  int grad_mode;  /* |grad C| and n: 0 = central differences (default), 1 = Youngs corner average    */
  int tune;       /* 0 = default launch shapes, 1 = autotuned (cached per shape)                    */
} vofp_opts;

typedef struct {
  double compat_defect; /* volume-weighted mean removed from the right-hand side (0 if L regular)     */
  double mean_removed;  /* volume-weighted mean subtracted from the potential to restore the zero-mean
                           gauge (FP32 spectra; 0 where the pinned mean mode keeps the gauge exactly)   */
  double rel_residual;  /* refinement plans: ||f - fbar - L p||_2 / ||f||_2 of the returned p (FP64
                           stencil); FP64 plans: not computed (0)                                       */
  double err_estimate;  /* estimated relative 2-norm error of p against the exact solution of the
                           discrete system.  Refinement plans (VOFP_MIXED, VOFP_FF): a posteriori -- the
                           FP64 residual of the returned p is solved once more in the plan's precision and
                           the size of that correction (not applied) relative to p is reported.  FP64
                           plans: -1, not estimated (an FP64 plan keeps no copy of the right-hand side;
                           an a-priori bound cond(L) * 2^-53 is vacuous on stretched grids, where cond(L)
                           reaches 1e13)                                                               */
  int refine_iters;     /* refinement plans: defect-correction iterations performed                     */
  int status;           /* same as the return value                                                     */
} vofp_info;

typedef struct vofp_plan vofp_plan;

/* Fill `opt` with the defaults (FP64, tol 1e-10, max_refine 3, central gradients, no tuning). */
void vofp_opts_default(vofp_opts* opt);

/*
 * Create a plan for an nx x ny x nz grid (each >= 1) with uniform spacings dx, dy > 0 and z cell widths
 * dz[0..nz-1] > 0 (HOST pointer, copied), boundary conditions bc[3] (x, y, z; each P, NN, DD, ND or DN),
 * options `opt` (NULL = defaults).  Builds the eigenvalue, twiddle and z-coefficient tables on the current CUDA
 * device and allocates the workspace.  §3 (grid), §3.2 (solver, boundary conditions).
 * Errors: INVALID_ARG (sizes, spacings, bc), UNSUPPORTED (an axis above 4096 cells, or above 2^31 - 1
 * cells in all), OOM, CUDA.
 */
int vofp_plan_create(int nx, int ny, int nz, double dx, double dy, const double* dz, const int bc[3],
                     const vofp_opts* opt, vofp_plan** out);

/*
 * Autotune the plan's launch shapes (line pairs per x block, columns per y block, the z kernel -- segmented
 * tiles, staged or streamed chains and their systems per block) and the order of the FFT radix stages on x
 * and y, by timing whole solves on the plan's scratch workspace (coordinate descent over the candidates that
 * fit in shared memory).  Results are cached per process and, if the environment variable VOFP_TUNE_CACHE names a
 * file, across processes.  Called by vofp_plan_create when opts.tune != 0.  Synchronises the device.
 * No counterpart in the paper (performance only; results stay within the parity tolerance).
 * Errors: INVALID_ARG, CUDA.
 */
int vofp_plan_tune(vofp_plan* plan);

/* Free the plan's device tables and workspace (NULL is ignored).  Synchronises the device first. */
void vofp_plan_destroy(vofp_plan* plan);

/* Device bytes held by the plan (tables + workspace). */
size_t vofp_plan_workspace_bytes(const vofp_plan* plan);

/*
 * Solve L p = f - fbar (§3.2, Eq. lap_p left-hand side; §3.6 Eq. ext_div).  f, p: device cell arrays
 * (may alias).  Errors: INVALID_ARG (NULL plan/pointers), CUDA, NONFINITE (only detected when info != NULL).
 */
int vofp_poisson_solve(vofp_plan* plan, const double* f, double* p, void* stream, vofp_info* info);

/*
 * Pressure projection (§3.2, Eq. lap_p with constant density and the correction step after it):
 *   f = (D u* - src) / dt_over_rho0,  L p = f - fbar,  u = u* - dt_over_rho0 G p   (u, v, w in place).
 * src: device cell array or NULL (no phase-change source).  p: device cell array or NULL (not returned).
 * dt_over_rho0 > 0.  Errors: INVALID_ARG, CUDA, NONFINITE (only with info).
 */
int vofp_project(vofp_plan* plan, double* u, double* v, double* w, const double* src, double dt_over_rho0,
                 double* p, void* stream, vofp_info* info);

/*
 * Pressure step with the variable-density pressure splitting of §3.2 (Eq. lap_p in full and the velocity
 * update after it):
 *   p_hat = (1 + dt/dt_prev) p^n - (dt/dt_prev) p^{n-1}   (p^n alone when p_nm1 is NULL),
 *   rho = rho1 C + rho2 (1 - C)  (Eq. material_prop),  rho0 = min(rho1, rho2),
 *   L p / rho0 = D[(1/rho0 - 1/rho_f) G p_hat] + (D u* - src) / dt,
 *   u = u* - dt [ (1/rho0) G p + (1/rho_f - 1/rho0) G p_hat ],
 * with rho_f on a face the mean of rho over its two cells (its one cell at a bounded end; no flux through an
 * N face).  Computed as one face pass u** = u* - dt (1/rho_f - 1/rho0) G p_hat followed by vofp_project(u**,
 * src, dt/rho0, p): the constant-coefficient solve the splitting exists for.
 * u, v, w: device face arrays, u* in, u^{n+1} out.  src: device cell array or NULL.  C, p_n: device cell
 * arrays (required); p_nm1: device cell array or NULL.  dt > 0; dt_prev > 0 when p_nm1 is given; rho1, rho2 > 0.
 * p: device cell array or NULL (p^{n+1}; may be the p_n buffer).  Errors: INVALID_ARG, CUDA, NONFINITE (only
 * with info).
 */
int vofp_project_vd(vofp_plan* plan, double* u, double* v, double* w, const double* src, const double* C,
                    const double* p_n, const double* p_nm1, double dt, double dt_prev, double rho1, double rho2,
                    double* p, void* stream, vofp_info* info);

/*
 * Liquid-velocity extension and interface velocity (§3.6):
 *   s = mdot (1/rho2 - 1/rho1) |grad C|  (Eq. ext_div),  L phi = s - sbar,
 *   u1e = u - G phi  (Eq. jump_subtr),
 *   uG = u1e - (mdot_f / rho1) n_f  (Eq. int_vel), n = -grad C / |grad C| (pointing into the gas, Eq.
 *   rankine), n = 0 where min(C, 1 - C) < 1e-8; face values of mdot and n are means of the two adjacent
 *   cells (the one adjacent cell on a boundary face).
 * u, v, w: device face arrays (input, not modified).  C, mdot: device cell arrays.  rho1, rho2 > 0.
 * ue, ve, we: device face arrays (output, required).  ug, vg, wg: output or all three NULL.  phi: device
 * cell array or NULL.  Errors: INVALID_ARG, CUDA, NONFINITE (only with info).
 */
int vofp_extend_liquid_velocity(vofp_plan* plan, const double* u, const double* v, const double* w,
                                const double* C, const double* mdot, double rho1, double rho2, double* ue,
                                double* ve, double* we, double* ug, double* vg, double* wg, double* phi,
                                void* stream, vofp_info* info);

/*
 * The boiling variant (Appendix A): the interface velocity from a divergence-free extension of the vapour
 * (phase 2) velocity.  Exchanging the phases in §3.6 leaves the Stefan potential phi and u - G phi unchanged,
 * so u2e = u - G phi as in vofp_extend_liquid_velocity and uG = u2e - (mdot_f / rho2) n_f (Eq. rankine on the
 * vapour side; n still points into phase 2).  Arguments, outputs and errors as vofp_extend_liquid_velocity.
 */
int vofp_extend_vapour_velocity(vofp_plan* plan, const double* u, const double* v, const double* w,
                                const double* C, const double* mdot, double rho1, double rho2, double* ue,
                                double* ve, double* we, double* ug, double* vg, double* wg, double* phi,
                                void* stream, vofp_info* info);

/*
 * Volume-of-fluid update with the interface velocity uG (§3.1): the directional split of Eq. fluxes (x, y, z,
 * each step implicit in its own result), then the correction with the implicit volume deflation of Eq.
 * final_corr_2, C^{n+1} (1 - dt div uG) = C*** - dt (C* du/dx + C** dv/dy + C*** dw/dz).  The numerical
 * fluxes are first-order upwind ones (the paper takes MTHINC fluxes from its reference; beyond a bounded end
 * the boundary cell is used).  C: device cell array (input); uG, vG, wG: device face arrays; dt > 0 (the
 * implicit factors 1 - dt du/dx etc. must stay positive: a Courant condition); C_out: device cell array
 * (may be C); work: device workspace of 2 * nx * ny * nz doubles, disjoint from C and C_out (used only when
 * C_out is C: the result is formed there and copied back).  One FP64 pass marching through the z planes.
 * Errors: INVALID_ARG, CUDA.
 */
int vofp_vof_update(vofp_plan* plan, const double* C, const double* uG, const double* vG, const double* wG,
                    double dt, double* C_out, double* work, void* stream);

/*
 * Stefan source s = mdot (1/rho2 - 1/rho1) |grad C| at cell centres (§3.2 last term of Eq. lap_p with the
 * regularised delta |grad C|; §3.6 Eq. ext_div right-hand side), |grad C| per opts.grad_mode.
 * C, mdot: device cell arrays; s: device cell array (output).  Errors: INVALID_ARG, CUDA.
 */
int vofp_stefan_source(vofp_plan* plan, const double* C, const double* mdot, double rho1, double rho2, double* s,
                       void* stream);

/*
 * Pressure projection whose phase-change source is the Stefan source of (C, mdot, rho1, rho2), computed
 * inside the divergence pass (same result as vofp_stefan_source followed by vofp_project with that src):
 *   f = (D u* - mdot (1/rho2 - 1/rho1) |grad C|) / dt_over_rho0   (Eq. lap_p, constant-density part).
 * Arguments as vofp_project plus the source inputs.  Errors: INVALID_ARG, CUDA, NONFINITE (only with info).
 */
int vofp_project_stefan(vofp_plan* plan, double* u, double* v, double* w, const double* C, const double* mdot,
                        double rho1, double rho2, double dt_over_rho0, double* p, void* stream, vofp_info* info);

/*
 * Both Poisson solves of one time step of the paper's solver (§3.7: the pressure correction, then the
 * interface-velocity construction of §3.6), sharing one interface-geometry pass (|grad C| and n computed once
 * per cell): the projection of vofp_project_stefan (u, v, w in place, p optional) followed by the extension
 * of vofp_extend_liquid_velocity applied to the projected velocity (ue, ve, we required; ug, vg, wg all or
 * none; phi optional).  Same results as calling the two entry points in that order.
 * Errors: INVALID_ARG, CUDA, NONFINITE (only with info; info reports the worse status of the two solves).
 */
int vofp_project_extend(vofp_plan* plan, double* u, double* v, double* w, const double* C, const double* mdot,
                        double rho1, double rho2, double dt_over_rho0, double* p, double* ue, double* ve,
                        double* we, double* ug, double* vg, double* wg, double* phi, void* stream,
                        vofp_info* info);

/*
 * The same time step (vofp_project_extend) on HOST buffers -- the call of a host code that keeps its fields
 * in host memory.  Inputs u, v, w (faces), C, mdot (cells) are copied to device fields owned by the plan
 * (allocated on its first host step), results are copied back: the projected u_out, v_out, w_out, the
 * pressure p_out and the interface velocity ug, vg, wg (layouts as on the device).  The copies run on two
 * streams of the plan and overlap the compute on `stream`: C and mdot go first and the geometry pass starts
 * while the velocities are still arriving; the projected fields leave while the extension solve runs.  The
 * call is asynchronous: `stream` completes after the last result has arrived, so the host buffers must stay
 * valid until then (pinned host memory makes the copies asynchronous; pageable memory works but serialises
 * them).  Errors: INVALID_ARG, OOM (device fields), CUDA.
 */
int vofp_project_extend_host(vofp_plan* plan, const double* u, const double* v, const double* w, const double* C,
                             const double* mdot, double rho1, double rho2, double dt_over_rho0, double* u_out,
                             double* v_out, double* w_out, double* p_out, double* ug, double* vg, double* wg,
                             void* stream);

/*
 * Batched projection of independent instances (an ensemble of droplet runs with uneven grids; the paper's
 * solver runs one instance, so this is the data-parallel form of vofp_project).  plans[0..n-1]: distinct
 * VOFP_MIXED plans on one device (each plan's workspace serves exactly one instance).  Every pass of the
 * mixed-precision projection runs as one launch over all instances and the whole sequence is captured once
 * into a CUDA graph and replayed per call.  Each instance runs the same kernels on the same data as in a batch
 * of one, so its result agrees with running it alone to rounding (1e-12 in the tests) -- not bit for bit: the
 * FP64 block partials of its norms and means are added with atomics, in an order that varies between runs.
 * Errors: INVALID_ARG (NULL, n < 1, repeated plan, mixed devices), UNSUPPORTED (an FP64 plan), OOM.
 */
typedef struct vofp_batch vofp_batch;
int vofp_batch_create(vofp_plan* const* plans, int n, vofp_batch** out);
/*
 * Project every instance i (vofp_project semantics): u[i], v[i], w[i] device face arrays in place;
 * src[i] device cell array or NULL (src itself may be NULL); dt_over_rho0[i] > 0 (HOST array);
 * p[i] device cell array or NULL (p itself may be NULL).  Asynchronous on `stream`.  The argument records
 * are re-uploaded only when a pointer or dt_over_rho0 changes (the call then waits for `stream`).
 */
int vofp_batch_project(vofp_batch* b, double* const* u, double* const* v, double* const* w,
                       const double* const* src, const double* dt_over_rho0, double* const* p, void* stream);
int vofp_batch_size(const vofp_batch* b);
void vofp_batch_destroy(vofp_batch* b);

/*
 * Serving (continuous batching of projection requests from an ensemble of independent runs; the paper
 * solves one run, so this is a deployment form of vofp_project).
 *
 * vofp_server_create: `mem_budget_bytes` of device memory (0 = half of the free memory) become the server's
 * arena, allocated once; `max_inflight` (1..256) requests may be on the GPU at once, each on its own stream;
 * `opt` (NULL = defaults) is the plan options of every request (precision, tolerance).
 * A request names its grid (n, dx, dy, dz HOST array copied at submission, bc) and its device fields
 * (u, v, w in place; src and p optional; dt_over_rho0 > 0); the caller keeps the fields valid and untouched
 * until the request completes.  vofp_server_submit returns at once with a ticket.  A worker thread admits
 * pending requests oldest first whenever a slot and an arena block of the plan's size are free (requests
 * arriving while others run are admitted as those complete), builds each plan in its arena block and runs
 * the projection asynchronously; no device memory is allocated or freed while serving.  A request whose
 * plan alone exceeds the arena completes with VOFP_ERR_BUSY.
 * Latency runs from the request's ARRIVAL to its completion: arrival_s is the time the request arrived on the
 * server clock (seconds since vofp_server_create, read with vofp_server_clock), so a request that waited on
 * the caller's side before it could be submitted is charged for that wait; arrival_s <= 0 (or later than the
 * submission) means the submission time.
 * vofp_server_poll: 0 = done (the ticket is consumed; *latency_s = completion - arrival), 1 = pending,
 * < 0 = the request's error (also consumes the ticket).  vofp_server_wait: the same, blocking up to
 * timeout_s (VOFP_ERR_TIMEOUT, ticket kept).  vofp_server_stats: out[0..VOFP_SERVER_STATS-1] (the first n are
 * written) = completed, admitted, rejected, queued (submitted, not yet admitted), arena bytes in use, arena
 * bytes, p50 and p99 latency (s, arrival -> completion), cells solved, seconds since creation or the last
 * reset, worker seconds spent building plans, worker seconds spent enqueuing work, worker loop iterations,
 * requests served by a resident plan, requests that needed a new plan, plans evicted, resident plans, p99 wait
 * from arrival to submission (s), p99 wait from submission to the launch of its work (s) (reset != 0 clears
 * the counters).  Plans
 * stay resident in the arena after their request and serve later requests of the same grid, spacings and
 * boundary conditions; idle ones are evicted, least recently used first, when a new plan needs the space.
 * vofp_server_destroy waits for in-flight work.
 */
typedef struct {
  int n[3];
  double dx, dy;
  const double* dz;
  int bc[3];
  double* u;
  double* v;
  double* w;
  const double* src;
  double dt_over_rho0;
  double* p;
  double arrival_s; /* arrival time on the server clock (vofp_server_clock); <= 0: the submission time */
} vofp_request;
#define VOFP_SERVER_STATS 19
typedef struct vofp_server vofp_server;
int vofp_server_create(size_t mem_budget_bytes, int max_inflight, const vofp_opts* opt, vofp_server** out);
int vofp_server_submit(vofp_server* s, const vofp_request* r, unsigned long long* ticket);
int vofp_server_poll(vofp_server* s, unsigned long long ticket, vofp_info* info, double* latency_s);
int vofp_server_wait(vofp_server* s, unsigned long long ticket, double timeout_s, vofp_info* info,
                     double* latency_s);
int vofp_server_stats(vofp_server* s, double* out, int n, int reset);
/* Seconds since the server's creation on its steady clock (the clock of vofp_request.arrival_s). */
int vofp_server_clock(vofp_server* s, double* seconds);
void vofp_server_destroy(vofp_server* s);

/*
 * Allocation-free FP64 Poisson solve (the paper has no counterpart; it is a deployment variant of
 * vofp_poisson_solve).  For callers that cannot call cudaMalloc when they need a solve -- e.g. a host code
 * whose device memory is handed out entirely by its own pool allocator at start-up, or a time-stepping loop
 * that must not pay cudaMalloc's implicit device synchronisation -- it takes no plan and allocates nothing:
 * its workspace and tables live in one fixed file-scope device array of the library, sized for at most
 * VOFP_NOALLOC_MAX_CELLS cells with no axis longer than VOFP_NOALLOC_MAX_N (about 16.3 MiB, held by every
 * GPU that loads the library until the process exits).
 *   Arguments: grid as vofp_plan_create (dz is a HOST array of nz widths, read during the call and passed to the kernels by value: it
 *   may be freed as soon as the call returns), f and p
 *   device cell arrays (may alias), stream as elsewhere.  Result identical (to rounding) to
 *   vofp_poisson_solve with a default FP64 plan.
 *   The first call on each device looks up the array's device address with that device current; make that
 *   first call before any stream capture.  All calls share the one array, which keeps the last call's
 *   contents (each call rebuilds what it reads): calls that overlap on the GPU race.
 *   Errors: INVALID_ARG, UNSUPPORTED (ND/DN on x or y), TOO_LARGE (beyond the limits above), CUDA.
 */
#define VOFP_ERR_TOO_LARGE -8
#define VOFP_NOALLOC_MAX_CELLS 2097152
#define VOFP_NOALLOC_MAX_N 1024
int vofp_poisson_solve_noalloc(int nx, int ny, int nz, double dx, double dy, const double* dz, const int bc[3],
                               const double* f, double* p, void* stream);

/* Number of kernels this library has launched in this process (all plans, all devices); diagnostics. */
unsigned long long vofp_launch_count(void);

/*
 * Kernel tracing (diagnostics; the paper has no counterpart).  While enabled, every launch is bracketed by
 * two CUDA events recorded on its stream.  vofp_trace_enable returns the previous state.
 * vofp_trace_collect waits for the recorded events, writes the summed device milliseconds and the launch
 * count of kernel class i to ms[i], count[i] for i < n (classes: vofp_trace_kernel_classes(), names:
 * vofp_trace_name(i)) and clears the record.  Errors: INVALID_ARG (NULL or n <= 0), CUDA.
 */
int vofp_trace_enable(int on);
int vofp_trace_collect(double* ms, unsigned long long* count, int n);
int vofp_trace_kernel_classes(void);
const char* vofp_trace_name(int id);

/*
 * Allocation-failure injection (diagnostics and tests of the out-of-memory paths; the paper has no
 * counterpart).  after >= 0: the next `after` device or pinned-host allocations of the library succeed and
 * the one after them fails once (the call that needed it returns VOFP_ERR_OOM and frees what it had taken);
 * after < 0 switches the injection off.  Process-wide.  Returns VOFP_OK.
 */
int vofp_debug_fail_alloc(long long after);

/*
 * Bounds-checked build (libvofp_checked.so, compiled with -DVOFP_CHECKED; a stand-in for a device memory
 * checker, no counterpart in the paper).  Its kernels test the index of each guarded global-memory access
 * against the array's extent; an index out of range skips the access and is counted, nothing traps.
 * vofp_debug_check_word synchronises the current device and reads the counts of all the library's
 * translation units: out[0] = number of failed tests, out[1] = site of the first (1 cell loads of the
 * stencils, 2 face loads, 3 x forward stores, 4 y pass, 5 x inverse, 6 z column, 7 z factor table, 8 face
 * stores, 9 face-gradient lines, 10 per-cell stores, 11 VoF loads, 12 TMA y pass, 13 TMA x inverse,
 * 14 tensor-core x passes, 15 batch block mapping, 99 self-test), out[2] its index, out[3] the extent;
 * reset != 0 clears the counts.  Returns 1 from the checked library, 0 from the plain one (out zeroed, no
 * device call), VOFP_ERR_CUDA if a read fails, VOFP_ERR_INVALID_ARG for out NULL.
 * vofp_debug_check_selftest launches, on `stream`, one test that fails by construction (index 5 against
 * extent 4, without an access): the checked library records it under site 99; the plain one does nothing.
 */
int vofp_debug_check_word(long long* out, int reset);
int vofp_debug_check_selftest(void* stream);

/* Static message for a status code. */
const char* vofp_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* VOFP_H */
