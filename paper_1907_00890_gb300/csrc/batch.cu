// Batched execution of independent projection instances (an ensemble of droplet runs with uneven grids).
//
// Every pass of the mixed-precision projection runs as ONE launch over all instances: the launch's blocks
// are partitioned among the instances by a prefix table (each instance keeps its own grid, boundary
// conditions, tables, launch shapes and convergence state), so small grids share the 152 SMs instead of
// queueing one after another.  The whole sequence -- initial FP32 solve, the defect-correction iterations
// with their device-side convergence tests, the gauge restoration and the velocity correction -- is captured
// once into a CUDA graph and replayed per call; a call only refreshes the per-instance argument records
// when the field pointers change.  Instances are independent and no kernel choice of one depends on the
// others, so an instance runs the same arithmetic alone and in any batch; its results agree to rounding, not
// bit for bit, because the FP64 block partials of its norms and means are added with atomics in an order
// that varies from run to run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "epilogue.cuh"
#include "passes.cuh"
#include "solve_internal.h"
#include "zsolve.cuh"

namespace vofp {

__device__ __forceinline__ int find_instance(const int* __restrict__ off, int n, int b) {
  int lo = 0, hi = n;  // off[lo] <= b < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= b) lo = mid;
    else hi = mid;
  }
  // (bounds-checked builds: the block lies in its instance's range; recorded, the accesses are checked on)
  (void)VOFP_IN(b - __ldg(off + lo), __ldg(off + lo + 1) - __ldg(off + lo), CHK_BATCH);
  return lo;
}

template <typename T, typename C, int MODE>
__global__ void __launch_bounds__(256) k_xfwd_batch(const XArgs* __restrict__ args, const int* __restrict__ off,
                                                     int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int i = find_instance(off, n, blockIdx.x);
  xfwd_block<T, C, MODE>(args[i], blockIdx.x - __ldg(off + i), smem_raw, red);
}

template <typename T, typename C, bool INV>
__global__ void __launch_bounds__(256) k_ypass_batch(const YArgs* __restrict__ args, const int* __restrict__ off,
                                                      int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = find_instance(off, n, blockIdx.x);
  const YArgs& a = args[i];
  const int l = blockIdx.x - __ldg(off + i);
  const int gx = (a.nx + a.tx - 1) / a.tx;
  ypass_block<T, C, INV>(a, l % gx, l / gx, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(128) k_zsolve_batch(const ZArgs* __restrict__ args, const int* __restrict__ off,
                                                      int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = find_instance(off, n, blockIdx.x);
  const ZArgs& a = args[i];
  const int l = blockIdx.x - __ldg(off + i);
  const int gx = (a.nx + a.ti - 1) / a.ti;
  zsolve_block<T, T>(a, l % gx, l / gx, smem_raw);
}

// Per-instance z records: the low-eigenvalue systems and (bounded z) the factor-table arguments.
struct LowArgs {
  const int2* modes;
  int nlow;
  const double2* tab;
  double* scratch;
  ZTabArgs zt;
  int smem_d;  // factor-table kernel: forward values in shared memory
};

// low-eigenvalue systems of all instances, periodic z: thread t of the flattened list
template <typename T>
__global__ void k_zlow_batch(const ZArgs* __restrict__ args, const LowArgs* __restrict__ low,
                             const int* __restrict__ off, int n, int total) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int i = find_instance(off, n, t);
  const ZArgs& a = args[i];
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const int q = t - __ldg(off + i);
  const LowArgs& L = low[i];
  zlow_system<T>(a, L.modes[q], q, L.nlow, L.tab, L.scratch);
}

// Bounded z: factor-table systems of all instances, 128 per block (one per thread).
template <typename T, typename TT>
__global__ void __launch_bounds__(128) k_ztab_batch(const ZArgs* __restrict__ args, const LowArgs* __restrict__ inst,
                                                    const int* __restrict__ off, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = find_instance(off, n, blockIdx.x);
  const ZArgs& a = args[i];
  const LowArgs& L = inst[i];
  const int l = blockIdx.x - __ldg(off + i);
  const int gx = (a.nx + 127) / 128;
  ztab_block<T, TT>(a, L.zt, L.smem_d, l % gx, l / gx, smem_raw);
}

// Bounded z, every instance's tile fitting: segmented tiles of 32 systems (kZSegW warps per block).
template <typename T, typename TT, bool LEAN>
__global__ void __launch_bounds__(256) k_ztab_seg_batch(const ZArgs* __restrict__ args,
                                                        const LowArgs* __restrict__ inst,
                                                        const int* __restrict__ off, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = find_instance(off, n, blockIdx.x);
  const ZArgs& a = args[i];
  const LowArgs& L = inst[i];
  const int l = blockIdx.x - __ldg(off + i);
  const int gx = (a.nx + kZSegTI - 1) / kZSegTI;
  ztab_seg_block<T, TT, LEAN>(a, L.zt, l % gx, l / gx, smem_raw);
}

// Bounded z: low-eigenvalue systems of all instances, one warp each.
template <typename T>
__global__ void __launch_bounds__(128) k_zlow_scan_batch(const ZArgs* __restrict__ args,
                                                         const LowArgs* __restrict__ low, const int* __restrict__ off,
                                                         int n, int total) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= total) return;  // uniform per warp
  const int i = find_instance(off, n, w);
  const ZArgs& a = args[i];
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const int q = w - __ldg(off + i);
  const LowArgs& L = low[i];
  zlow_scan_system<T>(a, L.modes[q], q, L.nlow, L.tab, L.scratch, threadIdx.x & 31);
}

template <typename T, typename C>
__global__ void __launch_bounds__(256) k_xinv_batch(const XInvArgs* __restrict__ args, const int* __restrict__ off,
                                                     int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int i = find_instance(off, n, blockIdx.x);
  xinv_block<T, C>(args[i], blockIdx.x - __ldg(off + i), smem_raw, red);
}

// Per-instance epilogue record: gauge shift of p and velocity correction u -= s G p.
struct EpiArgs {
  GridDev g;
  double* p;
  double* u;
  double* v;
  double* w;
  double s;           // dt / rho0
  double sx, sy;      // s / dx, s / dy
  const double* mean; // gauge sum (NULL: no shift)
  double mean_scale;
  double* conv;       // convergence slots, cleared by k_clear_batch
};

__global__ void k_clear_batch(const EpiArgs* __restrict__ e, int n) {
  const int i = blockIdx.x;
  if (i < n && threadIdx.x < VOFP_CONV_SLOTS) e[i].conv[threadIdx.x] = 0.0;
}

__global__ void k_shift_batch(const EpiArgs* __restrict__ e, const int* __restrict__ off, int n) {
  const int i = find_instance(off, n, blockIdx.x);
  const EpiArgs& a = e[i];
  if (!a.mean) return;
  const int nb = __ldg(off + i + 1) - __ldg(off + i);
  const int l = blockIdx.x - __ldg(off + i);
  const size_t cells = (size_t)a.g.nx * a.g.ny * a.g.nz;
  const double m = *a.mean * a.mean_scale;
  for (size_t t = (size_t)l * blockDim.x + threadIdx.x; t < cells; t += (size_t)nb * blockDim.x) a.p[t] -= m;
}

// Velocity correction of every instance: up to 512 blocks per instance striding over its faces (the
// instance lookup, a dependent binary search, is paid once per block: a block per 256 faces made it the
// kernel's cost).
__global__ void k_grad_batch(const EpiArgs* __restrict__ e, const int* __restrict__ off, int n) {
  const int inst = find_instance(off, n, blockIdx.x);
  const EpiArgs& a = e[inst];
  const int nb = __ldg(off + inst + 1) - __ldg(off + inst);
  const int l = blockIdx.x - __ldg(off + inst);
  const GridDev g = a.g;
  const size_t total = total_faces(g);
  for (size_t t = (size_t)l * blockDim.x + threadIdx.x; t < total; t += (size_t)nb * blockDim.x) {
    int i, j, k;
    size_t o;
    const int axis = decode_face(g, t, i, j, k, o);
    if (VOFP_IN(o, nfaces(g, axis), CHK_FACE_STORE)) grad_face(g, a.p, a.u, a.v, a.w, a.s, a.sx, a.sy, axis, i, j, k, o);
  }
}

static const int kMaxDynSmem = 200 * 1024;
template <typename K>
static void allow_smem(K kern) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

template <typename T, typename C>
static void allow_batch_kernels() {
  allow_smem(k_xfwd_batch<T, C, RHS_DIV>);
  allow_smem(k_xfwd_batch<T, C, RHS_RESID>);
  allow_smem(k_ypass_batch<T, C, false>);
  allow_smem(k_ypass_batch<T, C, true>);
  allow_smem(k_zsolve_batch<T>);
  allow_smem(k_ztab_batch<T, ZF<T>>);
  allow_smem(k_ztab_seg_batch<T, ZF<T>, false>);
  allow_smem(k_ztab_seg_batch<T, ZF<T>, true>);
  allow_smem(k_xinv_batch<T, C>);
}

}  // namespace vofp

using namespace vofp;

// Host object.  Device argument layout (one allocation): for each of the M + 1 solves s (0 = initial,
// k + 1 = correction k): XArgs[n], YArgs fwd[n], YArgs inv[n], ZArgs[n], XInvArgs[n]; then LowArgs[n],
// EpiArgs[n] and the prefix tables.
struct vofp_batch {
  int n;
  int M;
  std::vector<vofp_plan*> plans;
  int device;
  void* dmem;
  unsigned char* hstage;  // pinned host copy of the argument records
  size_t args_bytes;
  size_t o_x, o_yf, o_yi, o_z, o_xi, o_low, o_epi;  // per-solve stride arrays start offsets
  size_t o_offx, o_offy, o_offz, o_offlow, o_offepi;
  int tot_x, tot_y, tot_z, tot_low, tot_epi;
  bool ztab;  // every instance has a bounded z axis: factor-table z kernels
  bool zseg;  // ... and every instance's segmented tile fits in shared memory
  bool zlean;  // the segmented kernel's lean tile layout (some instance's full tile would hold an SM alone)
  int prec;   // VOFP_MIXED (FP32 spectrum) or VOFP_FF (FP32-pair spectrum), the same for every instance
  size_t sm_x, sm_y, sm_z;
  cudaGraphExec_t exec;
  cudaStream_t captured_on;
  int kernels_per_replay;
  std::vector<const void*> last_ptrs;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Systems per block of the general z kernel (used when some instance of the batch has a periodic z axis):
// as many as fit two or three columns each in 96 KB of shared memory, at most 32.
static int generic_ti(const vofp_plan* p, size_t rsz) {
  const int nvec = p->bc[2] == VOFP_BC_P ? 3 : 2;
  int ti = 32;
  while (ti > 1 && (size_t)nvec * ti * p->n[2] * rsz > 96 * 1024) ti /= 2;
  return ti;
}

extern "C" int vofp_batch_create(vofp_plan* const* plans, int n, vofp_batch** out) {
  if (!plans || n < 1 || !out) return VOFP_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = plans[0] ? plans[0]->device : -1;
  int M = 0;
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) return VOFP_ERR_INVALID_ARG;
    if (plans[i]->opts.prec != VOFP_MIXED && plans[i]->opts.prec != VOFP_FF) return VOFP_ERR_UNSUPPORTED;
    if (plans[i]->opts.prec != plans[0]->opts.prec) return VOFP_ERR_INVALID_ARG;  // one precision per batch
    if (plans[i]->device != dev) return VOFP_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return VOFP_ERR_INVALID_ARG;  // a plan's workspace serves one instance
    int m = plans[i]->opts.max_refine;
    if (m > VOFP_MAX_REFINE) m = VOFP_MAX_REFINE;
    if (m > M) M = m;
  }
  vofp_batch* b = new vofp_batch();
  b->n = n;
  b->M = M;
  b->plans.assign(plans, plans + n);
  b->device = dev;
  b->exec = nullptr;
  b->captured_on = nullptr;
  b->prec = plans[0]->opts.prec;
  const bool ffp = b->prec == VOFP_FF;
  const size_t csz = ffp ? sizeof(cff) : sizeof(float2), rsz = ffp ? sizeof(ff) : sizeof(float);
  const int S = M + 1;
  size_t o = 0;
  b->o_x = o;
  o = a256(o + sizeof(XArgs) * n * S);
  b->o_yf = o;
  o = a256(o + sizeof(YArgs) * n * S);
  b->o_yi = o;
  o = a256(o + sizeof(YArgs) * n * S);
  b->o_z = o;
  o = a256(o + sizeof(ZArgs) * n * S);
  b->o_xi = o;
  o = a256(o + sizeof(XInvArgs) * n * S);
  b->o_low = o;
  o = a256(o + sizeof(LowArgs) * n);
  b->o_epi = o;
  o = a256(o + sizeof(EpiArgs) * n);
  b->o_offx = o;
  o = a256(o + sizeof(int) * (n + 1));
  b->o_offy = o;
  o = a256(o + sizeof(int) * (n + 1));
  b->o_offz = o;
  o = a256(o + sizeof(int) * (n + 1));
  b->o_offlow = o;
  o = a256(o + sizeof(int) * (n + 1));
  b->o_offepi = o;
  o = a256(o + sizeof(int) * (n + 1));
  b->args_bytes = o;
  if (device_alloc(&b->dmem, o) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return VOFP_ERR_OOM;
  }
  if (pinned_alloc((void**)&b->hstage, o) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->dmem);
    delete b;
    return VOFP_ERR_OOM;
  }
  memset(b->hstage, 0, o);
  // prefix tables (sizes only) and shared-memory maxima
  int* offx = (int*)(b->hstage + b->o_offx);
  int* offy = (int*)(b->hstage + b->o_offy);
  int* offz = (int*)(b->hstage + b->o_offz);
  int* offl = (int*)(b->hstage + b->o_offlow);
  int* offe = (int*)(b->hstage + b->o_offepi);
  offx[0] = offy[0] = offz[0] = offl[0] = offe[0] = 0;
  b->sm_x = b->sm_y = b->sm_z = 0;
  b->ztab = true;
  for (int i = 0; i < n; ++i)
    if (!plans[i]->ztab) b->ztab = false;
  b->zseg = b->ztab;
  b->zlean = false;
  for (int i = 0; i < n; ++i)
    if (ztab_seg_code(plans[i]->n[2], rsz) != -1) b->zlean = true;
  for (int i = 0; i < n; ++i)
    if (ztab_seg_smem(plans[i]->n[2], rsz, b->zlean) > 200 * 1024) b->zseg = false;
  for (int i = 0; i < n; ++i) {
    const vofp_plan* p = plans[i];
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    offx[i + 1] = offx[i] + xpass_blocks(ny, nz, p->xpb);
    offy[i + 1] = offy[i] + (ny > 1 ? ((nx + p->ytx32 - 1) / p->ytx32) * nz : 0);
    const int gti = generic_ti(p, rsz);
    offz[i + 1] = offz[i] + (b->zseg ? (nx + kZSegTI - 1) / kZSegTI
                                     : (b->ztab ? (nx + 127) / 128 : (nx + gti - 1) / gti)) * ny;
    offl[i + 1] = offl[i] + p->nlow;
    // gauge shift and gradient: up to 512 blocks striding over the instance's cells / faces
    offe[i + 1] = offe[i] + (int)std::min<size_t>(512, (total_faces(grid_dev(p)) + 255) / 256);
    const size_t sx = 2 * (size_t)p->xpb * fft_span(p->ax[0].fd, p->ax[0].blu64) * csz;
    const size_t sy = 2 * (size_t)(p->ytx32 / 2) * y_ld(fft_span(p->ax[1].fd, p->ax[1].blu64)) * csz;
    const ZTabShape zs = ztab_shape(128, nz, rsz);
    const size_t sz = b->zseg ? ztab_seg_smem(nz, rsz, b->zlean)
                              : (b->ztab ? zs.smem : (size_t)(p->bc[2] == VOFP_BC_P ? 3 : 2) * gti * nz * rsz);
    if (sx > b->sm_x) b->sm_x = sx;
    if (sy > b->sm_y) b->sm_y = sy;
    if (sz > b->sm_z) b->sm_z = sz;
  }
  b->tot_x = offx[n];
  b->tot_y = offy[n];
  b->tot_z = offz[n];
  b->tot_low = offl[n];
  b->tot_epi = offe[n];
  if (first_use_on_device(2)) {
    allow_batch_kernels<float, float2>();
    allow_batch_kernels<ff, cff>();
  }
  *out = b;
  return VOFP_OK;
}

// Fill the argument records for the given field pointers.
static void fill_args(vofp_batch* b, double* const* u, double* const* v, double* const* w, const double* const* src,
                      const double* dt, double* const* p) {
  const int n = b->n, S = b->M + 1;
  const bool ffp = b->prec == VOFP_FF;
  XArgs* X = (XArgs*)(b->hstage + b->o_x);
  YArgs* YF = (YArgs*)(b->hstage + b->o_yf);
  YArgs* YI = (YArgs*)(b->hstage + b->o_yi);
  ZArgs* Z = (ZArgs*)(b->hstage + b->o_z);
  XInvArgs* XI = (XInvArgs*)(b->hstage + b->o_xi);
  LowArgs* L = (LowArgs*)(b->hstage + b->o_low);
  EpiArgs* E = (EpiArgs*)(b->hstage + b->o_epi);
  for (int i = 0; i < n; ++i) {
    vofp_plan* pl = b->plans[i];
    const int Mi = pl->opts.max_refine < b->M ? pl->opts.max_refine : b->M;
    const double tol2 = pl->opts.tol * pl->opts.tol;
    double* conv = pl->conv;
    double* pout = (p && p[i]) ? p[i] : pl->P;
    for (int s = 0; s < S; ++s) {
      const int k = s - 1;  // correction index (-1: initial solve)
      // x forward
      XArgs xa = {};
      xa.g = grid_dev(pl);
      xa.fd = pl->ax[0].fd;
      xa.tw = ffp ? (const void*)pl->ax[0].twff : (const void*)pl->ax[0].tw32;
      xa.quart = ffp ? (const void*)pl->ax[0].quartff : (const void*)pl->ax[0].quart32;
      xa.blu = ffp ? (const void*)pl->ax[0].bluff : (const void*)pl->ax[0].blu32;
      xa.pb = pl->xpb;
      xa.S = pl->S32;
      if (s == 0) {
        xa.u = u[i];
        xa.v = v[i];
        xa.w = w[i];
        xa.src = src ? src[i] : nullptr;
        xa.scale = 1.0 / dt[i];
        xa.fsave = pl->F;
        xa.sq_out = conv + 0;
        xa.fv_out = conv + 1;
        xa.abs_out = conv + 2;
        xa.skip_k = -1;
      } else {
        xa.f = pl->F;
        xa.p = pout;
        xa.defect_sum = pl->singular ? conv + 1 : nullptr;
        xa.inv_volume = 1.0 / pl->volume;
        xa.sq_out = conv + VOFP_CONV_RES + k;
        xa.skip_conv = conv;
        xa.skip_k = k;  // residual pass of correction s = k + 1: skipped when F_k
        xa.tol2 = tol2;
      }
      // corrections beyond this instance's own max_refine never run
      const bool off = s > Mi;
      YArgs ya = {};
      ya.nx = pl->n[0];
      ya.ny = pl->n[1];
      ya.nz = pl->n[2];
      ya.bc = pl->bc[1];
      ya.fd = pl->ax[1].fd;
      ya.tw = ffp ? (const void*)pl->ax[1].twff : (const void*)pl->ax[1].tw32;
      ya.quart = ffp ? (const void*)pl->ax[1].quartff : (const void*)pl->ax[1].quart32;
      ya.blu = ffp ? (const void*)pl->ax[1].bluff : (const void*)pl->ax[1].blu32;
      ya.tx = pl->ytx32;
      ya.S = pl->S32;
      ya.skip_conv = s == 0 ? nullptr : conv;
      ya.skip_k = s == 0 ? -1 : s;  // solve and inverse pass of correction s: skipped when F_s
      ya.tol2 = tol2;
      ZArgs za = z_args(pl, false);
      za.S = pl->S32;
      za.ti = generic_ti(pl, ffp ? sizeof(ff) : sizeof(float));  // general kernel only (bounded: 128)
      za.lowthr = pl->lowthr;
      za.skip_conv = ya.skip_conv;
      za.skip_k = ya.skip_k;
      za.tol2 = tol2;
      XInvArgs xi = {};
      xi.nx = pl->n[0];
      xi.ny = pl->n[1];
      xi.nz = pl->n[2];
      xi.bc = pl->bc[0];
      xi.fd = pl->ax[0].fd;
      xi.tw = ffp ? (const void*)pl->ax[0].twff : (const void*)pl->ax[0].tw32;
      xi.quart = ffp ? (const void*)pl->ax[0].quartff : (const void*)pl->ax[0].quart32;
      xi.blu = ffp ? (const void*)pl->ax[0].bluff : (const void*)pl->ax[0].blu32;
      xi.pb = pl->xpb;
      xi.S = pl->S32;
      xi.p = pout;
      xi.accumulate = s == 0 ? 0 : 1;
      xi.skip_conv = ya.skip_conv;
      xi.skip_k = ya.skip_k;
      xi.tol2 = tol2;
      xi.dz = pl->dz;
      xi.dzff = pl->dzff;
      xi.mean_out = (pl->singular && !ffp) ? conv + VOFP_CONV_MEAN : nullptr;  // FP32-pair: no gauge shift
      xi.d2_out = conv + VOFP_CONV_DEL + s;
      if (off) xa.skip_k = ya.skip_k = za.skip_k = xi.skip_k = -2;  // beyond this instance's own limit
      X[s * n + i] = xa;
      YF[s * n + i] = ya;
      YI[s * n + i] = ya;
      Z[s * n + i] = za;
      XI[s * n + i] = xi;
    }
    L[i].modes = pl->lowmodes;
    L[i].nlow = pl->nlow;
    L[i].scratch = pl->lowscratch;
    L[i].tab = pl->lowtab;
    L[i].zt = ztab_args(pl);
    L[i].smem_d = ztab_shape(128, pl->n[2], ffp ? sizeof(ff) : sizeof(float)).smem_d;
    EpiArgs e;
    e.g = grid_dev(pl);
    e.p = pout;
    e.u = u[i];
    e.v = v[i];
    e.w = w[i];
    e.s = dt[i];
    e.sx = dt[i] * e.g.rdx;
    e.sy = dt[i] * e.g.rdy;
    e.mean = (pl->singular && !ffp && p && p[i]) ? conv + VOFP_CONV_MEAN : nullptr;
    e.mean_scale = 1.0 / ((double)pl->n[0] * pl->n[1] * (pl->volume / (pl->n[0] * pl->dx * pl->n[1] * pl->dy)));
    e.conv = conv;
    E[i] = e;
  }
}

template <typename T, typename C>
static void launch_sequence_t(vofp_batch* b, cudaStream_t st) {
  const int n = b->n, S = b->M + 1;
  unsigned char* d = (unsigned char*)b->dmem;
  const int* offx = (const int*)(d + b->o_offx);
  const int* offy = (const int*)(d + b->o_offy);
  const int* offz = (const int*)(d + b->o_offz);
  const int* offl = (const int*)(d + b->o_offlow);
  const int* offe = (const int*)(d + b->o_offepi);
  const EpiArgs* E = (const EpiArgs*)(d + b->o_epi);
  const LowArgs* L = (const LowArgs*)(d + b->o_low);
  VOFP_LAUNCH(KID_BATCHED, st, k_clear_batch<<<n, 32, 0, st>>>(E, n));
  for (int s = 0; s < S; ++s) {
    const XArgs* X = (const XArgs*)(d + b->o_x) + (size_t)s * n;
    const YArgs* YF = (const YArgs*)(d + b->o_yf) + (size_t)s * n;
    const YArgs* YI = (const YArgs*)(d + b->o_yi) + (size_t)s * n;
    const ZArgs* Z = (const ZArgs*)(d + b->o_z) + (size_t)s * n;
    const XInvArgs* XI = (const XInvArgs*)(d + b->o_xi) + (size_t)s * n;
    if (s == 0)
      VOFP_LAUNCH(KID_XFWD_DIV, st, (k_xfwd_batch<T, C, RHS_DIV><<<b->tot_x, 256, b->sm_x, st>>>(X, offx, n)));
    else
      VOFP_LAUNCH(KID_RESID, st, (k_xfwd_batch<T, C, RHS_RESID><<<b->tot_x, 256, b->sm_x, st>>>(X, offx, n)));
    if (b->tot_y > 0)
      VOFP_LAUNCH(KID_YFWD, st, (k_ypass_batch<T, C, false><<<b->tot_y, 256, b->sm_y, st>>>(YF, offy, n)));
    if (b->ztab) {
      if (b->zseg && b->zlean)
        VOFP_LAUNCH(KID_ZSOLVE, st,
                    (k_ztab_seg_batch<T, ZF<T>, true><<<b->tot_z, 32 * kZSegW, b->sm_z, st>>>(Z, L, offz, n)));
      else if (b->zseg)
        VOFP_LAUNCH(KID_ZSOLVE, st,
                    (k_ztab_seg_batch<T, ZF<T>, false><<<b->tot_z, 32 * kZSegW, b->sm_z, st>>>(Z, L, offz, n)));
      else
        VOFP_LAUNCH(KID_ZSOLVE, st, k_ztab_batch<T, ZF<T>><<<b->tot_z, 128, b->sm_z, st>>>(Z, L, offz, n));
      if (b->tot_low > 0)
        VOFP_LAUNCH(KID_ZLOW, st,
                    k_zlow_scan_batch<T><<<(b->tot_low + 3) / 4, 128, 0, st>>>(Z, L, offl, n, b->tot_low));
    } else {
      VOFP_LAUNCH(KID_ZSOLVE, st, k_zsolve_batch<T><<<b->tot_z, 128, b->sm_z, st>>>(Z, offz, n));
      if (b->tot_low > 0)
        VOFP_LAUNCH(KID_ZLOW, st, k_zlow_batch<T><<<(b->tot_low + 63) / 64, 64, 0, st>>>(Z, L, offl, n, b->tot_low));
    }
    if (b->tot_y > 0)
      VOFP_LAUNCH(KID_YINV, st, (k_ypass_batch<T, C, true><<<b->tot_y, 256, b->sm_y, st>>>(YI, offy, n)));
    VOFP_LAUNCH(KID_XINV, st, (k_xinv_batch<T, C><<<b->tot_x, 256, b->sm_x, st>>>(XI, offx, n)));
  }
  VOFP_LAUNCH(KID_GAUGE, st, k_shift_batch<<<b->tot_epi, 256, 0, st>>>(E, offe, n));
  VOFP_LAUNCH(KID_GRAD, st, k_grad_batch<<<b->tot_epi, 256, 0, st>>>(E, offe, n));
}

static void launch_sequence(vofp_batch* b, cudaStream_t st) {
  if (b->prec == VOFP_FF)
    launch_sequence_t<ff, cff>(b, st);
  else
    launch_sequence_t<float, float2>(b, st);
}

extern "C" int vofp_batch_project(vofp_batch* b, double* const* u, double* const* v, double* const* w,
                                  const double* const* src, const double* dt_over_rho0, double* const* p,
                                  void* stream) {
  if (!b || !u || !v || !w || !dt_over_rho0) return VOFP_ERR_INVALID_ARG;
  for (int i = 0; i < b->n; ++i) {
    if (!u[i] || !v[i] || !w[i] || !(dt_over_rho0[i] > 0) || !std::isfinite(dt_over_rho0[i]))
      return VOFP_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // refresh the argument records when any pointer or scalar changed
  std::vector<const void*> key;
  key.reserve(6 * b->n);
  for (int i = 0; i < b->n; ++i) {
    key.push_back(u[i]);
    key.push_back(v[i]);
    key.push_back(w[i]);
    key.push_back(src ? src[i] : nullptr);
    key.push_back(p ? p[i] : nullptr);
    double d = dt_over_rho0[i];
    const void* dk;
    memcpy(&dk, &d, sizeof(dk));
    key.push_back(dk);
  }
  if (key != b->last_ptrs) {
    // the previous replay may still read the records: wait for this stream before rewriting them
    if (!b->last_ptrs.empty() && cudaStreamSynchronize(st) != cudaSuccess) return VOFP_ERR_CUDA;
    fill_args(b, u, v, w, src, dt_over_rho0, p);
    if (cudaMemcpyAsync(b->dmem, b->hstage, b->args_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return VOFP_ERR_CUDA;
    b->last_ptrs = key;
  }
  if (!b->exec || b->captured_on != st) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    // capture on a private stream so that the caller's stream may be the legacy default stream
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return VOFP_ERR_CUDA;
    cudaGraph_t g;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaStreamDestroy(cs);
      return VOFP_ERR_CUDA;
    }
    capture_begin();
    launch_sequence(b, cs);
    b->kernels_per_replay = (int)capture_end();
    const cudaError_t e1 = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (e1 != cudaSuccess) return VOFP_ERR_CUDA;
    const cudaError_t e2 = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
      b->exec = nullptr;
      return VOFP_ERR_CUDA;
    }
    b->captured_on = st;
  }
  TraceTok tk;
  trace_begin(KID_BATCHED, st, &tk);
  if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return VOFP_ERR_CUDA;
  trace_end(&tk, st);
  note_launches(b->kernels_per_replay);
  return VOFP_OK;
}

extern "C" int vofp_batch_size(const vofp_batch* b) { return b ? b->n : 0; }

extern "C" void vofp_batch_destroy(vofp_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->dmem);
  cudaFreeHost(b->hstage);
  delete b;
}
