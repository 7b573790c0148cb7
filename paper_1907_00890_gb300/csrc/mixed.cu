// Mixed-precision path: reduced-precision transforms and z recurrences for the bulk of the spectrum -- FP32
// (VOFP_MIXED) or FP32-pair float-float (VOFP_FF) -- and FP64 for the low-eigenvalue z systems, the
// right-hand side, the residual stencil, the accumulated potential and every reduction; defect-correction
// refinement (p += S(f - fbar - L p)) back to the accuracy of an FP64 solve.
//
// The loop is fully asynchronous: the residual norm of correction k is accumulated in FP64 by the residual
// pass itself, and every launch of the next correction reads it on the device and returns at once when the
// convergence test passes (so there is no host round trip and the whole sequence can be replayed as a
// graph).  The singular operator's mean is removed from the residual in FP64 (the compatibility defect is
// the FP64 volume-weighted mean of f, not the reduced-precision spectrum's), and the gauge of p (zero
// volume-weighted mean) is restored in FP64 at the end from the exact sums of the corrections.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "passes.cuh"
#include "solve_internal.h"
#include "xinv_tma.cuh"
#include "ypass_tma.cuh"
#include "zsolve.cuh"

namespace vofp {

static const int kMaxDynSmem = 200 * 1024;

template <typename K>
static void allow_smem(K kern) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

template <typename T, typename C, typename TT>
static void allow_all() {
  allow_smem(xfwd_kernel<T, C, RHS_F>());
  allow_smem(xfwd_kernel<T, C, RHS_DIV>());
  allow_smem(xfwd_kernel<T, C, RHS_DIV_STEFAN>());
  allow_smem(xfwd_kernel<T, C, RHS_RESID>());
  allow_smem(ypass_kernel<T, C, false>());
  allow_smem(ypass_kernel<T, C, true>());
  allow_smem(xinv_kernel<T, C>());
  allow_smem(k_zsolve<T, T>);
  allow_smem(k_ztab<T, TT>);
  allow_smem(k_ztab_staged<T, TT>);
  allow_smem(k_ztab_seg<T, TT, false>);
  allow_smem(k_ztab_seg<T, TT, true>);
}

// Shared memory a TMA y-pass CTA may take (of the 227 KiB an sm_103a CTA can opt into), and the tile budget
// per spectrum type: FP64 tiles of at most 112 KB (two CTAs per SM: ny = 512 passes 4% faster than with one
// CTA of 196 KB), FP32 and FP32-pair tiles up to the limit (measured the other way round: halving their
// tiles slowed the 512^3 FP32 + refinement solve from 20.05 to 20.21 ms).
static const int kYTmaSmem = 225 * 1024;
template <typename R>
constexpr size_t kYTmaTile = std::is_same<R, double>::value ? (size_t)112 * 1024 : (size_t)kYTmaSmem;

// The TMA inverse x-pass kernel for nx = 2^lgn (7, 8 or 9), with a tile (2^lgB complex lines) of about 100 KB
// of shared memory (8 KB of samples per line pair with the potential's rows), so that two CTAs share an SM:
// with one 512-thread CTA per SM (tiles of about 200 KB) the pass was issue-latency bound (25% of warps
// active); two CTAs took the FP32 inverse passes of a 512^3 solve from 2.73 to 2.30 ms.  NULL for other
// lengths.
typedef void (*XTmaKernel)(const XTmaArgs, const CUtensorMap, const CUtensorMap);
template <typename R>
static int xtma_lgB(int lgn) {
  return std::is_same<R, float>::value ? (lgn >= 9 ? 2 : 3) : (lgn >= 9 ? 2 : (lgn == 8 ? 3 : 4));
}
template <typename R>
static XTmaKernel xtma_kernel(int lgn) {
  constexpr bool F = std::is_same<R, float>::value;
  if (lgn == 9) return k_xinv_tma<R, 9, 2>;
  if (lgn == 8) return k_xinv_tma<R, 8, 3>;
  if (lgn == 7) return F ? k_xinv_tma<R, 7, 3> : k_xinv_tma<R, 7, 4>;
  return nullptr;
}

// The TMA y-pass kernel for a length 2^lgn and 2^lgB lines per tile: compiled for ny = 128, 256, 512 with the
// tile width ytma_setup picks for them, else the version that reads both from its arguments.
typedef void (*YTmaKernel)(const YTmaArgs, const CUtensorMap);
template <typename R>
static YTmaKernel ytma_kernel(bool inv, int lgn, int lgB) {
  constexpr bool F = std::is_same<R, float>::value;
  constexpr int B9 = F ? 4 : (std::is_same<R, double>::value ? 2 : 3);
  if (lgn == 9 && lgB == B9) return inv ? k_ypass_tma<R, true, 9, B9> : k_ypass_tma<R, false, 9, B9>;
  if (lgn == 8 && lgB == 4) return inv ? k_ypass_tma<R, true, 8, 4> : k_ypass_tma<R, false, 8, 4>;
  if (lgn == 7 && lgB == 4) return inv ? k_ypass_tma<R, true, 7, 4> : k_ypass_tma<R, false, 7, 4>;
  return inv ? k_ypass_tma<R, true> : k_ypass_tma<R, false>;
}

void init_kernel_attributes_mixed() {
  if (!first_use_on_device(1)) return;
  allow_all<float, float2, ZF<float>>();
  allow_all<ff, cff, ZF<ff>>();
  for (int inv = 0; inv < 2; ++inv)
    for (int lgn = 0; lgn <= 9; ++lgn)
      for (int lgB = 2; lgB <= 4; ++lgB) {
        cudaFuncSetAttribute(ytma_kernel<float>(inv, lgn, lgB), cudaFuncAttributeMaxDynamicSharedMemorySize, kYTmaSmem);
        cudaFuncSetAttribute(ytma_kernel<ff>(inv, lgn, lgB), cudaFuncAttributeMaxDynamicSharedMemorySize, kYTmaSmem);
        cudaFuncSetAttribute(ytma_kernel<double>(inv, lgn, lgB), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kYTmaSmem);
      }
  for (int lgn = 7; lgn <= 9; ++lgn) {
    cudaFuncSetAttribute(xtma_kernel<float>(lgn), cudaFuncAttributeMaxDynamicSharedMemorySize, kYTmaSmem);
    cudaFuncSetAttribute(xtma_kernel<ff>(lgn), cudaFuncAttributeMaxDynamicSharedMemorySize, kYTmaSmem);
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// First use of the TMA y pass on a reduced-precision plan: applicable when ny is a power of two of at least 8
// (the tile is loaded in boxes of at most 256 rows), a row of the spectrum is a multiple of 16 bytes (the
// tensor map's stride rule) and at least one tile wide; then the widest tile (2^lgB complex lines, lgB = 4, 3
// or 2) whose three buffers fit, the persistent grid (resident CTAs x SMs, at most one CTA per tile) and the
// tensor map over the plan's spectrum.
template <typename R>
static void ytma_setup(vofp_plan* pl, void* spectrum) {
  pl->ytma_state = -1;
  const char* env = getenv("VOFP_Y_TMA");
  if (env && env[0] == '0') return;
  const int nx = pl->n[0], ny = pl->n[1], nz = pl->n[2];
  if (ny < 8 || ny > 4096 || (ny & (ny - 1)) || ((size_t)nx * sizeof(R)) % 16) return;
  // FP64 spectra only from ny = 256: their passes are bound by the FP64 pipe, and at ny = 128 (under two tiles
  // per persistent CTA) the gather kernel was measured faster (128^3 droplet step 0.825 against 0.850 ms); at
  // 512^3 the tiles win by 9% per pass
  if (std::is_same<R, double>::value && ny < 256) return;
  int lgB = -1;
  for (int lb = 4; lb >= 2 && lgB < 0; --lb)
    if ((2 << lb) <= nx && ytma_smem_bytes(ny, lb, 2 * sizeof(R)) <= kYTmaTile<R>) lgB = lb;
  if (lgB < 0) return;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return;
  CUtensorMap tm;
  const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny * nz};
  const cuuint64_t strides[1] = {(cuuint64_t)nx * sizeof(R)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 << lgB), (cuuint32_t)(ny < 256 ? ny : 256)};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  if (enc(&tm, dt, 2, spectrum, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return;
  const size_t sm = ytma_smem_bytes(ny, lgB, 2 * sizeof(R));
  int per_sm = 0, nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ytma_kernel<R>(false, 31 - __builtin_clz((unsigned)ny), lgB),
                                                    kYTmaThreads, sm) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return;
  }
  const int tiles = ((nx + (2 << lgB) - 1) / (2 << lgB)) * nz;
  pl->ytma_lgB = lgB;
  pl->ytma_grid = tiles < per_sm * nsm ? tiles : per_sm * nsm;
  static_assert(sizeof(CUtensorMap) <= sizeof(pl->ytma_map), "tensor map storage");
  memcpy(pl->ytma_map, &tm, sizeof(tm));
  pl->ytma_state = 1;
}

// First use of the TMA inverse x pass: nx of 128, 256 or 512 (VOFP_X_TMA=0 switches it off); the tensor map
// views the spectrum as {min(nx, 256), nx / min(nx, 256), ny nz} so that one box is a tile of whole lines.
template <typename R>
static void xtma_setup(vofp_plan* pl) {
  pl->xtma_state = -1;
  const char* env = getenv("VOFP_X_TMA");
  if (env && env[0] == '0') return;
  const int nx = pl->n[0];
  if (nx != 128 && nx != 256 && nx != 512) return;
  const int lgn = 31 - __builtin_clz((unsigned)nx), lgB = xtma_lgB<R>(lgn);
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return;
  const int h = nx < 256 ? nx : 256;
  const long nlines = (long)pl->n[1] * pl->n[2];
  CUtensorMap tm;
  const cuuint64_t dims[3] = {(cuuint64_t)h, (cuuint64_t)(nx / h), (cuuint64_t)nlines};
  const cuuint64_t strides[2] = {(cuuint64_t)h * sizeof(R), (cuuint64_t)nx * sizeof(R)};
  const cuuint32_t box[3] = {(cuuint32_t)h, (cuuint32_t)(nx / h), (cuuint32_t)(2 << lgB)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  if (enc(&tm, dt, 3, pl->S32, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return;
  int per_sm = 0, nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xtma_kernel<R>(lgn), kXTmaThreads,
                                                    xtma_smem_bytes(nx, lgB, sizeof(R), true)) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return;
  }
  const long tiles = (nlines + (2 << lgB) - 1) / (2 << lgB);
  pl->xtma_grid = (int)(tiles < (long)per_sm * nsm ? tiles : (long)per_sm * nsm);
  static_assert(sizeof(CUtensorMap) <= sizeof(pl->xtma_map), "tensor map storage");
  memcpy(pl->xtma_map, &tm, sizeof(tm));
  pl->xtma_state = 1;
}

// Tensor map of the potential p for an accumulating inverse x pass: the spectrum's 3-D view with FP64 elements.
// (Encoded per call: the potential is the caller's array or the plan's scratch; a host-side encode takes about a
// microsecond.)
static bool xtma_potential_map(int nx, long nlines, double* p, int lgB, CUtensorMap* tm) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)p & 15)) return false;
  const int h = nx < 256 ? nx : 256;
  const cuuint64_t dims[3] = {(cuuint64_t)h, (cuuint64_t)(nx / h), (cuuint64_t)nlines};
  const cuuint64_t strides[2] = {(cuuint64_t)h * sizeof(double), (cuuint64_t)nx * sizeof(double)};
  const cuuint32_t box[3] = {(cuuint32_t)h, (cuuint32_t)(nx / h), (cuuint32_t)(2 << lgB)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <typename R>
static bool xinv_tma(vofp_plan* pl, const XInvArgs& xi, cudaStream_t st) {
  if (pl->xtma_state == 0) xtma_setup<R>(pl);
  if (pl->xtma_state != 1) return false;
  CUtensorMap tm, tp;
  memcpy(&tm, pl->xtma_map, sizeof(tm));
  const int lgn = 31 - __builtin_clz((unsigned)pl->n[0]);
  XTmaArgs ta;
  ta.xi = xi;
  ta.lgB = xtma_lgB<R>(lgn);
  ta.info = pl->info;
  const bool acc = xi.p && xi.accumulate;
  if (acc) {
    if (!xtma_potential_map(pl->n[0], (long)pl->n[1] * pl->n[2], xi.p, ta.lgB, &tp)) return false;
  } else {
    tp = tm;  // not read
  }
  const size_t sm = xtma_smem_bytes(pl->n[0], ta.lgB, sizeof(R), acc);
  VOFP_LAUNCH(KID_XINV, st, (xtma_kernel<R>(lgn)<<<pl->xtma_grid, kXTmaThreads, sm, st>>>(ta, tm, tp)));
  return true;
}

// The y pass through TMA-staged tiles when the plan allows it; false: the caller runs the gather kernel.
template <typename R>
static bool ypass_tma(vofp_plan* pl, const YArgs& ya, bool inv, cudaStream_t st) {
  if (pl->ytma_state == 0) ytma_setup<R>(pl, ya.S);
  if (pl->ytma_state != 1) return false;
  CUtensorMap tm;
  memcpy(&tm, pl->ytma_map, sizeof(tm));
  YTmaArgs ta;
  ta.y = ya;
  ta.lgB = pl->ytma_lgB;
  ta.tiles_x = (pl->n[0] + (2 << ta.lgB) - 1) / (2 << ta.lgB);
  ta.info = pl->info;
  const size_t sm = ytma_smem_bytes(pl->n[1], ta.lgB, 2 * sizeof(R));
  const YTmaKernel kern = ytma_kernel<R>(inv, 31 - __builtin_clz((unsigned)pl->n[1]), ta.lgB);
  VOFP_LAUNCH(inv ? KID_YINV : KID_YFWD, st, (kern<<<pl->ytma_grid, kYTmaThreads, sm, st>>>(ta, tm)));
  return true;
}

int build_low_factors(vofp_plan* pl, cudaStream_t st, bool sync) {
  ZArgs za = z_args(pl, false);
  k_zfactor_low<<<(pl->nlow + 127) / 128, 128, 0, st>>>(za, pl->lowmodes, pl->nlow, pl->lowtab);
  if (cudaGetLastError() != cudaSuccess) return VOFP_ERR_CUDA;
  if (sync && cudaStreamSynchronize(st) != cudaSuccess) return VOFP_ERR_CUDA;
  return VOFP_OK;
}

// p -= (*sum) * scale  (gauge restoration)
__global__ void k_shift(double* p, size_t n, const double* sum, double scale) {
  const double m = *sum * scale;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    p[t] -= m;
}

// Reduced-precision element types: R (real) / C (complex) of the spectrum and its tables.
template <typename R>
struct Red;
template <>
struct Red<float> {
  typedef float2 C;
  typedef ZF<float> TT;  // z factor entry
  static const void* tw(const AxisDev& a) { return a.tw32; }
  static const void* quart(const AxisDev& a) { return a.quart32; }
  static const void* blu(const AxisDev& a) { return a.blu32; }
};
template <>
struct Red<ff> {
  typedef cff C;
  typedef ZF<ff> TT;
  static const void* tw(const AxisDev& a) { return a.twff; }
  static const void* quart(const AxisDev& a) { return a.quartff; }
  static const void* blu(const AxisDev& a) { return a.bluff; }
};

// y forward, z (bulk + FP64 low modes), y inverse on the spectrum; skipped when converged.
template <typename R>
static void solve_red(vofp_plan* pl, cudaStream_t st, int skip_k, double tol2, bool stats) {
  typedef typename Red<R>::C C;
  const int nx = pl->n[0], ny = pl->n[1], nz = pl->n[2];
  YArgs ya = {};
  ya.nx = nx;
  ya.ny = ny;
  ya.nz = nz;
  ya.bc = pl->bc[1];
  ya.fd = pl->ax[1].fd;
  ya.tw = Red<R>::tw(pl->ax[1]);
  ya.quart = Red<R>::quart(pl->ax[1]);
  ya.blu = Red<R>::blu(pl->ax[1]);
  ya.tx = pl->ytx32;
  ya.S = pl->S32;
  ya.skip_conv = pl->conv;
  ya.skip_k = skip_k;
  ya.tol2 = tol2;
  const dim3 ygrid((nx + ya.tx - 1) / ya.tx, nz);
  const size_t ysm = 2 * (size_t)(ya.tx / 2) * y_ld(fft_span(ya.fd, ya.blu)) * sizeof(C);
  if (ny > 1 && !ypass_tma<R>(pl, ya, false, st))
    VOFP_LAUNCH(KID_YFWD, st, (ypass_kernel<R, C, false>()<<<ygrid, 256, ysm, st>>>(ya)));
  ZArgs za = z_args(pl, stats);
  za.S = pl->S32;
  za.ti = pl->zti32;
  za.lowthr = pl->lowthr;
  za.skip_conv = pl->conv;
  za.skip_k = skip_k;
  za.tol2 = tol2;
  if (pl->ztab) {
    // bulk systems from the factor table; the low-eigenvalue ones (a prefix of each row) by one warp each.
    // Small grids: the shared-memory staged kernel (too few systems to hide the row loads one thread each)
    if (pl->zti32 == -1 || pl->zti32 == -2) {
      const dim3 tgrid((nx + kZSegTI - 1) / kZSegTI, ny);
      const size_t sm = ztab_seg_smem(nz, sizeof(R), pl->zti32 == -2);
      if (pl->zti32 == -2)
        VOFP_LAUNCH(KID_ZSOLVE, st,
                    (k_ztab_seg<R, typename Red<R>::TT, true><<<tgrid, 32 * kZSegW, sm, st>>>(za, ztab_args(pl))));
      else
        VOFP_LAUNCH(KID_ZSOLVE, st,
                    (k_ztab_seg<R, typename Red<R>::TT, false><<<tgrid, 32 * kZSegW, sm, st>>>(za, ztab_args(pl))));
    } else if (pl->zti32 == 0) {
      const dim3 tgrid((nx + kZStagedTI - 1) / kZStagedTI, ny);
      VOFP_LAUNCH(KID_ZSOLVE, st,
                  (k_ztab_staged<R, typename Red<R>::TT><<<tgrid, 128, ztab_staged_smem(nz, sizeof(R)), st>>>(
                      za, ztab_args(pl))));
    } else {
      const ZTabShape zs = ztab_shape(pl->zti32, nz, sizeof(R));
      const dim3 tgrid((nx + zs.threads - 1) / zs.threads, ny);
      VOFP_LAUNCH(KID_ZSOLVE, st,
                  (k_ztab<R, typename Red<R>::TT><<<tgrid, zs.threads, zs.smem, st>>>(za, ztab_args(pl),
                                                                                     zs.smem_d)));
    }
    if (pl->nlow > 0)
      VOFP_LAUNCH(KID_ZLOW, st,
                  k_zlow_scan<R><<<(pl->nlow + 3) / 4, 128, 0, st>>>(za, pl->lowmodes, pl->nlow, pl->lowtab,
                                                                     pl->lowscratch));
  } else {
    const int nvec = pl->bc[2] == VOFP_BC_P ? 3 : 2;
    const dim3 zgrid((nx + za.ti - 1) / za.ti, ny);
    const size_t zsm = (size_t)nvec * za.ti * nz * sizeof(R);
    VOFP_LAUNCH(KID_ZSOLVE, st, (k_zsolve<R, R><<<zgrid, 128, zsm, st>>>(za)));
    if (pl->nlow > 0)
      VOFP_LAUNCH(KID_ZLOW, st,
                  k_zlow64<R><<<(pl->nlow + 63) / 64, 64, 0, st>>>(za, pl->lowmodes, pl->nlow, nullptr,
                                                                   pl->lowscratch));
  }
  if (ny > 1 && !ypass_tma<R>(pl, ya, true, st))
    VOFP_LAUNCH(KID_YINV, st, (ypass_kernel<R, C, true>()<<<ygrid, 256, ysm, st>>>(ya)));
}

// pout == NULL: norm only (d2_out), nothing stored and no gauge sum (the error-estimate solve).
template <typename R>
static void xinv_red(vofp_plan* pl, double* pout, int accumulate, int skip_k, double tol2, double* d2_out,
                     cudaStream_t st) {
  typedef typename Red<R>::C C;
  XInvArgs xi = {};
  xi.nx = pl->n[0];
  xi.ny = pl->n[1];
  xi.nz = pl->n[2];
  xi.bc = pl->bc[0];
  xi.fd = pl->ax[0].fd;
  xi.tw = Red<R>::tw(pl->ax[0]);
  xi.quart = Red<R>::quart(pl->ax[0]);
  xi.blu = Red<R>::blu(pl->ax[0]);
  xi.pb = pl->xpb;
  xi.S = pl->S32;
  xi.p = pout;
  xi.accumulate = accumulate;
  xi.skip_conv = pl->conv;
  xi.skip_k = skip_k;
  xi.tol2 = tol2;
  xi.dz = pl->dz;
  xi.dzff = pl->dzff;
  // gauge: the FP32 spectrum's rounding leaves p with a mean of ~1e-7 |p| that is removed in FP64 at the end;
  // FP32-pair transforms keep the zero-mean gauge of the pinned mean mode to ~1e-14 and need no shift
  xi.mean_out = (pout && pl->singular && pl->opts.prec == VOFP_MIXED) ? pl->conv + VOFP_CONV_MEAN : nullptr;
  xi.d2_out = d2_out;
  if (std::is_same<R, float>::value && xtc_xinv(pl, xi, st)) return;  // tensor-core transform
  if (xinv_tma<R>(pl, xi, st)) return;                                   // TMA-staged tiles
  const int xgrid = xpass_blocks(xi.ny, xi.nz, xi.pb);
  const size_t xsm = 2 * (size_t)xi.pb * fft_span(xi.fd, xi.blu) * sizeof(C);
  VOFP_LAUNCH(KID_XINV, st, (xinv_kernel<R, C>()<<<xgrid, 256, xsm, st>>>(xi)));
}

template <typename R>
static void xfwd_red(vofp_plan* pl, int mode, XArgs xa, cudaStream_t st) {
  typedef typename Red<R>::C C;
  xa.g = grid_dev(pl);
  xa.fd = pl->ax[0].fd;
  xa.tw = Red<R>::tw(pl->ax[0]);
  xa.quart = Red<R>::quart(pl->ax[0]);
  xa.blu = Red<R>::blu(pl->ax[0]);
  xa.pb = pl->xpb;
  xa.S = pl->S32;
  if (std::is_same<R, float>::value && xtc_xfwd(pl, mode, xa, st)) return;  // tensor-core transform
  const int xgrid = xpass_blocks(pl->n[1], pl->n[2], xa.pb);
  const size_t xsm = 2 * (size_t)xa.pb * fft_span(xa.fd, xa.blu) * sizeof(C);
  switch (mode) {
    case RHS_F: VOFP_LAUNCH(KID_XFWD, st, (xfwd_kernel<R, C, RHS_F>()<<<xgrid, 256, xsm, st>>>(xa))); break;
    case RHS_DIV: VOFP_LAUNCH(KID_XFWD_DIV, st, (xfwd_kernel<R, C, RHS_DIV>()<<<xgrid, 256, xsm, st>>>(xa))); break;
    case RHS_DIV_STEFAN:
      VOFP_LAUNCH(KID_XFWD_DIVSTEF, st, (xfwd_kernel<R, C, RHS_DIV_STEFAN>()<<<xgrid, 256, xsm, st>>>(xa)));
      break;
    default: VOFP_LAUNCH(KID_RESID, st, (xfwd_kernel<R, C, RHS_RESID>()<<<xgrid, 256, xsm, st>>>(xa))); break;
  }
}

template <typename R>
static void refine_sequence(vofp_plan* pl, int mode, XArgs xa, double* pout, int M, double tol2, bool stats,
                            cudaStream_t st) {
  double* conv = pl->conv;
  xfwd_red<R>(pl, mode, xa, st);
  solve_red<R>(pl, st, -1, tol2, stats);
  xinv_red<R>(pl, pout, 0, -1, tol2, (M > 0 || stats) ? conv + VOFP_CONV_DEL : nullptr, st);
  // correction j: residual pass R_j (skipped when F_{j-1}), solve S_j and inverse pass X_j (skipped when F_j)
  for (int j = 1; j <= M; ++j) {
    XArgs ra = {};
    ra.f = pl->F;
    ra.p = pout;
    ra.defect_sum = pl->singular ? conv + 1 : nullptr;
    ra.inv_volume = 1.0 / pl->volume;
    ra.sq_out = conv + VOFP_CONV_RES + j - 1;
    ra.skip_conv = conv;
    ra.skip_k = j - 1;
    ra.tol2 = tol2;
    xfwd_red<R>(pl, RHS_RESID, ra, st);
    solve_red<R>(pl, st, j, tol2, stats);
    xinv_red<R>(pl, pout, 1, j, tol2, conv + VOFP_CONV_DEL + j, st);
  }
}

// Error estimate of the returned p (with info only): its FP64 residual r = f - fbar - L p (squared norm into
// VOFP_CONV_FINAL) solved once more in the plan's precision, the correction S(r) not applied; ||S(r)|| is
// the error left in p to the relative accuracy of one reduced-precision solve (~1e-6 FP32, ~1e-13 FP32
// pairs), plus the rounding of r itself.
template <typename R>
static void estimate_sequence(vofp_plan* pl, double* pout, double tol2, cudaStream_t st) {
  double* conv = pl->conv;
  XArgs ra = {};
  ra.f = pl->F;
  ra.p = pout;
  ra.defect_sum = pl->singular ? conv + 1 : nullptr;
  ra.inv_volume = 1.0 / pl->volume;
  ra.sq_out = conv + VOFP_CONV_FINAL;
  ra.skip_conv = nullptr;
  ra.skip_k = -1;
  ra.tol2 = tol2;
  xfwd_red<R>(pl, RHS_RESID, ra, st);
  solve_red<R>(pl, st, -1, tol2, true);
  xinv_red<R>(pl, nullptr, 0, -1, tol2, conv + VOFP_CONV_EST, st);
}

int mixed_solve(vofp_plan* pl, int mode, const XArgs* xin, const double* f, double* pout, cudaStream_t st,
                vofp_info* info) {
  if (mode == RHS_STEFAN) return VOFP_ERR_UNSUPPORTED;  // the extension passes its source as RHS_F
  if (!pl->S32 || !pl->F) return VOFP_ERR_INVALID_ARG;  // an FP64 plan has no reduced-precision workspace
  const double tol2 = pl->opts.tol * pl->opts.tol;
  int M = pl->opts.max_refine;
  if (M > VOFP_MAX_REFINE) M = VOFP_MAX_REFINE;
  const size_t cells = (size_t)pl->n[0] * pl->n[1] * pl->n[2];
  double* conv = pl->conv;
  if (cudaMemsetAsync(conv, 0, sizeof(double) * VOFP_CONV_SLOTS, st) != cudaSuccess) return VOFP_ERR_CUDA;
  const bool stats = info != nullptr;

  // initial solve of f (kept in FP64 in pl->F), then the corrections
  XArgs xa = {};
  if (xin) xa = *xin;
  if (mode == RHS_F) {
    xa.f = f;
    xa.scale = 1.0;
  }
  // a direct solve without statistics (no correction, no info) needs neither the FP64 right-hand side nor
  // the norms: its x pass then does no FP64 arithmetic beyond the right-hand side itself
  const bool need = M > 0 || info != nullptr;
  xa.fsave = need ? pl->F : nullptr;
  xa.sq_out = need ? conv + 0 : nullptr;
  xa.fv_out = need ? conv + 1 : nullptr;
  xa.abs_out = need ? conv + 2 : nullptr;
  xa.skip_k = -1;
  xa.info = nullptr;
  if (pl->opts.prec == VOFP_FF)
    refine_sequence<ff>(pl, mode, xa, pout, M, tol2, stats, st);
  else
    refine_sequence<float>(pl, mode, xa, pout, M, tol2, stats, st);
  if (info) {
    if (pl->opts.prec == VOFP_FF)
      estimate_sequence<ff>(pl, pout, tol2, st);
    else
      estimate_sequence<float>(pl, pout, tol2, st);
  }
  if (pl->singular && pl->opts.prec == VOFP_MIXED && pout != pl->P) {
    const double scale = 1.0 / ((double)pl->n[0] * pl->n[1] * (pl->volume / (pl->n[0] * pl->dx * pl->n[1] * pl->dy)));
    VOFP_LAUNCH(KID_GAUGE, st,
                k_shift<<<grid_blocks(cells, 256), 256, 0, st>>>(pout, cells, conv + VOFP_CONV_MEAN, scale));
  }
  if (cudaGetLastError() != cudaSuccess) return VOFP_ERR_CUDA;
  if (!info) return VOFP_OK;

  double h[VOFP_CONV_SLOTS];
  vofp_devinfo hi;
  if (cudaMemcpyAsync(h, conv, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&hi, pl->info, sizeof(hi), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return VOFP_ERR_CUDA;
  int status = VOFP_OK;
  const double f2 = h[0];
  const double rr = f2 > 0 ? std::sqrt(h[VOFP_CONV_FINAL] / f2) : 0.0;
  int iters = 0;
  bool conv_ok;
  if (M == 0) {
    conv_ok = rr <= pl->opts.tol;  // no correction requested: judge the direct solve by its residual
  } else {
    // corrections that ran: up to the first m whose successor's solve was skipped (F_{m+1})
    iters = 1;
    while (iters < M && !refine_done(h, iters + 1, tol2)) ++iters;
    conv_ok = iters < M || (rr <= pl->opts.tol && refine_err_ok(h, M, tol2));
  }
  const double defect = pl->singular ? h[1] / pl->volume : 0.0;
  info->compat_defect = defect;
  // the gauge shift subtracted from p by k_shift (FP32 spectra); FP32-pair and FP64 keep the pinned mean
  // mode and subtract nothing
  info->mean_removed = (pl->singular && pl->opts.prec == VOFP_MIXED)
                           ? h[VOFP_CONV_MEAN] / ((double)pl->n[0] * pl->n[1] *
                                                  (pl->volume / (pl->n[0] * pl->dx * pl->n[1] * pl->dy)))
                           : 0.0;
  info->err_estimate = h[VOFP_CONV_DEL] > 0 ? std::sqrt(h[VOFP_CONV_EST] / h[VOFP_CONV_DEL]) : 0.0;
  info->rel_residual = rr;
  info->refine_iters = iters;
  if (hi.nonfinite || !std::isfinite(f2) || !std::isfinite(rr)) status = VOFP_ERR_NONFINITE;
  if (hi.timeout) status = VOFP_ERR_TIMEOUT;  // a bounded wait for a tile load gave up
  if (status == VOFP_OK && !conv_ok) status = VOFP_WARN_NOT_CONVERGED;
  if (status == VOFP_OK && pl->singular && std::fabs(defect) > 1e-12 * h[2] / pl->volume)
    status = VOFP_WARN_INCOMPATIBLE_RHS;
  info->status = status;
  return status;
}

// The FP64 plans' y pass on TMA tiles (same kernel, FP64 spectrum); false: the caller runs the gather kernel.
bool ypass_tma_f64(vofp_plan* pl, const YArgs& ya, bool inv, cudaStream_t st) {
  return ypass_tma<double>(pl, ya, inv, st);
}

}  // namespace vofp
