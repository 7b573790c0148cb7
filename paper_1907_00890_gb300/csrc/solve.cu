// Host orchestration of the FP64 path and the public entry points
// vofp_poisson_solve / vofp_project / vofp_extend_liquid_velocity.
//
// One solve = x pass (right-hand side fused) -> y pass -> z tridiagonal pass -> inverse y -> inverse x,
// then the face epilogue (§3.2 projection, §3.6 extension).  Every launch goes to the caller's stream.
#include <cmath>
#include <cstdio>

#include "epilogue.cuh"
#include "passes.cuh"
#include "solve_internal.h"
#include "zsolve.cuh"

using namespace vofp;

namespace vofp {

GridDev grid_dev(const vofp_plan* pl) {
  GridDev g;
  g.nx = pl->n[0];
  g.ny = pl->n[1];
  g.nz = pl->n[2];
  g.bcx = pl->bc[0];
  g.bcy = pl->bc[1];
  g.bcz = pl->bc[2];
  g.dx = pl->dx;
  g.dy = pl->dy;
  g.dz = pl->dz;
  g.hz = pl->hz;
  return g;
}

static const int kMaxDynSmem = 200 * 1024;

template <typename K>
static void allow_smem(K kern) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

void init_kernel_attributes_fp64() {
  allow_smem(k_xfwd<double, double2, RHS_F>);
  allow_smem(k_xfwd<double, double2, RHS_DIV>);
  allow_smem(k_xfwd<double, double2, RHS_STEFAN>);
  allow_smem(k_xfwd<double, double2, RHS_DIV_STEFAN>);
  allow_smem(k_ypass<double, double2, false>);
  allow_smem(k_ypass<double, double2, true>);
  allow_smem(k_xinv<double, double2>);
  allow_smem(k_zsolve64);
}

int grid_blocks(size_t total, int threads) {
  size_t b = (total + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// x forward + y forward + z solve + y inverse + x inverse into `pout`.
int fp64_solve(vofp_plan* pl, int mode, XArgs xa, double* pout, cudaStream_t st, bool stats) {
  const int nx = pl->n[0], ny = pl->n[1], nz = pl->n[2];
  xa.g = grid_dev(pl);
  xa.fd = pl->ax[0].fd;
  xa.tw = pl->ax[0].tw64;
  xa.quart = pl->ax[0].quart64;
  xa.pb = pl->xpb;
  xa.S = pl->S;
  xa.info = stats ? pl->info : nullptr;
  const long npairs = ((long)ny * nz + 1) / 2;
  const int xgrid = (int)((npairs + xa.pb - 1) / xa.pb);
  const size_t xsm = 2 * (size_t)xa.pb * nx * sizeof(double2);
  switch (mode) {
    case RHS_F: VOFP_LAUNCH(KID_XFWD, st, k_xfwd<double, double2, RHS_F><<<xgrid, 256, xsm, st>>>(xa)); break;
    case RHS_DIV: VOFP_LAUNCH(KID_XFWD_DIV, st, k_xfwd<double, double2, RHS_DIV><<<xgrid, 256, xsm, st>>>(xa)); break;
    case RHS_STEFAN:
      VOFP_LAUNCH(KID_XFWD_STEFAN, st, k_xfwd<double, double2, RHS_STEFAN><<<xgrid, 256, xsm, st>>>(xa));
      break;
    case RHS_DIV_STEFAN:
      VOFP_LAUNCH(KID_XFWD_DIVSTEF, st, k_xfwd<double, double2, RHS_DIV_STEFAN><<<xgrid, 256, xsm, st>>>(xa));
      break;
    default: return VOFP_ERR_INVALID_ARG;
  }
  YArgs ya;
  ya.nx = nx;
  ya.ny = ny;
  ya.nz = nz;
  ya.bc = pl->bc[1];
  ya.fd = pl->ax[1].fd;
  ya.tw = pl->ax[1].tw64;
  ya.quart = pl->ax[1].quart64;
  ya.tx = pl->ytx;
  ya.S = pl->S;
  const dim3 ygrid((nx + ya.tx - 1) / ya.tx, nz);
  const size_t ysm = 2 * (size_t)(ya.tx / 2) * ny * sizeof(double2);
  if (ny > 1) VOFP_LAUNCH(KID_YFWD, st, k_ypass<double, double2, false><<<ygrid, 256, ysm, st>>>(ya));
  ZArgs za;
  za.nx = nx;
  za.ny = ny;
  za.nz = nz;
  za.bcz = pl->bc[2];
  za.ti = pl->zti;
  za.singular = pl->singular;
  za.scale = 1.0 / ((double)nx * ny);
  za.lz = pl->volume / (nx * pl->dx * ny * pl->dy);
  za.lamx = pl->ax[0].lam;
  za.lamy = pl->ax[1].lam;
  za.za = pl->za;
  za.zb = pl->zb;
  za.zc = pl->zc;
  za.dz = pl->dz;
  za.info = stats ? pl->info : nullptr;
  za.S = pl->S;
  const int nvec = pl->bc[2] == VOFP_BC_P ? 3 : 2;
  const dim3 zgrid((nx + za.ti - 1) / za.ti, ny);
  const size_t zsm = (size_t)nvec * za.ti * nz * sizeof(double);
  VOFP_LAUNCH(KID_ZSOLVE, st, k_zsolve64<<<zgrid, 128, zsm, st>>>(za));
  if (ny > 1) VOFP_LAUNCH(KID_YINV, st, k_ypass<double, double2, true><<<ygrid, 256, ysm, st>>>(ya));
  XInvArgs xi;
  xi.nx = nx;
  xi.ny = ny;
  xi.nz = nz;
  xi.bc = pl->bc[0];
  xi.fd = pl->ax[0].fd;
  xi.tw = pl->ax[0].tw64;
  xi.quart = pl->ax[0].quart64;
  xi.pb = pl->xpb;
  xi.S = pl->S;
  xi.p = pout;
  xi.accumulate = 0;
  VOFP_LAUNCH(KID_XINV, st, k_xinv<double, double2><<<xgrid, 256, xsm, st>>>(xi));
  return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

int begin_info(vofp_plan* pl, cudaStream_t st, vofp_info* info) {
  if (!info) return VOFP_OK;
  if (cudaMemsetAsync(pl->info, 0, sizeof(vofp_devinfo), st) != cudaSuccess) return VOFP_ERR_CUDA;
  return VOFP_OK;
}

int finish_info(vofp_plan* pl, cudaStream_t st, vofp_info* info, int status) {
  if (!info) return status;
  vofp_devinfo h;
  if (cudaMemcpyAsync(&h, pl->info, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return VOFP_ERR_CUDA;
  info->compat_defect = pl->singular ? h.compat_defect : 0.0;
  if (status == VOFP_OK && h.nonfinite) status = VOFP_ERR_NONFINITE;
  if (status == VOFP_OK && pl->singular) {
    const double mean_abs = h.abs_sum / pl->volume;
    if (fabs(h.compat_defect) > 1e-12 * mean_abs) status = VOFP_WARN_INCOMPATIBLE_RHS;
  }
  if (status >= 0 && pl->opts.prec == VOFP_FP64) {
    info->rel_residual = 0;
    info->refine_iters = 0;
  }
  info->status = status;
  return status;
}

}  // namespace vofp

extern "C" int vofp_poisson_solve(vofp_plan* pl, const double* f, double* p, void* stream, vofp_info* info) {
  if (!pl || !f || !p) return VOFP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int s = begin_info(pl, st, info);
  if (s) return s;
  if (pl->opts.prec == VOFP_MIXED) {
    s = mixed_solve(pl, RHS_F, nullptr, f, p, st, info);
    return s;
  }
  XArgs xa = {};
  xa.f = f;
  xa.scale = 1.0;
  s = fp64_solve(pl, RHS_F, xa, p, st, info != nullptr);
  return finish_info(pl, st, info, s);
}

__global__ void k_stefan_source(GridDev g, const double* __restrict__ C, const double* __restrict__ mdot,
                                double coef, int mode, double* s) {
  const size_t total = (size_t)g.nx * g.ny * g.nz;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const size_t r = t / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const double3 gc = grad_c_at(g, C, i, j, k, mode);
    s[t] = __ldg(mdot + t) * coef * sqrt(gc.x * gc.x + gc.y * gc.y + gc.z * gc.z);
  }
}

extern "C" int vofp_stefan_source(vofp_plan* pl, const double* C, const double* mdot, double rho1, double rho2,
                                  double* s, void* stream) {
  if (!pl || !C || !mdot || !s || !(rho1 > 0) || !(rho2 > 0) || !std::isfinite(rho1) || !std::isfinite(rho2))
    return VOFP_ERR_INVALID_ARG;
  const GridDev g = grid_dev(pl);
  cudaStream_t st = (cudaStream_t)stream;
  VOFP_LAUNCH(KID_STEFAN, st,
              k_stefan_source<<<grid_blocks((size_t)g.nx * g.ny * g.nz, 256), 256, 0, st>>>(
                  g, C, mdot, 1.0 / rho2 - 1.0 / rho1, pl->opts.grad_mode, s));
  return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

static int project_common(vofp_plan* pl, int mode, XArgs& xa, double* u, double* v, double* w, double dt_over_rho0,
                          double* p, cudaStream_t st, vofp_info* info);

extern "C" int vofp_project(vofp_plan* pl, double* u, double* v, double* w, const double* src, double dt_over_rho0,
                            double* p, void* stream, vofp_info* info) {
  if (!pl || !u || !v || !w || !(dt_over_rho0 > 0) || !std::isfinite(dt_over_rho0)) return VOFP_ERR_INVALID_ARG;
  XArgs xa = {};
  xa.u = u;
  xa.v = v;
  xa.w = w;
  xa.src = src;
  xa.scale = 1.0 / dt_over_rho0;
  return project_common(pl, RHS_DIV, xa, u, v, w, dt_over_rho0, p, (cudaStream_t)stream, info);
}

extern "C" int vofp_project_stefan(vofp_plan* pl, double* u, double* v, double* w, const double* C,
                                   const double* mdot, double rho1, double rho2, double dt_over_rho0, double* p,
                                   void* stream, vofp_info* info) {
  if (!pl || !u || !v || !w || !C || !mdot || !(dt_over_rho0 > 0) || !std::isfinite(dt_over_rho0))
    return VOFP_ERR_INVALID_ARG;
  if (!(rho1 > 0) || !(rho2 > 0) || !std::isfinite(rho1) || !std::isfinite(rho2)) return VOFP_ERR_INVALID_ARG;
  XArgs xa = {};
  xa.u = u;
  xa.v = v;
  xa.w = w;
  xa.C = C;
  xa.mdot = mdot;
  xa.coef = 1.0 / rho2 - 1.0 / rho1;
  xa.grad_mode = pl->opts.grad_mode;
  xa.scale = 1.0 / dt_over_rho0;
  return project_common(pl, RHS_DIV_STEFAN, xa, u, v, w, dt_over_rho0, p, (cudaStream_t)stream, info);
}

static int project_common(vofp_plan* pl, int mode, XArgs& xa, double* u, double* v, double* w, double dt_over_rho0,
                          double* p, cudaStream_t st, vofp_info* info) {
  int s = begin_info(pl, st, info);
  if (s) return s;
  double* pout = p ? p : pl->P;
  if (pl->opts.prec == VOFP_MIXED) {
    s = mixed_solve(pl, mode, &xa, nullptr, pout, st, info);
    if (s < 0) return s;
  } else {
    s = fp64_solve(pl, mode, xa, pout, st, info != nullptr);
    if (s) return s;
  }
  const GridDev g = grid_dev(pl);
  const size_t total = (size_t)nface(g.nx, g.bcx) * g.ny * g.nz + (size_t)g.nx * nface(g.ny, g.bcy) * g.nz +
                       (size_t)g.nx * g.ny * nface(g.nz, g.bcz);
  VOFP_LAUNCH(KID_GRAD, st, k_grad_update<<<grid_blocks(total, 256), 256, 0, st>>>(g, pout, u, v, w, dt_over_rho0));
  const int ls = cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
  if (pl->opts.prec == VOFP_MIXED) {
    if (ls) return ls;
    if (info) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return VOFP_ERR_CUDA;
      info->status = s;
    }
    return s;
  }
  return finish_info(pl, st, info, ls);
}

extern "C" int vofp_extend_liquid_velocity(vofp_plan* pl, const double* u, const double* v, const double* w,
                                           const double* C, const double* mdot, double rho1, double rho2,
                                           double* ue, double* ve, double* we, double* ug, double* vg, double* wg,
                                           double* phi, void* stream, vofp_info* info) {
  if (!pl || !u || !v || !w || !C || !mdot || !ue || !ve || !we) return VOFP_ERR_INVALID_ARG;
  if (!(rho1 > 0) || !(rho2 > 0) || !std::isfinite(rho1) || !std::isfinite(rho2)) return VOFP_ERR_INVALID_ARG;
  const int nug = (ug != nullptr) + (vg != nullptr) + (wg != nullptr);
  if (nug != 0 && nug != 3) return VOFP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int s = begin_info(pl, st, info);
  if (s) return s;
  double* pout = phi ? phi : pl->P;
  XArgs xa = {};
  xa.C = C;
  xa.mdot = mdot;
  xa.coef = 1.0 / rho2 - 1.0 / rho1;
  xa.grad_mode = pl->opts.grad_mode;
  if (pl->opts.prec == VOFP_MIXED) {
    s = mixed_solve(pl, RHS_STEFAN, &xa, nullptr, pout, st, info);
    if (s < 0) return s;
  } else {
    s = fp64_solve(pl, RHS_STEFAN, xa, pout, st, info != nullptr);
    if (s) return s;
  }
  ExtArgs ea;
  ea.g = grid_dev(pl);
  ea.phi = pout;
  ea.u = u;
  ea.v = v;
  ea.w = w;
  ea.C = C;
  ea.mdot = mdot;
  ea.inv_rho1 = 1.0 / rho1;
  ea.grad_mode = pl->opts.grad_mode;
  ea.ue = ue;
  ea.ve = ve;
  ea.we = we;
  ea.ug = ug;
  ea.vg = vg;
  ea.wg = wg;
  const GridDev& g = ea.g;
  const size_t total = (size_t)nface(g.nx, g.bcx) * g.ny * g.nz + (size_t)g.nx * nface(g.ny, g.bcy) * g.nz +
                       (size_t)g.nx * g.ny * nface(g.nz, g.bcz);
  VOFP_LAUNCH(KID_EXTEND_EPI, st, k_extend_epi<<<grid_blocks(total, 256), 256, 0, st>>>(ea));
  const int ls = cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
  if (pl->opts.prec == VOFP_MIXED) {
    if (ls) return ls;
    if (info) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return VOFP_ERR_CUDA;
      info->status = s;
    }
    return s;
  }
  return finish_info(pl, st, info, ls);
}
