// Host orchestration of the FP64 path and the public entry points
// vofp_poisson_solve / vofp_project / vofp_project_stefan / vofp_stefan_source /
// vofp_extend_liquid_velocity / vofp_project_extend.
//
// One solve = x pass (right-hand side fused) -> y pass -> z tridiagonal pass -> inverse y -> inverse x,
// then the face epilogue (§3.2 projection, §3.6 extension).  Every launch goes to the caller's stream.
#include <cmath>
#include <mutex>
#include <set>
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
  g.rdx = 1.0 / pl->dx;
  g.rdy = 1.0 / pl->dy;
  g.rdx2 = g.rdx * g.rdx;
  g.rdy2 = g.rdy * g.rdy;
  g.hrdx = 0.5 * g.rdx;
  g.hrdy = 0.5 * g.rdy;
  g.dz = pl->dz;
  g.hz = pl->hz;
  g.rdz = pl->rdz;
  g.rhz = pl->rhz;
  g.rzc = pl->rzc;
  g.vol = pl->kz;
  g.czp = pl->kz ? pl->kz + pl->n[2] : nullptr;
  g.czm = pl->kz ? pl->kz + 2 * pl->n[2] : nullptr;
  g.czc = pl->kz ? pl->kz + 3 * pl->n[2] : nullptr;
  g.volf = pl->volf;
  g.dzff = pl->dzff;
  return g;
}

static const int kMaxDynSmem = 200 * 1024;

template <typename K>
static void allow_smem(K kern) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

bool first_use_on_device(int which) {
  static std::mutex mu;
  static std::set<std::pair<int, int>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  return done.insert(std::make_pair(dev, which)).second;
}

void init_kernel_attributes_fp64() {
  if (!first_use_on_device(0)) return;
  allow_smem(k_xfwd_f64<RHS_F>);
  allow_smem(k_xfwd_f64<RHS_DIV>);
  allow_smem(k_xfwd<double, double2, RHS_STEFAN>);
  allow_smem(k_xfwd<double, double2, RHS_DIV_STEFAN>);
  allow_smem(k_ypass_f64<false>);
  allow_smem(k_ypass_f64<true>);
  allow_smem(k_xinv_f64<0>);
  allow_smem(k_zsolve<double, double>);
  allow_smem(k_ztab<double, ZF<double>>);
  allow_smem(k_ztab_staged<double, ZF<double>>);
  allow_smem(k_ztab_seg<double, ZF<double>, false>);
  allow_smem(k_ztab_seg<double, ZF<double>, true>);
}

int grid_blocks(size_t total, int threads) {
  size_t b = (total + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

ZArgs z_args(const vofp_plan* pl, bool stats) {
  ZArgs za;
  za.nx = pl->n[0];
  za.ny = pl->n[1];
  za.nz = pl->n[2];
  za.bcz = pl->bc[2];
  za.ti = pl->zti;
  za.singular = pl->singular;
  // the forward x pass (always run) and y pass (run when ny > 1) each return twice the transform
  za.scale = 1.0 / ((double)pl->n[0] * pl->n[1] * 2.0 * (pl->n[1] > 1 ? 2.0 : 1.0));
  za.lz = pl->volume / (pl->n[0] * pl->dx * pl->n[1] * pl->dy);
  za.lamx = pl->ax[0].lam;
  za.lamy = pl->ax[1].lam;
  za.za = pl->za;
  za.zb = pl->zb;
  za.zc = pl->zc;
  za.dz = pl->dz;
  za.info = stats ? pl->info : nullptr;
  za.S = pl->S;
  za.lowthr = -1.0;
  za.skip_conv = nullptr;
  za.skip_k = -1;
  za.tol2 = 0.0;
  return za;
}

ZTabArgs ztab_args(const vofp_plan* pl) {
  ZTabArgs zt;
  zt.Ux = pl->Ux;
  zt.Uy = pl->Uy;
  zt.bcx = pl->bc[0];
  zt.bcy = pl->bc[1];
  zt.tab = pl->ztab;
  zt.za = pl->zaT;
  zt.lowcut = pl->lowcut;
  return zt;
}

int build_z_factors(vofp_plan* pl, cudaStream_t st, bool sync) {
  const ZArgs za = z_args(pl, false);
  const ZTabArgs zt = ztab_args(pl);
  const int n = pl->Ux * pl->Uy;
  const int nb = (n + 127) / 128;
  if (pl->opts.prec == VOFP_MIXED)
    k_zfactor<ZF<float>><<<nb, 128, 0, st>>>(za, zt, (ZF<float>*)pl->ztab);
  else if (pl->opts.prec == VOFP_FF)
    k_zfactor<ZF<ff>><<<nb, 128, 0, st>>>(za, zt, (ZF<ff>*)pl->ztab);
  else
    k_zfactor<ZF<double>><<<nb, 128, 0, st>>>(za, zt, (ZF<double>*)pl->ztab);
  if (cudaGetLastError() != cudaSuccess) return VOFP_ERR_CUDA;
  if (sync && cudaStreamSynchronize(st) != cudaSuccess) return VOFP_ERR_CUDA;
  return VOFP_OK;
}

// The plan's FP64 x transform -- forward (as applied to a right-hand side) or inverse -- of `nlines` lines of
// length nx from `in` into `out` (FP64, line-major).  The tensor-core x passes of the refinement plans take
// their transform matrices from it (identity lines in), so they share every convention of the FFT passes.
int fp64_x_lines(vofp_plan* pl, bool inverse, const double* in, double* out, int nlines, cudaStream_t st) {
  const AxisDev& ax = pl->ax[0];
  const int span = fft_span(ax.fd, ax.blu64);
  int pb = pl->xpb;
  while (pb > 1 && 2 * (size_t)pb * span * sizeof(double2) > 96 * 1024) --pb;
  const int xgrid = xpass_blocks(nlines, 1, pb);
  const size_t xsm = 2 * (size_t)pb * span * sizeof(double2);
  if (!inverse) {
    XArgs xa = {};
    xa.g = grid_dev(pl);
    xa.g.ny = nlines;
    xa.g.nz = 1;
    xa.fd = ax.fd;
    xa.tw = ax.tw64;
    xa.quart = ax.quart64;
    xa.blu = ax.blu64;
    xa.pb = pb;
    xa.S = out;
    xa.f = in;
    xa.scale = 1.0;
    xa.skip_k = -1;
    VOFP_LAUNCH(KID_XFWD, st, k_xfwd_f64<RHS_F><<<xgrid, 256, xsm, st>>>(xa));
  } else {
    XInvArgs xi = {};
    xi.skip_k = -1;
    xi.nx = pl->n[0];
    xi.ny = nlines;
    xi.nz = 1;
    xi.bc = pl->bc[0];
    xi.fd = ax.fd;
    xi.tw = ax.tw64;
    xi.quart = ax.quart64;
    xi.blu = ax.blu64;
    xi.pb = pb;
    xi.S = in;
    xi.p = out;
    xi.accumulate = 0;
    VOFP_LAUNCH(KID_XINV, st, k_xinv_f64<0><<<xgrid, 256, xsm, st>>>(xi));
  }
  return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

// x forward + y forward + z solve + y inverse + x inverse into `pout`.
int fp64_solve(vofp_plan* pl, int mode, XArgs xa, double* pout, cudaStream_t st, bool stats) {
  if (!pl->S) return VOFP_ERR_INVALID_ARG;  // a refinement plan has no FP64 spectrum
  const int nx = pl->n[0], ny = pl->n[1], nz = pl->n[2];
  xa.g = grid_dev(pl);
  xa.fd = pl->ax[0].fd;
  xa.tw = pl->ax[0].tw64;
  xa.quart = pl->ax[0].quart64;
  xa.blu = pl->ax[0].blu64;
  xa.pb = pl->xpb;
  xa.S = pl->S;
  xa.info = stats ? pl->info : nullptr;
  const long npairs = ((long)ny * nz + 1) / 2;
  const int xgrid = (int)((npairs + xa.pb - 1) / xa.pb);
  const size_t xsm = 2 * (size_t)xa.pb * fft_span(xa.fd, xa.blu) * sizeof(double2);
  switch (mode) {
    case RHS_F: VOFP_LAUNCH(KID_XFWD, st, k_xfwd_f64<RHS_F><<<xgrid, 256, xsm, st>>>(xa)); break;
    case RHS_DIV: VOFP_LAUNCH(KID_XFWD_DIV, st, k_xfwd_f64<RHS_DIV><<<xgrid, 256, xsm, st>>>(xa)); break;
    case RHS_STEFAN:
      VOFP_LAUNCH(KID_XFWD_STEFAN, st, k_xfwd<double, double2, RHS_STEFAN><<<xgrid, 256, xsm, st>>>(xa));
      break;
    case RHS_DIV_STEFAN:
      VOFP_LAUNCH(KID_XFWD_DIVSTEF, st, k_xfwd<double, double2, RHS_DIV_STEFAN><<<xgrid, 256, xsm, st>>>(xa));
      break;
    default: return VOFP_ERR_INVALID_ARG;
  }
  YArgs ya = {};
  ya.skip_k = -1;
  ya.nx = nx;
  ya.ny = ny;
  ya.nz = nz;
  ya.bc = pl->bc[1];
  ya.fd = pl->ax[1].fd;
  ya.tw = pl->ax[1].tw64;
  ya.quart = pl->ax[1].quart64;
  ya.blu = pl->ax[1].blu64;
  ya.tx = pl->ytx;
  ya.S = pl->S;
  const dim3 ygrid((nx + ya.tx - 1) / ya.tx, nz);
  const size_t ysm = 2 * (size_t)(ya.tx / 2) * y_ld(fft_span(ya.fd, ya.blu)) * sizeof(double2);
  if (ny > 1 && !ypass_tma_f64(pl, ya, false, st))
    VOFP_LAUNCH(KID_YFWD, st, k_ypass_f64<false><<<ygrid, 256, ysm, st>>>(ya));
  ZArgs za = z_args(pl, stats);
  if (pl->ztab && (pl->zti == -1 || pl->zti == -2)) {  // (only by the autotuner's choice on FP64 plans)
    const dim3 tgrid((nx + kZSegTI - 1) / kZSegTI, ny);
    const size_t sm = ztab_seg_smem(nz, sizeof(double), pl->zti == -2);
    if (pl->zti == -2)
      VOFP_LAUNCH(KID_ZSOLVE, st,
                  (k_ztab_seg<double, ZF<double>, true><<<tgrid, 32 * kZSegW, sm, st>>>(za, ztab_args(pl))));
    else
      VOFP_LAUNCH(KID_ZSOLVE, st,
                  (k_ztab_seg<double, ZF<double>, false><<<tgrid, 32 * kZSegW, sm, st>>>(za, ztab_args(pl))));
  } else if (pl->ztab && pl->zti == 0) {
    const dim3 tgrid((nx + kZStagedTI - 1) / kZStagedTI, ny);
    VOFP_LAUNCH(KID_ZSOLVE, st,
                (k_ztab_staged<double, ZF<double>><<<tgrid, 128, ztab_staged_smem(nz, sizeof(double)), st>>>(
                    za, ztab_args(pl))));
  } else if (pl->ztab) {
    const ZTabShape zs = ztab_shape(pl->zti, nz, sizeof(double));
    const dim3 tgrid((nx + zs.threads - 1) / zs.threads, ny);
    VOFP_LAUNCH(KID_ZSOLVE, st,
                (k_ztab<double, ZF<double>><<<tgrid, zs.threads, zs.smem, st>>>(za, ztab_args(pl), zs.smem_d)));
  } else {
    const int nvec = pl->bc[2] == VOFP_BC_P ? 3 : 2;
    const size_t zsm = (size_t)nvec * za.ti * nz * sizeof(double);
    const dim3 zgrid((nx + za.ti - 1) / za.ti, ny);
    VOFP_LAUNCH(KID_ZSOLVE, st, (k_zsolve<double, double><<<zgrid, 128, zsm, st>>>(za)));
  }
  if (ny > 1 && !ypass_tma_f64(pl, ya, true, st))
    VOFP_LAUNCH(KID_YINV, st, k_ypass_f64<true><<<ygrid, 256, ysm, st>>>(ya));
  XInvArgs xi = {};
  xi.skip_k = -1;
  xi.nx = nx;
  xi.ny = ny;
  xi.nz = nz;
  xi.bc = pl->bc[0];
  xi.fd = pl->ax[0].fd;
  xi.tw = pl->ax[0].tw64;
  xi.quart = pl->ax[0].quart64;
  xi.blu = pl->ax[0].blu64;
  xi.pb = pl->xpb;
  xi.S = pl->S;
  xi.p = pout;
  xi.accumulate = 0;
  VOFP_LAUNCH(KID_XINV, st, k_xinv_f64<0><<<xgrid, 256, xsm, st>>>(xi));
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
  if (status >= 0 && h.timeout) status = VOFP_ERR_TIMEOUT;  // a bounded wait for a tile load gave up
  if (status == VOFP_OK && pl->singular) {
    const double mean_abs = h.abs_sum / pl->volume;
    if (fabs(h.compat_defect) > 1e-12 * mean_abs) status = VOFP_WARN_INCOMPATIBLE_RHS;
  }
  if (status >= 0 && pl->opts.prec == VOFP_FP64) {
    info->rel_residual = 0;
    info->refine_iters = 0;
    info->mean_removed = 0;  // the mean mode is pinned at zero in the z pass: nothing is subtracted
    info->err_estimate = -1.0;  // not estimated (an FP64 plan keeps no copy of the right-hand side)
  }
  info->status = status;
  return status;
}

// Interface geometry into the plan's workspace: s (and n unless `with_n` is false).
static int launch_geometry(vofp_plan* pl, const double* C, const double* mdot, double coef, bool with_n,
                           double* s_out, cudaStream_t st) {
  if ((!s_out || with_n) && ensure_geometry(pl)) return VOFP_ERR_OOM;
  const GridDev g = grid_dev(pl);
  const size_t cells = (size_t)g.nx * g.ny * g.nz;
  double* G = pl->G;
  const int mode = pl->opts.grad_mode;
  double* sp = s_out ? s_out : G;
  double* n0 = with_n ? G + cells : nullptr;
  double* n1 = with_n ? G + 2 * cells : nullptr;
  double* n2 = with_n ? G + 3 * cells : nullptr;
  const int th = g.nx >= 128 ? 128 : 64;
  if (mode == 0 && pl->opts.prec != VOFP_FP64)  // reduced-precision plans: FP32-pair geometry
    VOFP_LAUNCH(KID_STEFAN, st, k_geometry_ff<<<cell_grid(g, th), th, 0, st>>>(g, C, mdot, coef, sp, n0, n1, n2));
  else if (mode == 1)
    VOFP_LAUNCH(KID_STEFAN, st, k_geometry<1><<<cell_grid(g, th), th, 0, st>>>(g, C, mdot, coef, sp, n0, n1, n2));
  else
    VOFP_LAUNCH(KID_STEFAN, st, k_geometry<0><<<cell_grid(g, th), th, 0, st>>>(g, C, mdot, coef, sp, n0, n1, n2));
  return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

// Pressure projection given the right-hand-side mode and inputs in `xa`; runs the correction epilogue.
static int project_common(vofp_plan* pl, int mode, XArgs& xa, double* u, double* v, double* w, double dt_over_rho0,
                          double* p, cudaStream_t st, vofp_info* info) {
  int s = begin_info(pl, st, info);
  if (s) return s;
  double* pout = p ? p : pl->P;
  if (pl->opts.prec != VOFP_FP64) {
    s = mixed_solve(pl, mode, &xa, nullptr, pout, st, info);
    if (s < 0) return s;
  } else {
    s = fp64_solve(pl, mode, xa, pout, st, info != nullptr);
    if (s) return s;
  }
  const GridDev g = grid_dev(pl);
  VOFP_LAUNCH(KID_GRAD, st,
              k_grad_update<<<face_grid(g, 256), 256, 0, st>>>(g, pout, u, v, w, dt_over_rho0,
                                                                      dt_over_rho0 * g.rdx, dt_over_rho0 * g.rdy));
  const int ls = cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
  if (pl->opts.prec != VOFP_FP64) {
    if (ls) return ls;
    if (info) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return VOFP_ERR_CUDA;
      info->status = s;
    }
    return s;
  }
  return finish_info(pl, st, info, ls);
}

// Extension solve on the source already in G[0:cells], normals in G[cells:4 cells]; runs the epilogue.
// rho_ext: the density of the phase whose velocity is extended (rho1, the liquid, for §3.6; rho2, the vapour,
// for the boiling variant of Appendix A), which divides mdot in the interface velocity.
static int extend_common(vofp_plan* pl, const double* u, const double* v, const double* w, const double* mdot,
                         double rho_ext, double* ue, double* ve, double* we, double* ug, double* vg, double* wg,
                         double* phi, cudaStream_t st, vofp_info* info) {
  int s = begin_info(pl, st, info);
  if (s) return s;
  double* pout = phi ? phi : pl->P;
  const size_t cells = (size_t)pl->n[0] * pl->n[1] * pl->n[2];
  XArgs xa = {};
  xa.f = pl->G;
  xa.scale = 1.0;
  if (pl->opts.prec != VOFP_FP64) {
    s = mixed_solve(pl, RHS_F, nullptr, pl->G, pout, st, info);
    if (s < 0) return s;
  } else {
    s = fp64_solve(pl, RHS_F, xa, pout, st, info != nullptr);
    if (s) return s;
  }
  ExtArgs ea;
  ea.g = grid_dev(pl);
  ea.phi = pout;
  ea.u = u;
  ea.v = v;
  ea.w = w;
  ea.mdot = mdot;
  ea.n[0] = pl->G + cells;
  ea.n[1] = pl->G + 2 * cells;
  ea.n[2] = pl->G + 3 * cells;
  ea.quarter_inv_rho1 = 0.25 / rho_ext;
  ea.ue = ue;
  ea.ve = ve;
  ea.we = we;
  ea.ug = ug;
  ea.vg = vg;
  ea.wg = wg;
  VOFP_LAUNCH(KID_EXTEND_EPI, st, k_extend_epi<<<face_grid(ea.g, 256), 256, 0, st>>>(ea));
  const int ls = cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
  if (pl->opts.prec != VOFP_FP64) {
    if (ls) return ls;
    if (info) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return VOFP_ERR_CUDA;
      info->status = s;
    }
    return s;
  }
  return finish_info(pl, st, info, ls);
}

}  // namespace vofp

static bool good_density(double r) { return r > 0 && std::isfinite(r); }

extern "C" int vofp_poisson_solve(vofp_plan* pl, const double* f, double* p, void* stream, vofp_info* info) {
  if (!pl || !f || !p) return VOFP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int s = begin_info(pl, st, info);
  if (s) return s;
  if (pl->opts.prec != VOFP_FP64) return mixed_solve(pl, RHS_F, nullptr, f, p, st, info);
  XArgs xa = {};
  xa.f = f;
  xa.scale = 1.0;
  s = fp64_solve(pl, RHS_F, xa, p, st, info != nullptr);
  return finish_info(pl, st, info, s);
}

extern "C" int vofp_stefan_source(vofp_plan* pl, const double* C, const double* mdot, double rho1, double rho2,
                                  double* s, void* stream) {
  if (!pl || !C || !mdot || !s || !good_density(rho1) || !good_density(rho2)) return VOFP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return launch_geometry(pl, C, mdot, 1.0 / rho2 - 1.0 / rho1, false, s, st);
}

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

extern "C" int vofp_project_vd(vofp_plan* pl, double* u, double* v, double* w, const double* src, const double* C,
                               const double* p_n, const double* p_nm1, double dt, double dt_prev, double rho1,
                               double rho2, double* p, void* stream, vofp_info* info) {
  if (!pl || !u || !v || !w || !C || !p_n || !(dt > 0) || !std::isfinite(dt)) return VOFP_ERR_INVALID_ARG;
  if (p_nm1 && (!(dt_prev > 0) || !std::isfinite(dt_prev))) return VOFP_ERR_INVALID_ARG;
  if (!good_density(rho1) || !good_density(rho2)) return VOFP_ERR_INVALID_ARG;
  const double rho0 = rho1 < rho2 ? rho1 : rho2;
  cudaStream_t st = (cudaStream_t)stream;
  VdArgs va;
  va.g = grid_dev(pl);
  va.pn = p_n;
  va.pm = p_nm1;
  va.r = p_nm1 ? dt / dt_prev : 0.0;
  va.opr = 1.0 + va.r;
  va.C = C;
  va.half_drho = 0.5 * (rho1 - rho2);
  va.rho2 = rho2;
  va.dt = dt;
  va.dt_over_rho0 = dt / rho0;
  va.u = u;
  va.v = v;
  va.w = w;
  VOFP_LAUNCH(KID_VD, st, k_vd_predict<<<face_grid(va.g, 256), 256, 0, st>>>(va));
  if (cudaGetLastError() != cudaSuccess) return VOFP_ERR_CUDA;
  return vofp_project(pl, u, v, w, src, dt / rho0, p, stream, info);
}

extern "C" int vofp_project_stefan(vofp_plan* pl, double* u, double* v, double* w, const double* C,
                                   const double* mdot, double rho1, double rho2, double dt_over_rho0, double* p,
                                   void* stream, vofp_info* info) {
  if (!pl || !u || !v || !w || !C || !mdot || !(dt_over_rho0 > 0) || !std::isfinite(dt_over_rho0))
    return VOFP_ERR_INVALID_ARG;
  if (!good_density(rho1) || !good_density(rho2)) return VOFP_ERR_INVALID_ARG;
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

extern "C" int vofp_extend_liquid_velocity(vofp_plan* pl, const double* u, const double* v, const double* w,
                                           const double* C, const double* mdot, double rho1, double rho2,
                                           double* ue, double* ve, double* we, double* ug, double* vg, double* wg,
                                           double* phi, void* stream, vofp_info* info) {
  if (!pl || !u || !v || !w || !C || !mdot || !ue || !ve || !we) return VOFP_ERR_INVALID_ARG;
  if (!good_density(rho1) || !good_density(rho2)) return VOFP_ERR_INVALID_ARG;
  const int nug = (ug != nullptr) + (vg != nullptr) + (wg != nullptr);
  if (nug != 0 && nug != 3) return VOFP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int gs = launch_geometry(pl, C, mdot, 1.0 / rho2 - 1.0 / rho1, ug != nullptr, nullptr, st);
  if (gs) return gs;
  return extend_common(pl, u, v, w, mdot, rho1, ue, ve, we, ug, vg, wg, phi, st, info);
}

extern "C" int vofp_extend_vapour_velocity(vofp_plan* pl, const double* u, const double* v, const double* w,
                                           const double* C, const double* mdot, double rho1, double rho2,
                                           double* ue, double* ve, double* we, double* ug, double* vg, double* wg,
                                           double* phi, void* stream, vofp_info* info) {
  if (!pl || !u || !v || !w || !C || !mdot || !ue || !ve || !we) return VOFP_ERR_INVALID_ARG;
  if (!good_density(rho1) || !good_density(rho2)) return VOFP_ERR_INVALID_ARG;
  const int nug = (ug != nullptr) + (vg != nullptr) + (wg != nullptr);
  if (nug != 0 && nug != 3) return VOFP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int gs = launch_geometry(pl, C, mdot, 1.0 / rho2 - 1.0 / rho1, ug != nullptr, nullptr, st);
  if (gs) return gs;
  return extend_common(pl, u, v, w, mdot, rho2, ue, ve, we, ug, vg, wg, phi, st, info);
}

extern "C" int vofp_project_extend(vofp_plan* pl, double* u, double* v, double* w, const double* C,
                                   const double* mdot, double rho1, double rho2, double dt_over_rho0, double* p,
                                   double* ue, double* ve, double* we, double* ug, double* vg, double* wg,
                                   double* phi, void* stream, vofp_info* info) {
  if (!pl || !u || !v || !w || !C || !mdot || !ue || !ve || !we) return VOFP_ERR_INVALID_ARG;
  if (!(dt_over_rho0 > 0) || !std::isfinite(dt_over_rho0) || !good_density(rho1) || !good_density(rho2))
    return VOFP_ERR_INVALID_ARG;
  const int nug = (ug != nullptr) + (vg != nullptr) + (wg != nullptr);
  if (nug != 0 && nug != 3) return VOFP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int gs = launch_geometry(pl, C, mdot, 1.0 / rho2 - 1.0 / rho1, ug != nullptr, nullptr, st);
  if (gs) return gs;
  XArgs xa = {};
  xa.u = u;
  xa.v = v;
  xa.w = w;
  xa.src = pl->G;
  xa.scale = 1.0 / dt_over_rho0;
  vofp_info i1;
  int s1 = project_common(pl, RHS_DIV, xa, u, v, w, dt_over_rho0, p, st, info ? &i1 : nullptr);
  if (s1 < 0) return s1;
  int s2 = extend_common(pl, u, v, w, mdot, rho1, ue, ve, we, ug, vg, wg, phi, st, info);
  if (s2 < 0) return s2;
  if (info) {
    // report the projection's defect and gauge shift, the worse of the two statuses, residuals and error
    // estimates
    info->compat_defect = i1.compat_defect;
    info->mean_removed = i1.mean_removed;
    if (i1.rel_residual > info->rel_residual) info->rel_residual = i1.rel_residual;
    if (i1.err_estimate > info->err_estimate) info->err_estimate = i1.err_estimate;
    info->refine_iters += i1.refine_iters;
    info->status = s1 > s2 ? s1 : s2;
  }
  return s1 > s2 ? s1 : s2;
}

// ---- the droplet step on host buffers, transfers overlapped with compute ------------------------------------

namespace vofp {

struct HostStep {
  double* buf;  // one allocation: u, v, w, ue, ve, we, ug, vg, wg (faces), C, mdot, p, phi (cells)
  double *u, *v, *w, *ue, *ve, *we, *ug, *vg, *wg, *C, *mdot, *p, *phi;
  size_t nu, nv, nw, cells;
  cudaStream_t sin, sout;
  cudaEvent_t start, in_cm, in_uvw, proj, ext, out;
};

static int ensure_host_step(vofp_plan* pl, HostStep** out) {
  if (pl->hstep) {
    *out = (HostStep*)pl->hstep;
    return VOFP_OK;
  }
  HostStep* h = new HostStep();
  const int nx = pl->n[0], ny = pl->n[1], nz = pl->n[2];
  h->nu = (size_t)nface(nx, pl->bc[0]) * ny * nz;
  h->nv = (size_t)nx * nface(ny, pl->bc[1]) * nz;
  h->nw = (size_t)nx * ny * nface(nz, pl->bc[2]);
  h->cells = (size_t)nx * ny * nz;
  const size_t faces = h->nu + h->nv + h->nw;
  if (device_alloc((void**)&h->buf, sizeof(double) * (3 * faces + 4 * h->cells)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return VOFP_ERR_OOM;
  }
  double* q = h->buf;
  double** f3[3][3] = {{&h->u, &h->v, &h->w}, {&h->ue, &h->ve, &h->we}, {&h->ug, &h->vg, &h->wg}};
  for (int s = 0; s < 3; ++s) {
    *f3[s][0] = q;
    q += h->nu;
    *f3[s][1] = q;
    q += h->nv;
    *f3[s][2] = q;
    q += h->nw;
  }
  h->C = q;
  h->mdot = q + h->cells;
  h->p = q + 2 * h->cells;
  h->phi = q + 3 * h->cells;
  cudaStreamCreateWithFlags(&h->sin, cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&h->sout, cudaStreamNonBlocking);
  cudaEvent_t* evs[6] = {&h->start, &h->in_cm, &h->in_uvw, &h->proj, &h->ext, &h->out};
  for (cudaEvent_t* e : evs) cudaEventCreateWithFlags(e, cudaEventDisableTiming);
  pl->bytes += sizeof(double) * (3 * faces + 4 * h->cells);
  pl->hstep = h;
  *out = h;
  return VOFP_OK;
}

void free_host_step(vofp_plan* pl) {
  HostStep* h = (HostStep*)pl->hstep;
  if (!h) return;
  cudaFree(h->buf);
  cudaStreamDestroy(h->sin);
  cudaStreamDestroy(h->sout);
  cudaEvent_t evs[6] = {h->start, h->in_cm, h->in_uvw, h->proj, h->ext, h->out};
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
  delete h;
  pl->hstep = nullptr;
}

}  // namespace vofp

static int h2d(double* d, const double* h, size_t n, cudaStream_t s) {
  return cudaMemcpyAsync(d, h, sizeof(double) * n, cudaMemcpyHostToDevice, s) == cudaSuccess ? 0 : 1;
}
static int d2h(double* h, const double* d, size_t n, cudaStream_t s) {
  return cudaMemcpyAsync(h, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s) == cudaSuccess ? 0 : 1;
}

extern "C" int vofp_project_extend_host(vofp_plan* pl, const double* u, const double* v, const double* w,
                                        const double* C, const double* mdot, double rho1, double rho2,
                                        double dt_over_rho0, double* u_out, double* v_out, double* w_out,
                                        double* p_out, double* ug, double* vg, double* wg, void* stream) {
  if (!pl || !u || !v || !w || !C || !mdot || !u_out || !v_out || !w_out || !p_out || !ug || !vg || !wg)
    return VOFP_ERR_INVALID_ARG;
  if (!(dt_over_rho0 > 0) || !std::isfinite(dt_over_rho0) || !good_density(rho1) || !good_density(rho2))
    return VOFP_ERR_INVALID_ARG;
  HostStep* h;
  int s = ensure_host_step(pl, &h);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // inputs on the copy-in stream, after whatever the caller queued before: C and mdot first (the geometry
  // pass needs only them), then the velocities
  int e = cudaEventRecord(h->start, st) != cudaSuccess;
  e |= cudaStreamWaitEvent(h->sin, h->start, 0) != cudaSuccess;
  e |= h2d(h->C, C, h->cells, h->sin) | h2d(h->mdot, mdot, h->cells, h->sin);
  e |= cudaEventRecord(h->in_cm, h->sin) != cudaSuccess;
  e |= h2d(h->u, u, h->nu, h->sin) | h2d(h->v, v, h->nv, h->sin) | h2d(h->w, w, h->nw, h->sin);
  e |= cudaEventRecord(h->in_uvw, h->sin) != cudaSuccess;
  if (e) return VOFP_ERR_CUDA;
  // compute on the caller's stream: geometry while the velocities arrive, then the projection
  e |= cudaStreamWaitEvent(st, h->in_cm, 0) != cudaSuccess;
  const int gs = launch_geometry(pl, h->C, h->mdot, 1.0 / rho2 - 1.0 / rho1, true, nullptr, st);
  if (gs) return gs;
  e |= cudaStreamWaitEvent(st, h->in_uvw, 0) != cudaSuccess;
  XArgs xa = {};
  xa.u = h->u;
  xa.v = h->v;
  xa.w = h->w;
  xa.src = pl->G;
  xa.scale = 1.0 / dt_over_rho0;
  const int s1 = project_common(pl, RHS_DIV, xa, h->u, h->v, h->w, dt_over_rho0, h->p, st, nullptr);
  if (s1 < 0) return s1;
  // the projected velocities and p leave on the copy-out stream while the extension solve runs
  e |= cudaEventRecord(h->proj, st) != cudaSuccess;
  e |= cudaStreamWaitEvent(h->sout, h->proj, 0) != cudaSuccess;
  e |= d2h(u_out, h->u, h->nu, h->sout) | d2h(v_out, h->v, h->nv, h->sout) | d2h(w_out, h->w, h->nw, h->sout);
  e |= d2h(p_out, h->p, h->cells, h->sout);
  const int s2 = extend_common(pl, h->u, h->v, h->w, h->mdot, rho1, h->ue, h->ve, h->we, h->ug, h->vg, h->wg,
                               h->phi, st, nullptr);
  if (s2 < 0) return s2;
  e |= cudaEventRecord(h->ext, st) != cudaSuccess;
  e |= cudaStreamWaitEvent(h->sout, h->ext, 0) != cudaSuccess;
  e |= d2h(ug, h->ug, h->nu, h->sout) | d2h(vg, h->vg, h->nv, h->sout) | d2h(wg, h->wg, h->nw, h->sout);
  // the caller's stream completes only after the results have arrived
  e |= cudaEventRecord(h->out, h->sout) != cudaSuccess;
  e |= cudaStreamWaitEvent(st, h->out, 0) != cudaSuccess;
  if (e) return VOFP_ERR_CUDA;
  return s1 > s2 ? s1 : s2;
}
