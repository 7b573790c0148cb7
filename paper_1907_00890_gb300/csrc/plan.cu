// Plan creation: validation, eigenvalue / twiddle / z-coefficient tables, workspace, launch shapes.
//
// Eigenvalues of the 1-D MAC second-difference operators (uniform spacing h, n cells; §3 grid, §3.2
// boundary conditions, ghost cell = p for N, -p for D):
//   periodic : -(4/h^2) sin^2(pi m / n) for both parts of Fourier mode m,
//   NN       : -(4/h^2) sin^2(pi m / (2n)),
//   DD       : -(4/h^2) sin^2(pi (m+1) / (2n)).
// z keeps its tridiagonal rows: a_k = 1/(dz_k h_{k-1/2}), c_k = 1/(dz_k h_{k+1/2}), b_k = -(a_k + c_k); an N
// end folds the outer coupling into the diagonal (+), a D end subtracts it (-), a periodic axis wraps.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "solve_internal.h"
#include "vofp_internal.cuh"

namespace vofp {

void factor_radices(int n, FftDesc* fd) {
  fd->n = n;
  fd->nst = 0;
  int m = n, e = 0;
  while (m % 2 == 0) {
    m /= 2;
    ++e;
  }
  // powers of two: radix 8 where possible, the remainder as 4 (or 4*4 instead of 8*2)
  int n8 = e / 3, rem = e % 3;
  if (rem == 1 && n8 > 0) {
    --n8;
    fd->radix[fd->nst++] = 4;
    fd->radix[fd->nst++] = 4;
  } else if (rem == 1) {
    fd->radix[fd->nst++] = 2;
  } else if (rem == 2) {
    fd->radix[fd->nst++] = 4;
  }
  for (int i = 0; i < n8; ++i) fd->radix[fd->nst++] = 8;
  const int small[2] = {3, 5};
  for (int s = 0; s < 2; ++s) {
    while (m % small[s] == 0) {
      m /= small[s];
      fd->radix[fd->nst++] = small[s];
    }
  }
  for (int p = 7; m > 1; p += 2) {
    while (m % p == 0) {
      m /= p;
      fd->radix[fd->nst++] = p;
    }
    if ((long long)p * p > m && m > 1) {
      fd->radix[fd->nst++] = m;
      m = 1;
    }
  }
}

static std::atomic<unsigned long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

}  // namespace vofp

using namespace vofp;

extern "C" unsigned long long vofp_launch_count(void) { return g_launches.load(); }

static const double kPi = 3.14159265358979323846;

extern "C" void vofp_opts_default(vofp_opts* opt) {
  if (!opt) return;
  opt->prec = VOFP_FP64;
  opt->tol = 1e-10;
  opt->max_refine = 6;
  opt->grad_mode = 0;
  opt->tune = 0;
}

extern "C" const char* vofp_error_string(int s) {
  switch (s) {
    case VOFP_OK: return "ok";
    case VOFP_WARN_INCOMPATIBLE_RHS: return "warning: right-hand side incompatible with the singular operator (mean removed)";
    case VOFP_WARN_NOT_CONVERGED: return "warning: mixed-precision refinement did not reach the tolerance";
    case VOFP_ERR_INVALID_ARG: return "invalid argument";
    case VOFP_ERR_UNSUPPORTED: return "unsupported configuration";
    case VOFP_ERR_OOM: return "out of device memory";
    case VOFP_ERR_CUDA: return "CUDA error";
    case VOFP_ERR_TIMEOUT: return "timed out";
    case VOFP_ERR_BUSY: return "busy: over the memory budget";
    case VOFP_ERR_NONFINITE: return "non-finite values in the result";
    case VOFP_ERR_TOO_LARGE: return "problem larger than the static scratch of the allocation-free solve";
    default: return "unknown status";
  }
}

static double eig_1d(int bc, int n, double h, int q) {
  int m;
  double arg;
  if (bc == VOFP_BC_P) {
    m = (q + 1) / 2;
    arg = kPi * m / n;
  } else if (bc == VOFP_BC_NN) {
    arg = kPi * q / (2.0 * n);
  } else {
    arg = kPi * (q + 1) / (2.0 * n);
  }
  const double s = std::sin(arg);
  return -4.0 / (h * h) * s * s;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" int vofp_plan_create(int nx, int ny, int nz, double dx, double dy, const double* dz, const int bc[3],
                                const vofp_opts* opt, vofp_plan** out) {
  if (!out || !dz || !bc) return VOFP_ERR_INVALID_ARG;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy))
    return VOFP_ERR_INVALID_ARG;
  if ((long long)nx * ny * nz > (1LL << 31) - 1) return VOFP_ERR_UNSUPPORTED;
  if (nx > 4096 || ny > 4096 || nz > 4096) return VOFP_ERR_UNSUPPORTED;
  for (int a = 0; a < 3; ++a)
    if (bc[a] < VOFP_BC_P || bc[a] > VOFP_BC_DN) return VOFP_ERR_INVALID_ARG;
  if (bc[0] > VOFP_BC_DD || bc[1] > VOFP_BC_DD) return VOFP_ERR_UNSUPPORTED;
  for (int k = 0; k < nz; ++k)
    if (!(dz[k] > 0) || !std::isfinite(dz[k])) return VOFP_ERR_INVALID_ARG;
  vofp_opts o;
  vofp_opts_default(&o);
  if (opt) o = *opt;
  if (o.prec != VOFP_FP64 && o.prec != VOFP_MIXED) return VOFP_ERR_INVALID_ARG;
  if (o.prec == VOFP_MIXED) return VOFP_ERR_UNSUPPORTED;
  if (o.grad_mode != 0 && o.grad_mode != 1) return VOFP_ERR_INVALID_ARG;
  if (o.max_refine < 1) o.max_refine = 1;
  if (!(o.tol > 0)) o.tol = 1e-10;

  vofp_plan* p = (vofp_plan*)calloc(1, sizeof(vofp_plan));
  if (!p) return VOFP_ERR_OOM;
  p->n[0] = nx;
  p->n[1] = ny;
  p->n[2] = nz;
  for (int a = 0; a < 3; ++a) p->bc[a] = bc[a];
  p->dx = dx;
  p->dy = dy;
  p->opts = o;
  cudaGetDevice(&p->device);
  p->dz_host = (double*)malloc(sizeof(double) * nz);
  memcpy(p->dz_host, dz, sizeof(double) * nz);
  auto is_nd = [](int b) { return b == VOFP_BC_P || b == VOFP_BC_NN; };
  p->singular = is_nd(bc[0]) && is_nd(bc[1]) && is_nd(bc[2]);
  double lz = 0;
  for (int k = 0; k < nz; ++k) lz += dz[k];
  p->volume = nx * dx * ny * dy * lz;

  // ---- host tables ----
  const int nn[2] = {nx, ny};
  const double hh[2] = {dx, dy};
  std::vector<double> lam[2];
  std::vector<double2> tw[2], quart[2];
  std::vector<float2> tw32[2], quart32[2];
  for (int a = 0; a < 2; ++a) {
    const int n = nn[a];
    lam[a].resize(n);
    tw[a].resize(n);
    quart[a].resize(n);
    tw32[a].resize(n);
    quart32[a].resize(n);
    for (int q = 0; q < n; ++q) {
      lam[a][q] = eig_1d(bc[a], n, hh[a], q);
      const double t = -2.0 * kPi * q / n;
      tw[a][q] = make_double2(std::cos(t), std::sin(t));
      const double u = -kPi * q / (2.0 * n);
      quart[a][q] = make_double2(std::cos(u), std::sin(u));
      tw32[a][q] = make_float2((float)tw[a][q].x, (float)tw[a][q].y);
      quart32[a][q] = make_float2((float)quart[a][q].x, (float)quart[a][q].y);
    }
    factor_radices(n, &p->ax[a].fd);
    p->ax[a].n = n;
    p->ax[a].bc = bc[a];
  }
  std::vector<double> za(nz), zb(nz), zc(nz), hz(nz + 1);
  const bool zper = bc[2] == VOFP_BC_P;
  const double hper = 0.5 * (dz[nz - 1] + dz[0]);
  for (int k = 0; k <= nz; ++k) {
    if (k == 0)
      hz[k] = zper ? hper : dz[0];
    else if (k == nz)
      hz[k] = zper ? hper : dz[nz - 1];
    else
      hz[k] = 0.5 * (dz[k - 1] + dz[k]);
  }
  for (int k = 0; k < nz; ++k) {
    const double a = 1.0 / (dz[k] * hz[k]);
    const double c = 1.0 / (dz[k] * hz[k + 1]);
    double b = -(a + c);
    double aa = a, cc = c;
    if (!zper && k == 0) {
      b += (bc[2] == VOFP_BC_NN || bc[2] == VOFP_BC_ND) ? a : -a;
      aa = 0;
    }
    if (!zper && k == nz - 1) {
      b += (bc[2] == VOFP_BC_NN || bc[2] == VOFP_BC_DN) ? c : -c;
      cc = 0;
    }
    za[k] = aa;
    zb[k] = b;
    zc[k] = cc;
  }

  // ---- one device block for all tables ----
  size_t off = 0;
  size_t o_lam[2], o_tw[2], o_q[2], o_tw32[2], o_q32[2];
  for (int a = 0; a < 2; ++a) {
    o_lam[a] = off;
    off = align256(off + sizeof(double) * nn[a]);
    o_tw[a] = off;
    off = align256(off + sizeof(double2) * nn[a]);
    o_q[a] = off;
    off = align256(off + sizeof(double2) * nn[a]);
    o_tw32[a] = off;
    off = align256(off + sizeof(float2) * nn[a]);
    o_q32[a] = off;
    off = align256(off + sizeof(float2) * nn[a]);
  }
  const size_t o_za = off;
  off = align256(off + sizeof(double) * nz);
  const size_t o_zb = off;
  off = align256(off + sizeof(double) * nz);
  const size_t o_zc = off;
  off = align256(off + sizeof(double) * nz);
  const size_t o_dz = off;
  off = align256(off + sizeof(double) * nz);
  const size_t o_hz = off;
  off = align256(off + sizeof(double) * (nz + 1));
  const size_t o_info = off;
  off = align256(off + sizeof(vofp_devinfo));
  const size_t table_bytes = off;

  std::vector<unsigned char> host(table_bytes, 0);
  for (int a = 0; a < 2; ++a) {
    memcpy(&host[o_lam[a]], lam[a].data(), sizeof(double) * nn[a]);
    memcpy(&host[o_tw[a]], tw[a].data(), sizeof(double2) * nn[a]);
    memcpy(&host[o_q[a]], quart[a].data(), sizeof(double2) * nn[a]);
    memcpy(&host[o_tw32[a]], tw32[a].data(), sizeof(float2) * nn[a]);
    memcpy(&host[o_q32[a]], quart32[a].data(), sizeof(float2) * nn[a]);
  }
  memcpy(&host[o_za], za.data(), sizeof(double) * nz);
  memcpy(&host[o_zb], zb.data(), sizeof(double) * nz);
  memcpy(&host[o_zc], zc.data(), sizeof(double) * nz);
  memcpy(&host[o_dz], dz, sizeof(double) * nz);
  memcpy(&host[o_hz], hz.data(), sizeof(double) * (nz + 1));

  const size_t cells = (size_t)nx * ny * nz;
  const bool mixed = o.prec == VOFP_MIXED;
  size_t ws = 0;
  const size_t o_S = ws;
  ws = align256(ws + sizeof(double) * cells);
  const size_t o_P = ws;
  ws = align256(ws + sizeof(double) * cells);
  size_t o_S32 = 0, o_F = 0, o_R = 0;
  if (mixed) {
    o_S32 = ws;
    ws = align256(ws + sizeof(float) * cells);
    o_F = ws;
    ws = align256(ws + sizeof(double) * cells);
    o_R = ws;
    ws = align256(ws + sizeof(double) * cells);
  }
  void* block = nullptr;
  if (cudaMalloc(&block, table_bytes + ws) != cudaSuccess) {
    cudaGetLastError();
    free(p->dz_host);
    free(p);
    return VOFP_ERR_OOM;
  }
  if (cudaMemcpy(block, host.data(), table_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(block);
    free(p->dz_host);
    free(p);
    return VOFP_ERR_CUDA;
  }
  unsigned char* b = (unsigned char*)block;
  p->table_block = block;
  p->bytes = table_bytes + ws;
  for (int a = 0; a < 2; ++a) {
    p->ax[a].lam = (const double*)(b + o_lam[a]);
    p->ax[a].tw64 = (const double2*)(b + o_tw[a]);
    p->ax[a].quart64 = (const double2*)(b + o_q[a]);
    p->ax[a].tw32 = (const float2*)(b + o_tw32[a]);
    p->ax[a].quart32 = (const float2*)(b + o_q32[a]);
  }
  p->za = (double*)(b + o_za);
  p->zb = (double*)(b + o_zb);
  p->zc = (double*)(b + o_zc);
  p->dz = (double*)(b + o_dz);
  p->hz = (double*)(b + o_hz);
  p->info = (vofp_devinfo*)(b + o_info);
  unsigned char* w = b + table_bytes;
  p->S = (double*)(w + o_S);
  p->P = (double*)(w + o_P);
  p->S32 = mixed ? (float*)(w + o_S32) : nullptr;
  p->F = mixed ? (double*)(w + o_F) : nullptr;
  p->R = mixed ? (double*)(w + o_R) : nullptr;

  // launch shapes (defaults; the tuner may override them)
  p->xpb = nx >= 1024 ? 1 : (1024 / nx > 16 ? 16 : 1024 / nx);
  if (p->xpb < 1) p->xpb = 1;
  int tx = 16;
  while (tx > 2 && (size_t)16 * tx * ny > 96 * 1024) tx -= 2;
  p->ytx = tx;
  const int nvec = zper ? 3 : 2;
  int ti = 32;
  while (ti > 1 && (size_t)nvec * ti * nz * sizeof(double) > 96 * 1024) ti /= 2;
  p->zti = ti;
  init_kernel_attributes_fp64();
  init_kernel_attributes_mixed();
  *out = p;
  return VOFP_OK;
}

extern "C" void vofp_plan_destroy(vofp_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  cudaFree(p->table_block);
  cudaSetDevice(cur);
  free(p->dz_host);
  free(p);
}

extern "C" size_t vofp_plan_workspace_bytes(const vofp_plan* p) { return p ? p->bytes : 0; }
