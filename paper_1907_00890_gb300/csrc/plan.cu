// Plan creation: validation, eigenvalue / twiddle / z-coefficient tables, workspace, launch shapes.
//
// Eigenvalues of the 1-D MAC second-difference operators (uniform spacing h, n cells; §3 grid, §3.2
// boundary conditions, ghost cell = p for N, -p for D):
//   periodic : -(4/h^2) sin^2(pi m / n) for both parts of Fourier mode m,
//   NN       : -(4/h^2) sin^2(pi m / (2n)),
//   DD       : -(4/h^2) sin^2(pi (m+1) / (2n)).
// z keeps its tridiagonal rows: a_k = 1/(dz_k h_{k-1/2}), c_k = 1/(dz_k h_{k+1/2}), b_k = -(a_k + c_k); an N
// end folds the outer coupling into the diagonal (+), a D end subtracts it (-), a periodic axis wraps.
//
// Creation is split in two: plan_prepare validates and builds every table on the host (and reports the
// device bytes the plan needs), plan_bind places the plan in device memory -- its own cudaMalloc, or a block
// handed in by the caller (the server's arena) with asynchronous uploads on a stream.
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "solve_internal.h"
#include "zsolve.cuh"
#include "vofp_internal.cuh"

namespace vofp {

// The direct stages of a length-n transform (radices 8, 4, 2, 3, 5, then 7, 11, 13 and any remaining prime).
static void factor_radices_direct(int n, FftDesc* fd) {
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

void factor_radices(int n, FftDesc* fd) {
  factor_radices_direct(n, fd);
  // a prime factor above 13 (no hand-written butterfly) makes a stage cost O(p) per point: such lengths also
  // get the Bluestein form
  int maxp = 1;
  for (int s = 0; s < fd->nst; ++s)
    if (fd->radix[s] > maxp && fd->radix[s] != 8 && fd->radix[s] != 4) maxp = fd->radix[s];
  fd->bm = 0;
  fd->bst = 0;
  if (maxp > 13 && 2 * n - 1 <= 4096) {  // (longer lines would not fit in shared memory twice over)
    // the shortest convolution length >= 2n - 1 of the form c * 2^k, c in {1, 3, 5, 15}: all its stages have
    // hand-written butterflies
    int M = 0;
    const int cs[4] = {1, 3, 5, 15};
    for (int c : cs) {
      int m = c;
      while (m < 2 * n - 1) m *= 2;
      if (M == 0 || m < M) M = m;
    }
    FftDesc b;
    factor_radices_direct(M, &b);
    fd->bm = M;
    fd->bst = b.nst;
    for (int s = 0; s < b.nst; ++s) fd->bradix[s] = b.radix[s];
  }
}

// In-place forward DFT in FP64 on the host for lengths whose prime factors are 2, 3 and 5 (recursive
// decimation in time), for the Bluestein kernel spectrum.  W holds e^{-2 pi i t / N} for the top-level
// length N; a sub-transform of length n = N / s uses every s-th entry.
static void host_fft(std::vector<std::complex<double>>& x, const std::vector<std::complex<double>>& W) {
  const size_t n = x.size();
  if (n <= 1) return;
  const size_t s = W.size() / n;
  const size_t r = n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : 5);
  const size_t m = n / r;
  std::vector<std::vector<std::complex<double>>> sub(r, std::vector<std::complex<double>>(m));
  for (size_t q = 0; q < r; ++q)
    for (size_t j = 0; j < m; ++j) sub[q][j] = x[j * r + q];
  for (auto& v : sub) host_fft(v, W);
  for (size_t k = 0; k < n; ++k) {
    std::complex<double> acc(0.0, 0.0);
    for (size_t q = 0; q < r; ++q) acc += W[((q * k) % n) * s] * sub[q][k % m];
    x[k] = acc;
  }
}

// Bluestein tables of an axis (see fft_smem): chirp (n), kernel spectrum / M (M), M-point twiddles (M).
static std::vector<double2> bluestein_tables(const FftDesc& fd) {
  const int n = fd.n, M = fd.bm;
  std::vector<double2> t((size_t)n + 2 * (size_t)M);
  std::vector<std::complex<double>> h(M, std::complex<double>(0.0, 0.0));
  for (int j = 0; j < n; ++j) {
    const long long r = ((long long)j * j) % (2LL * n);  // exact reduction of j^2 modulo 2n
    const double ang = -3.14159265358979323846 * (double)r / (double)n;
    t[j] = make_double2(std::cos(ang), std::sin(ang));
    const std::complex<double> c(std::cos(ang), -std::sin(ang));  // conj(w_j)
    h[j] = c;
    if (j > 0) h[M - j] = c;
  }
  std::vector<std::complex<double>> W(M);
  for (int q = 0; q < M; ++q) {
    const double ang = -2.0 * 3.14159265358979323846 * q / M;
    W[q] = std::complex<double>(std::cos(ang), std::sin(ang));
  }
  host_fft(h, W);
  for (int k = 0; k < M; ++k) t[n + k] = make_double2(h[k].real() / M, h[k].imag() / M);
  for (int q = 0; q < M; ++q) {
    const double ang = -2.0 * 3.14159265358979323846 * q / M;
    t[n + M + q] = make_double2(std::cos(ang), std::sin(ang));
  }
  return t;
}

static std::atomic<unsigned long long> g_launches{0};
// While this thread captures a graph its launches are not executions: count them apart (they are added
// once per replay instead) and do not trace them.
static thread_local int t_capturing = 0;
static thread_local unsigned long long t_captured = 0;
void note_launches(int n) {
  if (t_capturing)
    t_captured += (unsigned long long)n;
  else
    g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
}
bool capturing() { return t_capturing != 0; }
void capture_begin() {
  t_capturing = 1;
  t_captured = 0;
}
unsigned long long capture_end() {
  t_capturing = 0;
  return t_captured;
}

static const double kPi = 3.14159265358979323846;

static double eig_1d(int bc, int n, double h, int q) {
  double arg;
  if (bc == VOFP_BC_P)
    arg = kPi * ((q + 1) / 2) / n;
  else if (bc == VOFP_BC_NN)
    arg = kPi * q / (2.0 * n);
  else if (bc == VOFP_BC_DD)
    arg = kPi * (q + 1) / (2.0 * n);
  else  // ND, DN: cos / sin (pi (2q+1)(2j+1) / (4n))
    arg = kPi * (2 * q + 1) / (4.0 * n);
  const double s = std::sin(arg);
  return -4.0 / (h * h) * s * s;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static int zdistinct(int n, int bc) { return bc == VOFP_BC_P ? n / 2 + 1 : n; }

// Validate, fill the host-side plan and build all tables on the host.
int plan_prepare(int nx, int ny, int nz, double dx, double dy, const double* dz, const int bc[3],
                 const vofp_opts* opt, PlanPrep* pp) {
  if (!dz || !bc) return VOFP_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy))
    return VOFP_ERR_INVALID_ARG;
  if ((long long)nx * ny * nz > (1LL << 31) - 1) return VOFP_ERR_UNSUPPORTED;
  if (nx > 4096 || ny > 4096 || nz > 4096) return VOFP_ERR_UNSUPPORTED;
  for (int a = 0; a < 3; ++a)
    if (bc[a] < VOFP_BC_P || bc[a] > VOFP_BC_DN) return VOFP_ERR_INVALID_ARG;
  for (int k = 0; k < nz; ++k)
    if (!(dz[k] > 0) || !std::isfinite(dz[k])) return VOFP_ERR_INVALID_ARG;
  vofp_opts o;
  vofp_opts_default(&o);
  if (opt) o = *opt;
  if (o.prec != VOFP_FP64 && o.prec != VOFP_MIXED && o.prec != VOFP_FF) return VOFP_ERR_INVALID_ARG;
  if (o.grad_mode != 0 && o.grad_mode != 1) return VOFP_ERR_INVALID_ARG;
  if (o.max_refine < 1) o.max_refine = o.prec == VOFP_FF ? 0 : 1;  // FP32-pair solves may skip confirmation
  if (o.max_refine > VOFP_MAX_REFINE) o.max_refine = VOFP_MAX_REFINE;
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
  const bool mixed = o.prec != VOFP_FP64;  // the refinement path (FP32 or FP32-pair spectrum)
  const bool ffp = o.prec == VOFP_FF;
  const size_t rs = ffp ? sizeof(ff) : sizeof(float);  // bytes per real of the reduced-precision spectrum
  const bool zper = bc[2] == VOFP_BC_P;

  // ---- host tables ----
  const int nn[2] = {nx, ny};
  const double hh[2] = {dx, dy};
  std::vector<double> lam[2];
  std::vector<double2> tw[2], quart[2];
  std::vector<float2> tw32[2], quart32[2];
  std::vector<cff> twff[2], quartff[2];
  std::vector<double2> blu[2];  // Bluestein tables (empty when the axis needs none)
  auto to_cff = [](double2 z) {
    cff c;
    c.x = ff(z.x);
    c.y = ff(z.y);
    return c;
  };
  for (int a = 0; a < 2; ++a) {
    const int n = nn[a];
    const int nq = quarter_bc(bc[a]) ? 2 * n : n;
    lam[a].resize(n);
    tw[a].resize(n);
    quart[a].resize(nq);
    tw32[a].resize(n);
    quart32[a].resize(nq);
    twff[a].resize(n);
    quartff[a].resize(nq);
    for (int q = 0; q < n; ++q) {
      lam[a][q] = eig_1d(bc[a], n, hh[a], q);
      const double t = -2.0 * kPi * q / n;
      tw[a][q] = make_double2(std::cos(t), std::sin(t));
      tw32[a][q] = make_float2((float)tw[a][q].x, (float)tw[a][q].y);
      twff[a][q] = to_cff(tw[a][q]);
    }
    // quarter-wave twiddles: DCT-II / DST-II e^{-i pi q / (2n)}; ND / DN (DCT-IV / DST-IV) the pre-twiddles
    // e^{-i pi q / n} (q < n), then the post-twiddles e^{-i pi (2q+1) / (4n)}
    for (int q = 0; q < nq; ++q) {
      const double u = !quarter_bc(bc[a]) ? -kPi * q / (2.0 * n)
                                          : (q < n ? -kPi * q / n : -kPi * (2 * (q - n) + 1) / (4.0 * n));
      quart[a][q] = make_double2(std::cos(u), std::sin(u));
      quart32[a][q] = make_float2((float)quart[a][q].x, (float)quart[a][q].y);
      quartff[a][q] = to_cff(quart[a][q]);
    }
    factor_radices(n, &p->ax[a].fd);
    p->ax[a].n = n;
    p->ax[a].bc = bc[a];
    if (p->ax[a].fd.bm) blu[a] = bluestein_tables(p->ax[a].fd);
  }
  std::vector<double> za(nz), zb(nz), zc(nz), hz(nz + 1), rdz(nz), rhz(nz + 1), rzc(nz), kz(4 * (size_t)nz);
  const double hper = 0.5 * (dz[nz - 1] + dz[0]);
  for (int k = 0; k <= nz; ++k) {
    if (k == 0)
      hz[k] = zper ? hper : dz[0];
    else if (k == nz)
      hz[k] = zper ? hper : dz[nz - 1];
    else
      hz[k] = 0.5 * (dz[k - 1] + dz[k]);
    rhz[k] = 1.0 / hz[k];
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
    rdz[k] = 1.0 / dz[k];
    rzc[k] = 1.0 / (hz[k] + hz[k + 1]);
    // per-plane constants of the residual stencil and the reductions
    const double czp = rhz[k + 1] * rdz[k], czm = rhz[k] * rdz[k];
    kz[k] = dx * dy * dz[k];  // cell volume
    kz[nz + k] = czp;
    kz[2 * nz + k] = czm;
    kz[3 * nz + k] = -2.0 * (1.0 / (dx * dx) + 1.0 / (dy * dy)) - czp - czm;
  }
  // refinement plans: the low-eigenvalue (x, y) pairs, |lx + ly| <= 64 * (smallest positive |eigenvalue|).
  // Every eigenvalue is <= 0 and |lx_i| is non-decreasing in the packed index i for each boundary
  // condition, so the low pairs of row j are a prefix i < lowcut[j] of it.
  std::vector<int2> low;
  std::vector<int> lowcut(ny, 0);
  p->lowthr = -1.0;
  if (mixed) {
    double l1 = 0;
    for (int a = 0; a < 2; ++a)
      for (int q = 0; q < nn[a]; ++q) {
        const double v = std::fabs(lam[a][q]);
        if (v > 0 && (l1 == 0 || v < l1)) l1 = v;
      }
    p->lowthr = 64.0 * l1;
    for (int j = 0; j < ny; ++j) {
      int cut = 0;
      while (cut < nx && std::fabs(lam[0][cut] + lam[1][j]) <= p->lowthr) ++cut;
      lowcut[j] = cut;
      for (int i = 0; i < cut; ++i) low.push_back(make_int2(i, j));
    }
  }
  p->nlow = (int)low.size();

  // ---- layout ----
  PlanLayout& L = pp->L;
  size_t off = 0;
  for (int a = 0; a < 2; ++a) {
    L.lam[a] = off;
    off = align256(off + sizeof(double) * nn[a]);
    L.tw[a] = off;
    off = align256(off + sizeof(double2) * nn[a]);
    L.q[a] = off;
    off = align256(off + sizeof(double2) * quart[a].size());
    L.tw32[a] = off;
    off = align256(off + sizeof(float2) * nn[a]);
    L.q32[a] = off;
    off = align256(off + sizeof(float2) * quart32[a].size());
    L.twff[a] = off;
    off = align256(off + sizeof(cff) * nn[a]);
    L.qff[a] = off;
    off = align256(off + sizeof(cff) * quartff[a].size());
    L.blu64[a] = L.blu32[a] = L.bluff[a] = 0;
    if (!blu[a].empty()) {
      L.blu64[a] = off;
      off = align256(off + sizeof(double2) * blu[a].size());
      L.blu32[a] = off;
      off = align256(off + sizeof(float2) * blu[a].size());
      L.bluff[a] = off;
      off = align256(off + sizeof(cff) * blu[a].size());
    }
  }
  L.za = off;
  off = align256(off + sizeof(double) * nz);
  L.zb = off;
  off = align256(off + sizeof(double) * nz);
  L.zc = off;
  off = align256(off + sizeof(double) * nz);
  L.dz = off;
  off = align256(off + sizeof(double) * nz);
  L.hz = off;
  off = align256(off + sizeof(double) * (nz + 1));
  L.rdz = off;
  off = align256(off + sizeof(double) * nz);
  L.rhz = off;
  off = align256(off + sizeof(double) * (nz + 1));
  L.rzc = off;
  off = align256(off + sizeof(double) * nz);
  L.kz = off;
  off = align256(off + sizeof(double) * 4 * nz);
  L.volf = off;
  off = align256(off + sizeof(float) * nz);
  L.dzff = off;
  off = align256(off + sizeof(ff) * nz);
  L.za32 = off;
  off = align256(off + sizeof(float) * nz);
  L.zaff = off;
  off = align256(off + sizeof(ff) * nz);
  L.lowcut = off;
  off = align256(off + sizeof(int) * ny);
  L.low = off;
  off = align256(off + sizeof(int2) * low.size());
  L.conv = off;
  off = align256(off + sizeof(double) * VOFP_CONV_SLOTS);
  L.info = off;
  off = align256(off + sizeof(vofp_devinfo));
  L.table_bytes = off;
  // workspace: both paths keep a scratch potential; FP64 plans the FP64 spectrum and the z factor table,
  // mixed plans the FP32 spectrum, the FP64 right-hand side and FP64 columns for the low-eigenvalue systems
  const size_t cells = (size_t)nx * ny * nz;
  const int Ux = zdistinct(nx, bc[0]), Uy = zdistinct(ny, bc[1]);
  L.P = off;
  off = align256(off + sizeof(double) * cells);
  L.S = L.T = L.S32 = L.F = L.lowscr = L.lowtab = 0;
  // bounded z: Thomas factor table per distinct eigenvalue pair in the plan's arithmetic type
  const size_t tsz = o.prec == VOFP_MIXED ? 3 * sizeof(float) : (o.prec == VOFP_FF ? 3 * sizeof(ff) : 3 * sizeof(double));
  if (!mixed) {
    L.S = off;
    off = align256(off + sizeof(double) * cells);
  } else {
    L.S32 = off;  // FP32 or FP32-pair spectrum
    off = align256(off + rs * cells);
    L.F = off;
    off = align256(off + sizeof(double) * cells);
    L.lowscr = off;
    off = align256(off + sizeof(double) * 3 * (size_t)nz * low.size());
    if (!zper && !low.empty()) {
      L.lowtab = off;
      off = align256(off + sizeof(double2) * (size_t)nz * low.size());
    }
  }
  if (!zper) {
    L.T = off;
    off = align256(off + tsz * (size_t)Ux * Uy * nz);
  }
  // FP32 refinement plans: the x transform matrices of the tensor-core x passes
  L.xtc = 0;
  const size_t xb = xtc_table_bytes(nx, (long)ny * nz, o.prec);
  if (xb) {
    L.xtc = off;
    off = align256(off + xb);
  }
  L.total = off;
  p->Ux = Ux;
  p->Uy = Uy;

  std::vector<unsigned char>& host = pp->host;
  host.assign(L.table_bytes, 0);
  for (int a = 0; a < 2; ++a) {
    memcpy(&host[L.lam[a]], lam[a].data(), sizeof(double) * nn[a]);
    memcpy(&host[L.tw[a]], tw[a].data(), sizeof(double2) * nn[a]);
    memcpy(&host[L.q[a]], quart[a].data(), sizeof(double2) * quart[a].size());
    memcpy(&host[L.tw32[a]], tw32[a].data(), sizeof(float2) * nn[a]);
    memcpy(&host[L.q32[a]], quart32[a].data(), sizeof(float2) * quart32[a].size());
    memcpy(&host[L.twff[a]], twff[a].data(), sizeof(cff) * nn[a]);
    memcpy(&host[L.qff[a]], quartff[a].data(), sizeof(cff) * quartff[a].size());
    if (!blu[a].empty()) {
      const size_t m = blu[a].size();
      memcpy(&host[L.blu64[a]], blu[a].data(), sizeof(double2) * m);
      float2* f2 = (float2*)&host[L.blu32[a]];
      cff* fc = (cff*)&host[L.bluff[a]];
      for (size_t q = 0; q < m; ++q) {
        f2[q] = make_float2((float)blu[a][q].x, (float)blu[a][q].y);
        fc[q] = to_cff(blu[a][q]);
      }
    }
  }
  memcpy(&host[L.za], za.data(), sizeof(double) * nz);
  memcpy(&host[L.zb], zb.data(), sizeof(double) * nz);
  memcpy(&host[L.zc], zc.data(), sizeof(double) * nz);
  memcpy(&host[L.dz], dz, sizeof(double) * nz);
  memcpy(&host[L.hz], hz.data(), sizeof(double) * (nz + 1));
  memcpy(&host[L.rdz], rdz.data(), sizeof(double) * nz);
  memcpy(&host[L.rhz], rhz.data(), sizeof(double) * (nz + 1));
  memcpy(&host[L.rzc], rzc.data(), sizeof(double) * nz);
  {
    std::vector<float> z32(nz);
    std::vector<ff> zff(nz);
    for (int k = 0; k < nz; ++k) {
      z32[k] = (float)za[k];
      zff[k] = ff(za[k]);
    }
    memcpy(&host[L.za32], z32.data(), sizeof(float) * nz);
    std::vector<float> vf(nz);
    std::vector<ff> dzf(nz);
    for (int k = 0; k < nz; ++k) {
      vf[k] = (float)kz[k];
      dzf[k] = ff(dz[k]);
    }
    memcpy(&host[L.volf], vf.data(), sizeof(float) * nz);
    memcpy(&host[L.dzff], dzf.data(), sizeof(ff) * nz);
    memcpy(&host[L.kz], kz.data(), sizeof(double) * 4 * nz);
    memcpy(&host[L.zaff], zff.data(), sizeof(ff) * nz);
  }
  memcpy(&host[L.lowcut], lowcut.data(), sizeof(int) * ny);
  if (!low.empty()) memcpy(&host[L.low], low.data(), sizeof(int2) * low.size());

  // launch shapes
  // shared-memory line lengths (the Bluestein length where an axis uses it)
  const int sx = p->ax[0].fd.bm ? p->ax[0].fd.bm : nx, sy = p->ax[1].fd.bm ? p->ax[1].fd.bm : ny;
  p->xpb = sx >= 1024 ? 1 : (1024 / sx > 16 ? 16 : 1024 / sx);
  // reduced-precision x passes of long lines: twice the line pairs per block (the autotuner's choice at 256^3
  // and 512^3 for both FP32 and FP32 pairs: the 512^3 FP32 + refinement projection 23.4 -> 22.2 ms)
  if (mixed && sx >= 256 && sx <= 1024) p->xpb = 2048 / sx;
  if (p->xpb < 1) p->xpb = 1;
  // y pass: columns per block so that each row segment read is 128 bytes (full cache lines), shrunk while the
  // tile (two buffers of tx/2 complex lines) exceeds its shared-memory budget: 96 KB for the FP64 pass (two
  // blocks per SM keep its FP64 pipe busy; measured faster than full lines at 512^3), 132 KB for the
  // reduced-precision passes
  int tx = 16;
  while (tx > 2 && (size_t)16 * tx * y_ld(sy) > 96 * 1024) tx -= 2;
  p->ytx = tx;
  // the reduced-precision path's shapes, sized by its element (FP32 or FP32-pair)
  tx = (int)(128 / rs);
  while (tx > 2 && (size_t)(4 * rs) * tx * y_ld(sy) > 132 * 1024) tx -= 2;
  p->ytx32 = tx;
  if (zper) {
    // periodic z (general column solver): systems per 128-thread block, three columns each in shared memory
    int ti = 32;
    while (ti > 1 && (size_t)3 * ti * nz * sizeof(double) > 96 * 1024) ti /= 2;
    p->zti = ti;
    ti = 32;
    while (ti > 1 && (size_t)3 * ti * nz * rs > 96 * 1024) ti /= 2;
    p->zti32 = ti;
  } else {
    // factor-table kernels: -1 / -2 = the segmented tile kernel with the full / lean tile layout (FP32 and
    // FP32 pairs whenever two tiles fit per SM), 0 = the shared-memory staged kernel (grids with few
    // systems), otherwise the streaming kernel's threads per block (forward values in shared memory when 64
    // or 128 threads' columns fit in 96 KB, else kept in place in the spectrum)
    auto table_ti = [&](size_t elem, bool fp64) {
      if (!fp64 && ztab_seg_code(nz, elem) != 0) return ztab_seg_code(nz, elem);
      if (ztab_use_staged(nx, ny, nz, elem)) return 0;
      if ((size_t)128 * nz * elem <= 96 * 1024) return 128;
      if ((size_t)64 * nz * elem <= 96 * 1024) return 64;
      return 128;
    };
    p->zti = table_ti(sizeof(double), true);
    p->zti32 = table_ti(rs, false);
  }
  pp->p = p;
  return VOFP_OK;
}

// Place a prepared plan in device memory.  `block` NULL: the plan allocates (and later frees) its own
// block and uploads synchronously.  Otherwise `block` (L.total bytes, owned by the caller) receives the
// tables by an asynchronous copy on `st` from `stage` (pinned host memory of L.table_bytes bytes that must
// stay valid until the copy has run).
int plan_bind(PlanPrep* pp, void* block, cudaStream_t st, unsigned char* stage) {
  vofp_plan* p = pp->p;
  const PlanLayout& L = pp->L;
  const bool own = block == nullptr;
  if (own) {
    if (device_alloc(&block, L.total) != cudaSuccess) {
      cudaGetLastError();
      return VOFP_ERR_OOM;
    }
    if (cudaMemcpy(block, pp->host.data(), L.table_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(block);
      return VOFP_ERR_CUDA;
    }
    p->table_block = block;
  } else {
    memcpy(stage, pp->host.data(), L.table_bytes);
    if (cudaMemcpyAsync(block, stage, L.table_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return VOFP_ERR_CUDA;
    p->table_block = nullptr;  // not owned
  }
  unsigned char* b = (unsigned char*)block;
  p->bytes = L.total;
  for (int a = 0; a < 2; ++a) {
    p->ax[a].lam = (const double*)(b + L.lam[a]);
    p->ax[a].tw64 = (const double2*)(b + L.tw[a]);
    p->ax[a].quart64 = (const double2*)(b + L.q[a]);
    p->ax[a].tw32 = (const float2*)(b + L.tw32[a]);
    p->ax[a].quart32 = (const float2*)(b + L.q32[a]);
    p->ax[a].twff = (const cff*)(b + L.twff[a]);
    p->ax[a].quartff = (const cff*)(b + L.qff[a]);
    p->ax[a].blu64 = L.blu64[a] ? (const double2*)(b + L.blu64[a]) : nullptr;
    p->ax[a].blu32 = L.blu32[a] ? (const float2*)(b + L.blu32[a]) : nullptr;
    p->ax[a].bluff = L.bluff[a] ? (const cff*)(b + L.bluff[a]) : nullptr;
  }
  p->za = (double*)(b + L.za);
  p->zb = (double*)(b + L.zb);
  p->zc = (double*)(b + L.zc);
  p->dz = (double*)(b + L.dz);
  p->hz = (double*)(b + L.hz);
  p->rdz = (double*)(b + L.rdz);
  p->rhz = (double*)(b + L.rhz);
  p->rzc = (double*)(b + L.rzc);
  p->kz = (double*)(b + L.kz);
  p->volf = (float*)(b + L.volf);
  p->dzff = (ff*)(b + L.dzff);
  p->conv = (double*)(b + L.conv);
  p->info = (vofp_devinfo*)(b + L.info);
  p->lowmodes = p->nlow ? (int2*)(b + L.low) : nullptr;
  p->P = (double*)(b + L.P);
  const bool mixed = p->opts.prec != VOFP_FP64;
  p->S = mixed ? nullptr : (double*)(b + L.S);
  p->ztab = L.T ? (void*)(b + L.T) : nullptr;
  p->zaT = p->opts.prec == VOFP_MIXED ? (const void*)(b + L.za32)
           : (p->opts.prec == VOFP_FF ? (const void*)(b + L.zaff) : (const void*)p->za);
  p->lowcut = mixed ? (int*)(b + L.lowcut) : nullptr;
  p->S32 = mixed ? (float*)(b + L.S32) : nullptr;
  p->F = mixed ? (double*)(b + L.F) : nullptr;
  p->lowscratch = (mixed && p->nlow) ? (double*)(b + L.lowscr) : nullptr;
  p->lowtab = (mixed && L.lowtab) ? (double2*)(b + L.lowtab) : nullptr;
  p->R = nullptr;
  p->G = nullptr;  // interface geometry: allocated on first use (extension / Stefan source)
  init_kernel_attributes_fp64();
  init_kernel_attributes_mixed();
  if (p->ztab) {
    const int s = build_z_factors(p, st, own);
    if (s) return s;
  }
  if (p->lowtab) {
    const int s = build_low_factors(p, st, own);
    if (s) return s;
  }
  p->xtc_fwd = p->xtc_inv = nullptr;
  p->xtc_grid = 0;
  if (L.xtc) {
    const int s = xtc_build(p, b + L.xtc, st);
    if (s) return s;
    if (own && cudaStreamSynchronize(st) != cudaSuccess) return VOFP_ERR_CUDA;
  }
  return VOFP_OK;
}

size_t plan_prep_device_bytes(const PlanPrep* pp) { return pp->L.total; }
size_t plan_prep_stage_bytes(const PlanPrep* pp) { return pp->L.table_bytes; }

void plan_free_host(vofp_plan* p) {
  if (!p) return;
  free(p->dz_host);
  free(p);
}

int ensure_geometry(vofp_plan* p) {
  if (p->G) return VOFP_OK;
  const size_t cells = (size_t)p->n[0] * p->n[1] * p->n[2];
  void* m = nullptr;
  if (device_alloc(&m, 4 * sizeof(double) * cells) != cudaSuccess) {
    cudaGetLastError();
    return VOFP_ERR_OOM;
  }
  p->G = (double*)m;
  p->bytes += 4 * sizeof(double) * cells;
  return VOFP_OK;
}

}  // namespace vofp

using namespace vofp;

extern "C" unsigned long long vofp_launch_count(void) { return g_launches.load(); }

extern "C" void vofp_opts_default(vofp_opts* opt) {
  if (!opt) return;
  opt->prec = VOFP_FP64;
  opt->tol = 1e-10;
  opt->max_refine = 3;
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

extern "C" int vofp_plan_create(int nx, int ny, int nz, double dx, double dy, const double* dz, const int bc[3],
                                const vofp_opts* opt, vofp_plan** out) {
  if (!out) return VOFP_ERR_INVALID_ARG;
  *out = nullptr;
  PlanPrep pp;
  int s = plan_prepare(nx, ny, nz, dx, dy, dz, bc, opt, &pp);
  if (s) return s;
  s = plan_bind(&pp, nullptr, nullptr, nullptr);
  if (s) {
    vofp_plan_destroy(pp.p);
    return s;
  }
  if (pp.p->opts.tune) vofp_plan_tune(pp.p);
  *out = pp.p;
  return VOFP_OK;
}

extern "C" void vofp_plan_destroy(vofp_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  if (p->table_block) cudaFree(p->table_block);
  if (p->G) cudaFree(p->G);
  free_host_step(p);
  cudaSetDevice(cur);
  plan_free_host(p);
}

extern "C" size_t vofp_plan_workspace_bytes(const vofp_plan* p) { return p ? p->bytes : 0; }
