// Allocation-free FP64 Poisson solve.
//
// Some host codes cannot call cudaMalloc when they need a solve: a solver whose device memory is handed
// out entirely by its own pool allocator at start-up, or a time-stepping loop that must not pay the
// implicit device-wide synchronisation and latency of cudaMalloc / cudaFree.  vofp_poisson_solve_noalloc
// serves them: it needs no plan and allocates nothing.  Its spectrum workspace and its tables live in one
// file-scope __device__ array of fixed size (VOFP_NOALLOC_MAX_CELLS cells plus tables for axes of up to
// VOFP_NOALLOC_MAX_N cells); every GPU that loads the library holds that array until the process exits.
//
// On the host the array's name is only a stand-in, not a device address, so the first call on each device
// fetches the real address with cudaGetSymbolAddress (with that device current) and keeps it.  That first
// call should therefore come before any stream capture.  Every call rebuilds the tables in the array and
// overwrites the whole spectrum region it uses, so no state from an earlier call leaks into a later one,
// but all calls share the one array: calls whose work overlaps on the GPU (different streams, threads or
// processes sharing a context) race and corrupt each other.
#include <cmath>
#include <mutex>

#include "solve_internal.h"
#include "passes.cuh"

namespace {

constexpr size_t kMaxCells = VOFP_NOALLOC_MAX_CELLS;
constexpr int kMaxN = VOFP_NOALLOC_MAX_N;
constexpr size_t kSpecBytes = kMaxCells * sizeof(double);
// table region, fixed offsets (bytes from its start)
constexpr size_t kOffLamX = 0;
constexpr size_t kOffLamY = kOffLamX + kMaxN * sizeof(double);
constexpr size_t kOffTwX = kOffLamY + kMaxN * sizeof(double);
constexpr size_t kOffTwY = kOffTwX + kMaxN * sizeof(double2);
constexpr size_t kOffQX = kOffTwY + kMaxN * sizeof(double2);
constexpr size_t kOffQY = kOffQX + kMaxN * sizeof(double2);
constexpr size_t kOffZa = kOffQY + kMaxN * sizeof(double2);
constexpr size_t kOffZb = kOffZa + kMaxN * sizeof(double);
constexpr size_t kOffZc = kOffZb + kMaxN * sizeof(double);
constexpr size_t kOffDz = kOffZc + kMaxN * sizeof(double);
constexpr size_t kOffHz = kOffDz + kMaxN * sizeof(double);
constexpr size_t kOffRdz = kOffHz + (kMaxN + 1) * sizeof(double);
constexpr size_t kOffRhz = kOffRdz + kMaxN * sizeof(double);
constexpr size_t kOffRzc = kOffRhz + (kMaxN + 1) * sizeof(double);
constexpr size_t kTableBytes = kOffRzc + kMaxN * sizeof(double) + 256;
constexpr size_t kScratchBytes = kSpecBytes + ((kTableBytes + 255) / 256) * 256;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace vofp {

// The z widths travel by value in the launch's parameters (8 KiB at most), so the call reads the caller's
// host array once, when it returns nothing refers to it any more, and no host-to-device copy is needed.
struct NoallocDz {
  double w[kMaxN];
};

// Eigenvalue of packed spectral index q (same conventions as the plan's tables), twiddles and z rows; the
// widths are stored into the table region for the solve's later kernels.
__global__ void k_noalloc_tables(int nx, int ny, int nz, double dx, double dy, int bcx, int bcy, int bcz,
                                 unsigned char* tab, const __grid_constant__ NoallocDz dzp) {
  double* lam[2] = {(double*)(tab + kOffLamX), (double*)(tab + kOffLamY)};
  double2* tw[2] = {(double2*)(tab + kOffTwX), (double2*)(tab + kOffTwY)};
  double2* qt[2] = {(double2*)(tab + kOffQX), (double2*)(tab + kOffQY)};
  const int nn[2] = {nx, ny};
  const double hh[2] = {dx, dy};
  const int bb[2] = {bcx, bcy};
  const double* dz = dzp.w;
  double* za = (double*)(tab + kOffZa);
  double* zb = (double*)(tab + kOffZb);
  double* zc = (double*)(tab + kOffZc);
  double* hz = (double*)(tab + kOffHz);
  double* rdz = (double*)(tab + kOffRdz);
  double* rhz = (double*)(tab + kOffRhz);
  double* rzc = (double*)(tab + kOffRzc);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int a = 0; a < 2; ++a) {
    const int n = nn[a];
    if (t < n) {
      double arg;  // argument / pi
      if (bb[a] == VOFP_BC_P)
        arg = (double)((t + 1) / 2) / n;
      else if (bb[a] == VOFP_BC_NN)
        arg = t / (2.0 * n);
      else
        arg = (t + 1) / (2.0 * n);
      const double s = sinpi(arg);
      lam[a][t] = -4.0 / (hh[a] * hh[a]) * s * s;
      double sn, cs;
      sincospi(-2.0 * t / n, &sn, &cs);
      tw[a][t] = make_double2(cs, sn);
      sincospi(-(double)t / (2.0 * n), &sn, &cs);
      qt[a][t] = make_double2(cs, sn);
    }
  }
  const bool zper = bcz == VOFP_BC_P;
  if (t <= nz) {
    double h;
    if (t == 0)
      h = zper ? 0.5 * (dz[nz - 1] + dz[0]) : dz[0];
    else if (t == nz)
      h = zper ? 0.5 * (dz[nz - 1] + dz[0]) : dz[nz - 1];
    else
      h = 0.5 * (dz[t - 1] + dz[t]);
    hz[t] = h;
    rhz[t] = 1.0 / h;
  }
  if (t < nz) {
    const double hlo = t == 0 ? (zper ? 0.5 * (dz[nz - 1] + dz[0]) : dz[0]) : 0.5 * (dz[t - 1] + dz[t]);
    const double hhi =
        t == nz - 1 ? (zper ? 0.5 * (dz[nz - 1] + dz[0]) : dz[nz - 1]) : 0.5 * (dz[t] + dz[t + 1]);
    const double a = 1.0 / (dz[t] * hlo);
    const double c = 1.0 / (dz[t] * hhi);
    double b = -(a + c), aa = a, cc = c;
    if (!zper && t == 0) {
      b += (bcz == VOFP_BC_NN || bcz == VOFP_BC_ND) ? a : -a;
      aa = 0;
    }
    if (!zper && t == nz - 1) {
      b += (bcz == VOFP_BC_NN || bcz == VOFP_BC_DN) ? c : -c;
      cc = 0;
    }
    za[t] = aa;
    zb[t] = b;
    zc[t] = cc;
    ((double*)(tab + kOffDz))[t] = dz[t];
    rdz[t] = 1.0 / dz[t];
    rzc[t] = 1.0 / (hlo + hhi);
  }
}

}  // namespace vofp

using namespace vofp;

static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_addr[64];

// Device address of the scratch array for the current device (fetched once per device).
static int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VOFP_ERR_CUDA;
  if (dev < 0 || dev >= 64) return VOFP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return VOFP_ERR_CUDA;
    }
    init_kernel_attributes_fp64();
    g_noalloc_addr[dev] = (unsigned char*)ptr;
  }
  *out = g_noalloc_addr[dev];
  return VOFP_OK;
}

extern "C" int vofp_poisson_solve_noalloc(int nx, int ny, int nz, double dx, double dy, const double* dz,
                                          const int bc[3], const double* f, double* p, void* stream) {
  if (!dz || !bc || !f || !p) return VOFP_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy))
    return VOFP_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (bc[a] < VOFP_BC_P || bc[a] > VOFP_BC_DN) return VOFP_ERR_INVALID_ARG;
  if (bc[0] > VOFP_BC_DD || bc[1] > VOFP_BC_DD) return VOFP_ERR_UNSUPPORTED;
  double lz = 0;
  for (int k = 0; k < nz; ++k) {
    if (!(dz[k] > 0) || !std::isfinite(dz[k])) return VOFP_ERR_INVALID_ARG;
    lz += dz[k];
  }
  if (nx > kMaxN || ny > kMaxN || nz > kMaxN || (size_t)nx * ny * nz > kMaxCells) return VOFP_ERR_TOO_LARGE;
  unsigned char* base = nullptr;
  int s = noalloc_scratch(&base);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* tab = base + kSpecBytes;
  NoallocDz dzp;
  for (int k = 0; k < nz; ++k) dzp.w[k] = dz[k];
  const int tmax = (nx > ny ? nx : ny) > nz + 1 ? (nx > ny ? nx : ny) : nz + 1;
  VOFP_LAUNCH(KID_NOALLOC_TABLES, st,
              k_noalloc_tables<<<(tmax + 127) / 128, 128, 0, st>>>(nx, ny, nz, dx, dy, bc[0], bc[1], bc[2], tab,
                                                                   dzp));

  // a plan that lives on this stack frame and points into the scratch array
  vofp_plan pl = {};
  pl.n[0] = nx;
  pl.n[1] = ny;
  pl.n[2] = nz;
  for (int a = 0; a < 3; ++a) pl.bc[a] = bc[a];
  pl.dx = dx;
  pl.dy = dy;
  vofp_opts_default(&pl.opts);
  auto is_nd = [](int b) { return b == VOFP_BC_P || b == VOFP_BC_NN; };
  pl.singular = is_nd(bc[0]) && is_nd(bc[1]) && is_nd(bc[2]);
  pl.volume = nx * dx * ny * dy * lz;
  const int nn[2] = {nx, ny};
  const size_t olam[2] = {kOffLamX, kOffLamY}, otw[2] = {kOffTwX, kOffTwY}, oq[2] = {kOffQX, kOffQY};
  for (int a = 0; a < 2; ++a) {
    pl.ax[a].n = nn[a];
    pl.ax[a].bc = bc[a];
    factor_radices(nn[a], &pl.ax[a].fd);
    pl.ax[a].lam = (const double*)(tab + olam[a]);
    pl.ax[a].tw64 = (const double2*)(tab + otw[a]);
    pl.ax[a].quart64 = (const double2*)(tab + oq[a]);
  }
  pl.za = (double*)(tab + kOffZa);
  pl.zb = (double*)(tab + kOffZb);
  pl.zc = (double*)(tab + kOffZc);
  pl.dz = (double*)(tab + kOffDz);
  pl.hz = (double*)(tab + kOffHz);
  pl.rdz = (double*)(tab + kOffRdz);
  pl.rhz = (double*)(tab + kOffRhz);
  pl.rzc = (double*)(tab + kOffRzc);
  pl.ztab = nullptr;
  pl.S = (double*)base;
  pl.info = nullptr;
  pl.xpb = nx >= 1024 ? 1 : (1024 / nx > 16 ? 16 : 1024 / nx);
  int tx = 16;
  while (tx > 2 && (size_t)16 * tx * y_ld(ny) > 96 * 1024) tx -= 2;
  pl.ytx = tx;
  const int nvec = bc[2] == VOFP_BC_P ? 3 : 2;
  int ti = 32;
  while (ti > 1 && (size_t)nvec * ti * nz * sizeof(double) > 96 * 1024) ti /= 2;
  pl.zti = ti;
  XArgs xa = {};
  xa.f = f;
  xa.scale = 1.0;
  return fp64_solve(&pl, RHS_F, xa, p, st, false);
}
