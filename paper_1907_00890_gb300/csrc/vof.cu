// Volume-of-fluid update with the interface velocity (§3.1): the directional split of Eq. fluxes, each
// one-dimensional step implicit in its own result, then the correction of Eq. final_corr_1 with the implicit
// volume deflation of Eq. final_corr_2:
//
//   C*   (1 - dt du/dx) = C^n  - (f_{i+1/2} - f_{i-1/2}) / dx        f = dt uG C_upwind(C^n)
//   C**  (1 - dt dv/dy) = C*   - (g_{j+1/2} - g_{j-1/2}) / dy        g = dt vG C_upwind(C*)
//   C*** (1 - dt dw/dz) = C**  - (h_{k+1/2} - h_{k-1/2}) / dz_k      h = dt wG C_upwind(C**)
//   C^{n+1} (1 - dt div uG) = C*** - dt (C* du/dx + C** dv/dy + C*** dw/dz)
//
// with du/dx = (uG_{i+1/2} - uG_{i-1/2}) / dx and so on.  The paper takes f, g, h from an MTHINC reconstruction
// it does not restate; these are first-order upwind fluxes (the cell the face velocity comes from; beyond a
// bounded end the boundary cell itself).  One FP64 pass per direction, one thread per cell; C* and C** live in
// a caller-provided workspace.  The passes are bound by FP64 arithmetic, not by their ~32 bytes per cell, so the
// implicit steps divide through an FP32-seeded Newton reciprocal and pick upwind cells by an integer sign test.
#include <cmath>
#include <cstdint>

#include "solve_internal.h"
#include "stencil.cuh"

namespace vofp {

// Upwind value C_upwind across face f (the low face of cell f) of a line of n cells at `base` with stride
// `st`, for the face velocity `vel`: the cell the flow comes from (sign bit of vel, an integer test; a zero
// velocity of either sign gives a zero flux whichever cell is taken), beyond a bounded end the boundary cell.
__device__ __forceinline__ double upwind_value(const double* __restrict__ q, size_t base, size_t st, int n, int bc,
                                               int f, double vel) {
  int lo = f - 1, hi = f;  // the cells across the face
  if (bc == VOFP_BC_P) {
    if (lo < 0) lo += n;
    if (hi >= n) hi -= n;
  } else {
    if (lo < 0) lo = 0;
    if (hi >= n) hi = n - 1;
  }
  return __ldg(q + base + (size_t)(__double2hiint(vel) >= 0 ? lo : hi) * st);
}

// One implicit directional step along `axis` for cell (i, j, k): returns the new value of q there and sets
// `du` to the face-velocity difference over the cell width.  With dt factored out of the fluxes,
//   q_new = (q - dt/w (v_hi q_up(hi) - v_lo q_up(lo))) / (1 - dt/w (v_hi - v_lo)),
// the quotient taken as a product with the Newton reciprocal of the denominator.
__device__ __forceinline__ double vof_step(const GridDev& g, const double* __restrict__ q,
                                           const double* __restrict__ vel, int axis, int i, int j, int k, double dt,
                                           double& du) {
  const size_t plane = (size_t)g.nx * g.ny;
  int n, bc, f;
  size_t base, st, fbase, fst;
  double rw;
  if (axis == 0) {
    n = g.nx, bc = g.bcx, f = i, base = (size_t)k * plane + (size_t)j * g.nx, st = 1;
    fbase = ((size_t)k * g.ny + j) * nface(g.nx, g.bcx), fst = 1, rw = g.rdx;
  } else if (axis == 1) {
    n = g.ny, bc = g.bcy, f = j, base = (size_t)k * plane + i, st = g.nx;
    fbase = (size_t)k * nface(g.ny, g.bcy) * g.nx + i, fst = g.nx, rw = g.rdy;
  } else {
    n = g.nz, bc = g.bcz, f = k, base = (size_t)j * g.nx + i, st = plane;
    fbase = (size_t)j * g.nx + i, fst = plane, rw = __ldg(g.rdz + k);
  }
  const int fp = (bc == VOFP_BC_P && f + 1 == n) ? 0 : f + 1;  // the high face of the cell
  const double vlo = __ldg(vel + fbase + (size_t)f * fst), vhi = __ldg(vel + fbase + (size_t)fp * fst);
  const double qlo = upwind_value(q, base, st, n, bc, f, vlo);
  const double qhi = upwind_value(q, base, st, n, bc, f + 1, vhi);
  const double dtrw = dt * rw, dv = vhi - vlo;
  du = dv * rw;
  const double num = fma(-dtrw, fma(vhi, qhi, -vlo * qlo), __ldg(q + base + (size_t)f * st));
  return num * recip_newton(fma(-dtrw, dv, 1.0));
}

// x or y step: out = the implicit step of q along `axis`.
static __global__ void __launch_bounds__(128) k_vof_step(GridDev g, const double* __restrict__ q,
                                                        const double* __restrict__ vel, int axis, double dt,
                                                        double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= g.nx) return;
  double du;
  out[((size_t)k * g.ny + j) * g.nx + i] = vof_step(g, q, vel, axis, i, j, k, dt, du);
}

// z step, then the correction and the implicit deflation of Eq. final_corr_2.
static __global__ void __launch_bounds__(128) k_vof_final(GridDev g, const double* __restrict__ c1,
                                                         const double* __restrict__ c2,
                                                         const double* __restrict__ uG,
                                                         const double* __restrict__ vG,
                                                         const double* __restrict__ wG, double dt,
                                                         double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= g.nx) return;
  const size_t c = ((size_t)k * g.ny + j) * g.nx + i;
  double dw, du, dv;
  const double c3 = vof_step(g, c2, wG, 2, i, j, k, dt, dw);
  // face differences of uG and vG at this cell (the x and y steps' du, dv)
  {
    const int nxf = nface(g.nx, g.bcx), nyf = nface(g.ny, g.bcy);
    const int ip = (g.bcx == VOFP_BC_P && i + 1 == g.nx) ? 0 : i + 1;
    const size_t ub = ((size_t)k * g.ny + j) * nxf;
    du = (__ldg(uG + ub + ip) - __ldg(uG + ub + i)) * g.rdx;
    const int jp = (g.bcy == VOFP_BC_P && j + 1 == g.ny) ? 0 : j + 1;
    const size_t vb = (size_t)k * nyf * g.nx + i;
    dv = (__ldg(vG + vb + (size_t)jp * g.nx) - __ldg(vG + vb + (size_t)j * g.nx)) * g.rdy;
  }
  const double F = fma(__ldg(c1 + c), du, fma(__ldg(c2 + c), dv, c3 * dw));
  out[c] = fma(-dt, F, c3) * recip_newton(fma(-dt, du + dv + dw, 1.0));
}

}  // namespace vofp

using namespace vofp;

extern "C" int vofp_vof_update(vofp_plan* pl, const double* C, const double* uG, const double* vG, const double* wG,
                               double dt, double* C_out, double* work, void* stream) {
  if (!pl || !C || !uG || !vG || !wG || !C_out || !work || !(dt > 0) || !std::isfinite(dt))
    return VOFP_ERR_INVALID_ARG;
  const GridDev g = grid_dev(pl);
  const size_t cells = (size_t)g.nx * g.ny * g.nz;
  // the workspace [work, work + 2 cells) must not overlap C or C_out (the passes read and write through
  // restrict pointers)
  auto overlaps = [](const double* a, size_t na, const double* b, size_t nb) {
    const uintptr_t a0 = (uintptr_t)a, a1 = a0 + na * sizeof(double);
    const uintptr_t b0 = (uintptr_t)b, b1 = b0 + nb * sizeof(double);
    return a0 < b1 && b0 < a1;
  };
  if (overlaps(work, 2 * cells, C, cells) || overlaps(work, 2 * cells, C_out, cells)) return VOFP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double* c1 = work;          // C*
  double* c2 = work + cells;  // C**
  const dim3 grid((unsigned)((g.nx + 127) / 128), (unsigned)g.ny, (unsigned)g.nz);
  VOFP_LAUNCH(KID_VOF, st, k_vof_step<<<grid, 128, 0, st>>>(g, C, uG, 0, dt, c1));
  VOFP_LAUNCH(KID_VOF, st, k_vof_step<<<grid, 128, 0, st>>>(g, c1, vG, 1, dt, c2));
  VOFP_LAUNCH(KID_VOF, st, k_vof_final<<<grid, 128, 0, st>>>(g, c1, c2, uG, vG, wG, dt, C_out));
  return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}
