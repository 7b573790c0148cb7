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
// bounded end the boundary cell itself).  All steps run in one FP64 pass that marches through the planes (see
// k_vof_fused); the implicit steps divide through an FP32-seeded reciprocal with one Newton step (relative
// error about 1e-14; the pass is bound by its FP64 arithmetic) and pick upwind cells by an integer sign test.
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
  if (!VOFP_IN(base + (size_t)(n - 1) * st, ncells(g), CHK_VOF_LOAD) ||
      !VOFP_IN(fbase + (size_t)(nface(n, bc) - 1) * fst, nfaces(g, axis), CHK_VOF_LOAD) ||
      !VOFP_IN(f, n, CHK_VOF_LOAD)) {
    du = 0.0;
    return 0.0;
  }
  const double vlo = __ldg(vel + fbase + (size_t)f * fst), vhi = __ldg(vel + fbase + (size_t)fp * fst);
  const double qlo = upwind_value(q, base, st, n, bc, f, vlo);
  const double qhi = upwind_value(q, base, st, n, bc, f + 1, vhi);
  const double dtrw = dt * rw, dv = vhi - vlo;
  du = dv * rw;
  const double num = fma(-dtrw, fma(vhi, qhi, -vlo * qlo), __ldg(q + base + (size_t)f * st));
  return num * recip_newton1(fma(-dtrw, dv, 1.0));
}

// ---- the fused update: one pass marching through the planes -------------------------------------------------
// A CTA owns a column of kVofTX x kVofTY cells and a run of kVofKC planes [k0, k1).  Marching from plane k0 - 1
// to k1 (wrapped on a periodic z axis, clamped on a bounded one -- the upwind rule takes the boundary plane
// itself beyond an end), it forms for each plane m C* (the x step, from C^n in global memory) on its rows plus
// one halo row on each side (recomputed: the y step needs its y neighbours), then C** (the y step, from C* in
// shared memory) into a ring of three planes, and once C** of m is there, the z step and the correction of Eq.
// final_corr_2 for plane m - 1, which needs C** of m - 2, m - 1 and m.  C^n, uG, vG, wG are read and C^{n+1}
// written once per cell (40 bytes) and C*, C** never leave shared memory; the price is the recomputed halo rows
// and planes (x step x (1 + 2/kVofTY)(1 + 2/kVofKC), y step x (1 + 2/kVofKC)).
constexpr int kVofTX = 32, kVofTY = 16, kVofKC = 16;

__device__ __forceinline__ int wrap_clamp(int j, int n, int bc) {
  if (j < 0) return bc == VOFP_BC_P ? j + n : 0;
  if (j >= n) return bc == VOFP_BC_P ? j - n : n - 1;
  return j;
}

// The implicit one-dimensional step of a cell from its value q, its neighbours' values across the low and
// high faces (qm, qp) and the two face velocities (as vof_step); sets dv_rw to the velocity difference over
// the width.
__device__ __forceinline__ double vof_step_local(double qm, double q, double qp, double vlo, double vhi, double rw,
                                                 double dt, double& dv_rw) {
  const double qlo = __double2hiint(vlo) >= 0 ? qm : q;  // upwind across the low face
  const double qhi = __double2hiint(vhi) >= 0 ? q : qp;  // upwind across the high face
  const double dtrw = dt * rw, dv = vhi - vlo;
  dv_rw = dv * rw;
  const double num = fma(-dtrw, fma(vhi, qhi, -vlo * qlo), q);
  return num * recip_newton1(fma(-dtrw, dv, 1.0));
}

static __global__ void __launch_bounds__(kVofTX * kVofTY) k_vof_fused(GridDev g, const double* __restrict__ C,
                                                                     const double* __restrict__ uG,
                                                                     const double* __restrict__ vG,
                                                                     const double* __restrict__ wG, double dt,
                                                                     double* __restrict__ out) {
  __shared__ double cs[2][kVofTY + 2][kVofTX];  // C* of the last two planes, with the halo rows
  __shared__ double css[3][kVofTY][kVofTX];     // C** of the last three planes
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * kVofTX, j0 = blockIdx.y * kVofTY;
  const int k0 = blockIdx.z * kVofKC;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int k1 = k0 + kVofKC < nz ? k0 + kVofKC : nz;
  const int i = i0 + tx, j = j0 + ty;
  const bool act = i < nx && j < ny;
  const size_t plane = (size_t)nx * ny;
  const int nyf = nface(ny, g.bcy);
  // local row r of cs <-> grid row j0 - 1 + r (wrapped or clamped at the ends); rows past ny are unused
  auto row_used = [&](int r) { return j0 - 1 + r <= ny && i < nx; };
  auto x_step = [&](int k, double* dst) {  // C* of plane k: each thread its row, rows 0 / 1 the halo rows
    double du;
    if (row_used(ty + 1)) dst[(ty + 1) * kVofTX + tx] = vof_step(g, C, uG, 0, i, wrap_clamp(j, ny, g.bcy), k, dt, du);
    if (ty < 2) {
      const int r = ty == 0 ? 0 : kVofTY + 1;
      if (row_used(r)) dst[r * kVofTX + tx] = vof_step(g, C, uG, 0, i, wrap_clamp(j0 - 1 + r, ny, g.bcy), k, dt, du);
    }
  };
  auto y_step = [&](int k, const double* src, double* dst) {  // C** of plane k from C* in shared memory
    if (!act) return;
    const int jp = (g.bcy == VOFP_BC_P && j + 1 == ny) ? 0 : j + 1;
    const size_t vb = (size_t)k * nyf * nx + i;
    const double vlo = ldg_in(vG, vb + (size_t)j * nx, nfaces(g, 1), CHK_VOF_LOAD);
    const double vhi = ldg_in(vG, vb + (size_t)jp * nx, nfaces(g, 1), CHK_VOF_LOAD);
    double dv;
    dst[ty * kVofTX + tx] = vof_step_local(src[ty * kVofTX + tx], src[(ty + 1) * kVofTX + tx],
                                           src[(ty + 2) * kVofTX + tx], vlo, vhi, g.rdy, dt, dv);
  };
  // z step and correction of plane k from C** of planes k - 1, k, k + 1 and C* of plane k
  auto finish = [&](int k, const double* qm, const double* q, const double* qp, const double* c1) {
    if (!act) return;
    const int o = ty * kVofTX + tx;
    const size_t fb = (size_t)j * nx + i;
    const int kp = (g.bcz == VOFP_BC_P && k + 1 == nz) ? 0 : k + 1;
    const double wlo = ldg_in(wG, fb + (size_t)k * plane, nfaces(g, 2), CHK_VOF_LOAD);
    const double whi = ldg_in(wG, fb + (size_t)kp * plane, nfaces(g, 2), CHK_VOF_LOAD);
    double dw;
    const double c3 = vof_step_local(qm[o], q[o], qp[o], wlo, whi, __ldg(g.rdz + k), dt, dw);
    const int nxf = nface(nx, g.bcx);
    const int ip = (g.bcx == VOFP_BC_P && i + 1 == nx) ? 0 : i + 1;
    const size_t ub = ((size_t)k * ny + j) * nxf;
    const double du =
        (ldg_in(uG, ub + ip, nfaces(g, 0), CHK_VOF_LOAD) - ldg_in(uG, ub + i, nfaces(g, 0), CHK_VOF_LOAD)) * g.rdx;
    const int jp = (g.bcy == VOFP_BC_P && j + 1 == ny) ? 0 : j + 1;
    const size_t vb = (size_t)k * nyf * nx + i;
    const double dv = (ldg_in(vG, vb + (size_t)jp * nx, nfaces(g, 1), CHK_VOF_LOAD) -
                       ldg_in(vG, vb + (size_t)j * nx, nfaces(g, 1), CHK_VOF_LOAD)) * g.rdy;
    const double F = fma(c1[(ty + 1) * kVofTX + tx], du, fma(q[o], dv, c3 * dw));
    if (VOFP_IN((size_t)k * plane + fb, plane * nz, CHK_CELL_STORE))
      out[(size_t)k * plane + fb] = fma(-dt, F, c3) * recip_newton1(fma(-dt, du + dv + dw, 1.0));
  };
  for (int m = k0 - 1; m <= k1; ++m) {
    const int s = m - (k0 - 1);  // march step: ring slots s & 1 (C*) and s % 3 (C**)
    const int pm = wrap_clamp(m, nz, g.bcz);
    x_step(pm, &cs[s & 1][0][0]);
    __syncthreads();
    y_step(pm, &cs[s & 1][0][0], &css[s % 3][0][0]);
    __syncthreads();
    if (m >= k0 + 1)
      finish(m - 1, &css[(s + 1) % 3][0][0], &css[(s + 2) % 3][0][0], &css[s % 3][0][0], &cs[(s + 1) & 1][0][0]);
    __syncthreads();
  }
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
  // the CTAs read C in their neighbours' columns while others already write theirs: an output over C goes to
  // the workspace first and is copied back
  const bool in_place = overlaps(C_out, cells, C, cells);
  double* dst = in_place ? work : C_out;
  const dim3 grid((unsigned)((g.nx + kVofTX - 1) / kVofTX), (unsigned)((g.ny + kVofTY - 1) / kVofTY),
                  (unsigned)((g.nz + kVofKC - 1) / kVofKC));
  VOFP_LAUNCH(KID_VOF, st, (k_vof_fused<<<grid, dim3(kVofTX, kVofTY), 0, st>>>(g, C, uG, vG, wG, dt, dst)));
  if (in_place && cudaMemcpyAsync(C_out, work, cells * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return VOFP_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}
