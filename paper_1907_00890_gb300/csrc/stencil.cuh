// MAC-grid stencils shared by the transform passes and the epilogues (device code).
//
// Face arrays: index i along the face's axis is the low face of cell i; a periodic axis stores n faces,
// a bounded axis n + 1.  Divergence (Eq. mass, discretised): sum over axes of (F_{i+1} - F_i) / w_i.
// Gradient on faces (correction after Eq. lap_p): (p_i - p_{i-1}) / h with h the centre distance; an N
// boundary face is left untouched, a D boundary face uses the ghost value -p (2 p_0 / w_0 low end,
// -2 p_{n-1} / w_{n-1} high end).  |grad C| and n (§3.2 regularised delta, §3.6 Eq. int_vel): central or
// Youngs corner-averaged differences with C copied into ghost cells at bounded ends and wrapped at periodic
// ends; n = -grad C / |grad C|, zero where min(C, 1 - C) < 1e-8 or |grad C| = 0.
// FP64 divisions are replaced by multiplications with reciprocal tables built once per plan (the FP64 pipe
// of the GB300 is narrow; a division costs about ten multiply-adds).
#pragma once

#include "vofp_internal.cuh"

namespace vofp {

struct GridDev {
  int nx, ny, nz;
  int bcx, bcy, bcz;
  double dx, dy;
  double rdx, rdy;    // 1/dx, 1/dy
  double rdx2, rdy2;  // 1/dx^2, 1/dy^2
  double hrdx, hrdy;  // 1/(2 dx), 1/(2 dy): central differences
  const double* dz;   // nz widths
  const double* hz;   // nz + 1 centre distances across z faces (ghost distances at the ends)
  const double* rdz;  // 1/dz
  const double* rhz;  // 1/hz
  const double* rzc;  // 1/(hz[k] + hz[k+1]): central difference in z
  const double* vol;  // cell volume per plane (dx dy dz_k)
  const double* czp;  // residual stencil: coefficient of p_{k+1}, rhz[k+1] / dz_k
  const double* czm;  //   of p_{k-1}, rhz[k] / dz_k
  const double* czc;  //   of p_k, -2 (1/dx^2 + 1/dy^2) - czp - czm
  const float* volf;  // cell volume per plane, FP32
  const ff* dzff;     // dz per plane, FP32 pair
};

__host__ __device__ __forceinline__ int nface(int n, int bc) { return n + (bc != VOFP_BC_P); }
__host__ __device__ __forceinline__ size_t ncells(const GridDev& g) { return (size_t)g.nx * g.ny * g.nz; }
// the u, v, w face arrays: nface cells along their own axis
__host__ __device__ __forceinline__ size_t nfaces(const GridDev& g, int axis) {
  return (size_t)(axis == 0 ? nface(g.nx, g.bcx) : g.nx) * (axis == 1 ? nface(g.ny, g.bcy) : g.ny) *
         (axis == 2 ? nface(g.nz, g.bcz) : g.nz);
}

// Neighbour index for a cell field: wrapped on a periodic axis, clamped (ghost copy) on a bounded one.
__device__ __forceinline__ int cw(int i, int n, int bc) {
  if (i < 0) return bc == VOFP_BC_P ? i + n : 0;
  if (i >= n) return bc == VOFP_BC_P ? i - n : n - 1;
  return i;
}

// Divergence of the face field (u, v, w) at cell (i, j, k) plus `addend`, the addend taken into the last
// multiply-add (three subtractions and three multiply-adds in FP64).
__device__ __forceinline__ double divergence_at(const GridDev& g, const double* __restrict__ u,
                                                const double* __restrict__ v, const double* __restrict__ w, int i,
                                                int j, int k, double addend = 0.0) {
  const int nxf = nface(g.nx, g.bcx), nyf = nface(g.ny, g.bcy);
  const size_t ub = ((size_t)k * g.ny + j) * nxf;
  const int ip = (g.bcx == VOFP_BC_P && i + 1 == g.nx) ? 0 : i + 1;
  const size_t nu = nfaces(g, 0), nv = nfaces(g, 1), nw = nfaces(g, 2);
  const double du = ldg_in(u, ub + ip, nu, CHK_FACE_LOAD) - ldg_in(u, ub + i, nu, CHK_FACE_LOAD);
  const size_t vb = (size_t)k * nyf * g.nx + i;
  const int jp = (g.bcy == VOFP_BC_P && j + 1 == g.ny) ? 0 : j + 1;
  const double dv = ldg_in(v, vb + (size_t)jp * g.nx, nv, CHK_FACE_LOAD) -
                    ldg_in(v, vb + (size_t)j * g.nx, nv, CHK_FACE_LOAD);
  const size_t plane = (size_t)g.ny * g.nx;
  const int kp = (g.bcz == VOFP_BC_P && k + 1 == g.nz) ? 0 : k + 1;
  const size_t wb = (size_t)j * g.nx + i;
  const double dw = ldg_in(w, wb + kp * plane, nw, CHK_FACE_LOAD) - ldg_in(w, wb + k * plane, nw, CHK_FACE_LOAD);
  return fma(du, g.rdx, fma(dv, g.rdy, fma(dw, __ldg(g.rdz + k), addend)));
}

__device__ __forceinline__ double cval(const GridDev& g, const double* __restrict__ C, int i, int j, int k) {
  i = cw(i, g.nx, g.bcx);
  j = cw(j, g.ny, g.bcy);
  k = cw(k, g.nz, g.bcz);
  return ldg_in(C, ((size_t)k * g.ny + j) * g.nx + i, ncells(g), CHK_CELL_LOAD);
}

// Cell-centred gradient of C: mode 0 central, mode 1 Youngs.
__device__ __forceinline__ double3 grad_c_at(const GridDev& g, const double* __restrict__ C, int i, int j, int k,
                                             int mode) {
  double3 r;
  if (mode == 0) {
    r.x = (cval(g, C, i + 1, j, k) - cval(g, C, i - 1, j, k)) * g.hrdx;
    r.y = (cval(g, C, i, j + 1, k) - cval(g, C, i, j - 1, k)) * g.hrdy;
    r.z = (cval(g, C, i, j, k + 1) - cval(g, C, i, j, k - 1)) * __ldg(g.rzc + k);
    return r;
  }
  const double wt[3] = {0.25, 0.5, 0.25};
  double gx = 0, gy = 0, gz = 0;
  for (int s = 0; s < 2; ++s) {
    double ax = 0, ay = 0, az = 0;
    for (int a = -1; a <= 1; ++a) {
      for (int b = -1; b <= 1; ++b) {
        const double wab = wt[a + 1] * wt[b + 1];
        ax += wab * (cval(g, C, i + s, j + a, k + b) - cval(g, C, i + s - 1, j + a, k + b));
        ay += wab * (cval(g, C, i + a, j + s, k + b) - cval(g, C, i + a, j + s - 1, k + b));
        az += wab * (cval(g, C, i + a, j + b, k + s) - cval(g, C, i + a, j + b, k + s - 1));
      }
    }
    gx += ax * g.rdx;
    gy += ay * g.rdy;
    gz += az * __ldg(g.rhz + k + s);
  }
  r.x = 0.5 * gx;
  r.y = 0.5 * gy;
  r.z = 0.5 * gz;
  return r;
}

// |grad C| and the unit normal n = -grad C / |grad C| (zero where clipped) at one cell.
__device__ __forceinline__ double geometry_at(const GridDev& g, const double* __restrict__ C, int i, int j, int k,
                                              int mode, double3& n) {
  const double3 gc = grad_c_at(g, C, i, j, k, mode);
  const double m2 = fma(gc.x, gc.x, fma(gc.y, gc.y, gc.z * gc.z));
  n = make_double3(0.0, 0.0, 0.0);
  if (m2 == 0.0) return 0.0;
  const double r = rsqrt(m2);
  const double c = ldg_in(C, ((size_t)k * g.ny + j) * g.nx + i, ncells(g), CHK_CELL_LOAD);
  if (fmin(c, 1.0 - c) >= 1e-8) {
    n.x = -gc.x * r;
    n.y = -gc.y * r;
    n.z = -gc.z * r;
  }
  return m2 * r;
}

__device__ __forceinline__ double3 normal_at(const GridDev& g, const double* __restrict__ C, int i, int j, int k,
                                             int mode) {
  double3 n;
  geometry_at(g, C, i, j, k, mode, n);
  return n;
}

}  // namespace vofp
