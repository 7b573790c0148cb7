// Face epilogues: pressure correction u = u* - (dt/rho0) G p (§3.2, the step after Eq. lap_p) and the
// liquid-velocity extension u1e = u - G phi (Eq. jump_subtr) with the interface velocity
// uG = u1e - (mdot_f / rho1) n_f (Eq. int_vel).
#pragma once

#include "stencil.cuh"

namespace vofp {

// Face-normal gradient of a cell field at face `f` (low face of cell f) along a line of n cells with
// stride `st` starting at `base`.  Returns false for an N boundary face (left unchanged).
__device__ __forceinline__ bool face_grad(const double* __restrict__ p, size_t base, size_t st, int n, int bc, int f,
                                          double h_lo_ghost, double h_interior_or_wrap, double w_lo, double w_hi,
                                          double& g) {
  if (bc == VOFP_BC_P) {
    const int fm = f == 0 ? n - 1 : f - 1;
    g = (__ldg(p + base + f * st) - __ldg(p + base + fm * st)) / h_interior_or_wrap;
    return true;
  }
  const bool lowN = bc == VOFP_BC_NN || bc == VOFP_BC_ND;
  const bool highN = bc == VOFP_BC_NN || bc == VOFP_BC_DN;
  if (f == 0) {
    if (lowN) return false;
    g = 2.0 * __ldg(p + base) / w_lo;
    return true;
  }
  if (f == n) {
    if (highN) return false;
    g = -2.0 * __ldg(p + base + (size_t)(n - 1) * st) / w_hi;
    return true;
  }
  g = (__ldg(p + base + f * st) - __ldg(p + base + (size_t)(f - 1) * st)) / h_interior_or_wrap;
  (void)h_lo_ghost;
  return true;
}

// Decode a flat face index over the three face arrays; returns the axis and sets (i, j, k) and the offset.
__device__ __forceinline__ int decode_face(const GridDev& g, size_t t, int& i, int& j, int& k, size_t& off) {
  const int nxf = nface(g.nx, g.bcx), nyf = nface(g.ny, g.bcy), nzf = nface(g.nz, g.bcz);
  const size_t nu = (size_t)nxf * g.ny * g.nz, nv = (size_t)g.nx * nyf * g.nz;
  if (t < nu) {
    off = t;
    i = (int)(t % nxf);
    const size_t r = t / nxf;
    j = (int)(r % g.ny);
    k = (int)(r / g.ny);
    return 0;
  }
  t -= nu;
  if (t < nv) {
    off = t;
    i = (int)(t % g.nx);
    const size_t r = t / g.nx;
    j = (int)(r % nyf);
    k = (int)(r / nyf);
    return 1;
  }
  t -= nv;
  off = t;
  i = (int)(t % g.nx);
  const size_t r = t / g.nx;
  j = (int)(r % g.ny);
  k = (int)(r / g.ny);
  (void)nzf;
  return 2;
}

__device__ __forceinline__ bool grad_on_face(const GridDev& g, const double* __restrict__ p, int axis, int i, int j,
                                             int k, double& gr) {
  const size_t plane = (size_t)g.nx * g.ny;
  if (axis == 0) {
    return face_grad(p, (size_t)k * plane + (size_t)j * g.nx, 1, g.nx, g.bcx, i, 0, g.dx, g.dx, g.dx, gr);
  } else if (axis == 1) {
    return face_grad(p, (size_t)k * plane + i, g.nx, g.ny, g.bcy, j, 0, g.dy, g.dy, g.dy, gr);
  }
  const double h = __ldg(g.hz + k);  // centre distance across z face k (wrap distance at k = 0 if periodic)
  return face_grad(p, (size_t)j * g.nx + i, plane, g.nz, g.bcz, k, 0, h, __ldg(g.dz), __ldg(g.dz + g.nz - 1), gr);
}

// u -= s * G p on all three face arrays (one flat index space).
__global__ void k_grad_update(GridDev g, const double* __restrict__ p, double* u, double* v, double* w, double s) {
  const size_t total = (size_t)nface(g.nx, g.bcx) * g.ny * g.nz + (size_t)g.nx * nface(g.ny, g.bcy) * g.nz +
                       (size_t)g.nx * g.ny * nface(g.nz, g.bcz);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int i, j, k;
    size_t off;
    const int axis = decode_face(g, t, i, j, k, off);
    double gr;
    if (!grad_on_face(g, p, axis, i, j, k, gr)) continue;
    double* F = axis == 0 ? u : (axis == 1 ? v : w);
    F[off] -= s * gr;
  }
}

// Mean of a cell quantity over the cells adjacent to face (axis, i, j, k).
template <typename FN>
__device__ __forceinline__ double face_mean(const GridDev& g, int axis, int i, int j, int k, FN cell) {
  int n, bc, f;
  if (axis == 0) {
    n = g.nx;
    bc = g.bcx;
    f = i;
  } else if (axis == 1) {
    n = g.ny;
    bc = g.bcy;
    f = j;
  } else {
    n = g.nz;
    bc = g.bcz;
    f = k;
  }
  int lo = f - 1, hi = f;
  if (bc == VOFP_BC_P) {
    if (lo < 0) lo += n;
  } else {
    if (lo < 0) lo = 0;
    if (hi >= n) hi = n - 1;
  }
  auto at = [&](int c) {
    if (axis == 0) return cell(c, j, k);
    if (axis == 1) return cell(i, c, k);
    return cell(i, j, c);
  };
  return 0.5 * (at(lo) + at(hi));
}

struct ExtArgs {
  GridDev g;
  const double* phi;
  const double* u;
  const double* v;
  const double* w;
  const double* C;
  const double* mdot;
  double inv_rho1;
  int grad_mode;
  double* ue;
  double* ve;
  double* we;
  double* ug;
  double* vg;
  double* wg;
};

__global__ void k_extend_epi(ExtArgs a) {
  const GridDev& g = a.g;
  const size_t total = (size_t)nface(g.nx, g.bcx) * g.ny * g.nz + (size_t)g.nx * nface(g.ny, g.bcy) * g.nz +
                       (size_t)g.nx * g.ny * nface(g.nz, g.bcz);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int i, j, k;
    size_t off;
    const int axis = decode_face(g, t, i, j, k, off);
    const double* U = axis == 0 ? a.u : (axis == 1 ? a.v : a.w);
    double gr = 0;
    grad_on_face(g, a.phi, axis, i, j, k, gr);
    const double ue = __ldg(U + off) - gr;
    (axis == 0 ? a.ue : (axis == 1 ? a.ve : a.we))[off] = ue;
    if (a.ug) {
      const double md = face_mean(g, axis, i, j, k, [&](int ci, int cj, int ck) {
        return __ldg(a.mdot + ((size_t)ck * g.ny + cj) * g.nx + ci);
      });
      const double nf = face_mean(g, axis, i, j, k, [&](int ci, int cj, int ck) {
        const double3 n = normal_at(g, a.C, ci, cj, ck, a.grad_mode);
        return axis == 0 ? n.x : (axis == 1 ? n.y : n.z);
      });
      (axis == 0 ? a.ug : (axis == 1 ? a.vg : a.wg))[off] = ue - md * a.inv_rho1 * nf;
    }
  }
}

}  // namespace vofp
