// Face epilogues and the interface-geometry pass:
//   * pressure correction u = u* - (dt/rho0) G p (§3.2, the step after Eq. lap_p);
//   * interface geometry per cell: s = mdot (1/rho2 - 1/rho1) |grad C| (Eq. ext_div right-hand side, the
//     source of Eq. lap_p) and n = -grad C / |grad C| (Eq. int_vel), computed once and kept in the plan;
//   * liquid-velocity extension u1e = u - G phi (Eq. jump_subtr) and interface velocity
//     uG = u1e - (mdot_f / rho1) n_f (Eq. int_vel), reading the stored n.
#pragma once

#include "stencil.cuh"

namespace vofp {

// The cell line along `axis` through (i, j, k) lies inside the cell array (bounds-checked builds; offsets along
// the line then run over 0 .. n - 1).
__device__ __forceinline__ bool line_in(const GridDev& g, int axis, int i, int j, int k) {
  const size_t plane = (size_t)g.nx * g.ny;
  const size_t last = axis == 0 ? (size_t)k * plane + (size_t)j * g.nx + (g.nx - 1)
                                : (axis == 1 ? (size_t)k * plane + i + (size_t)(g.ny - 1) * g.nx
                                             : (size_t)j * g.nx + i + (size_t)(g.nz - 1) * plane);
  return VOFP_IN(last, ncells(g), CHK_FACE_LINE);
}

// The difference d of a cell field across face f (low face of cell f) of a line of n cells with stride `st`
// from `base`: returns -1 on an N face (no difference), 0 inside or across a periodic wrap (d = q_f - q_{f-1}),
// 1 / 2 on the low / high D face (d = the adjacent value with the ghost's sign, the distance half a cell).  The
// face-normal gradient is d * face_rdist(...).
__device__ __forceinline__ int line_diff(const double* __restrict__ p, size_t base, size_t st, int n, int bc, int f,
                                         double& d) {
  if (bc == VOFP_BC_P) {
    const int fm = f == 0 ? n - 1 : f - 1;
    d = __ldg(p + base + f * st) - __ldg(p + base + fm * st);
    return 0;
  }
  if (f == 0) {
    if (bc == VOFP_BC_NN || bc == VOFP_BC_ND) return -1;
    d = __ldg(p + base);
    return 1;
  }
  if (f == n) {
    if (bc == VOFP_BC_NN || bc == VOFP_BC_DN) return -1;
    d = -__ldg(p + base + (size_t)(n - 1) * st);
    return 2;
  }
  d = __ldg(p + base + f * st) - __ldg(p + base + (size_t)(f - 1) * st);
  return 0;
}
__device__ __forceinline__ int face_diff_axis(const GridDev& g, const double* __restrict__ p, int axis, int i, int j,
                                              int k, double& d) {
  if (!line_in(g, axis, i, j, k)) return -1;
  const size_t plane = (size_t)g.nx * g.ny;
  if (axis == 0) return line_diff(p, (size_t)k * plane + (size_t)j * g.nx, 1, g.nx, g.bcx, i, d);
  if (axis == 1) return line_diff(p, (size_t)k * plane + i, g.nx, g.ny, g.bcy, j, d);
  return line_diff(p, (size_t)j * g.nx + i, plane, g.nz, g.bcz, k, d);
}

// 1 / distance between the two values that face_diff_axis differences (return code e >= 0): the centre distance
// inside and across a periodic wrap, half the end cell's width at a D face.
__device__ __forceinline__ double face_rdist(const GridDev& g, int axis, int k, int e) {
  const double h = axis == 0 ? g.rdx
                             : (axis == 1 ? g.rdy : (e == 0 ? __ldg(g.rhz + k) : __ldg(g.rdz + (e == 1 ? 0 : g.nz - 1))));
  return e > 0 ? h + h : h;
}

// Blocks per plane and axis of the face launch shape (face_grid).
__host__ __device__ __forceinline__ int face_blocks_per_plane(const GridDev& g, int threads) {
  const long a = (long)nface(g.nx, g.bcx) * g.ny, b = (long)g.nx * nface(g.ny, g.bcy), c = (long)g.nx * g.ny;
  const long m = a > b ? (a > c ? a : c) : (b > c ? b : c);
  return (int)((m + threads - 1) / threads);
}
// Face launch shape: blockIdx.z = plane k, blockIdx.y = axis, blockIdx.x * blockDim.x + threadIdx.x = index
// within the plane of that axis' face array (32-bit arithmetic; no 64-bit division per face).  Blocks run
// x fastest, then y: the three face arrays of plane k are done back to back, so the cell fields they share
// (the potential, mdot, C) are read from DRAM once and then hit L2, instead of once per axis.
inline dim3 face_grid(const GridDev& g, int threads) {
  return dim3((unsigned)face_blocks_per_plane(g, threads), 3, (unsigned)(g.nz + 1));
}
// Decode a flat face index over the three face arrays (u, then v, then w); returns the axis and sets (i, j, k)
// and the offset in that axis' array.
__device__ __forceinline__ int decode_face(const GridDev& g, size_t t, int& i, int& j, int& k, size_t& off) {
  const int nxf = nface(g.nx, g.bcx), nyf = nface(g.ny, g.bcy);
  const size_t nu = (size_t)nxf * g.ny * g.nz, nv = (size_t)g.nx * nyf * g.nz;
  int fx = nxf, fy = g.ny, axis = 0;
  if (t >= nu) {
    t -= nu;
    fx = g.nx;
    fy = nyf;
    axis = 1;
    if (t >= nv) {
      t -= nv;
      fy = g.ny;
      axis = 2;
    }
  }
  off = t;
  i = (int)(t % fx);
  const size_t r = t / fx;
  j = (int)(r % fy);
  k = (int)(r / fy);
  return axis;
}
__host__ __device__ __forceinline__ size_t total_faces(const GridDev& g) {
  return (size_t)nface(g.nx, g.bcx) * g.ny * g.nz + (size_t)g.nx * nface(g.ny, g.bcy) * g.nz +
         (size_t)g.nx * g.ny * nface(g.nz, g.bcz);
}

// Face `idx` of plane k of the `axis` face array: sets (i, j) and the offset; false past the plane or the
// array.  (32-bit arithmetic, one division.)
__device__ __forceinline__ bool face_at(const GridDev& g, int axis, int k, int idx, int& i, int& j, size_t& off) {
  const int fx = axis == 0 ? nface(g.nx, g.bcx) : g.nx;
  const int fy = axis == 1 ? nface(g.ny, g.bcy) : g.ny;
  const int fz = axis == 2 ? nface(g.nz, g.bcz) : g.nz;
  if (k >= fz || idx >= fx * fy) return false;
  j = idx / fx;
  i = idx - j * fx;
  off = ((size_t)k * fy + j) * fx + i;
  return VOFP_IN(off, (size_t)fx * fy * fz, CHK_FACE_STORE);
}
__device__ __forceinline__ bool face_coord(const GridDev& g, int& axis, int& i, int& j, int& k, size_t& off) {
  axis = blockIdx.y;
  k = blockIdx.z;
  return face_at(g, axis, k, blockIdx.x * blockDim.x + threadIdx.x, i, j, off);
}

// u -= s * G p on all three face arrays; sx = s / dx, sy = s / dy (the x and y scales folded into one product,
// so that an x or y face costs one subtraction and one multiply-add in FP64).
__device__ __forceinline__ void grad_face(const GridDev& g, const double* __restrict__ p, double* u, double* v,
                                          double* w, double s, double sx, double sy, int axis, int i, int j, int k,
                                          size_t off) {
  double d;
  const int e = face_diff_axis(g, p, axis, i, j, k, d);
  if (e < 0) return;  // N face
  double c = axis == 0 ? sx : (axis == 1 ? sy : s * (e == 0 ? __ldg(g.rhz + k) : __ldg(g.rdz + (e == 1 ? 0 : g.nz - 1))));
  if (e > 0) c = c + c;
  double* F = axis == 0 ? u : (axis == 1 ? v : w);
  F[off] = fma(-c, d, F[off]);
}
static __global__ void __launch_bounds__(256) k_grad_update(GridDev g, const double* __restrict__ p, double* u,
                                                           double* v, double* w, double s, double sx, double sy) {
  int axis, i, j, k;
  size_t off;
  if (!face_coord(g, axis, i, j, k, off)) return;
  grad_face(g, p, u, v, w, s, sx, sy, axis, i, j, k, off);
}

// Interface geometry per cell: s = coef * mdot * |grad C| and n = -grad C / |grad C| (clipped).  The
// gradient stencil is a template argument (0 central, 1 Youngs) so each kernel carries only its own.
template <int MODE>
static __global__ void __launch_bounds__(256) k_geometry(GridDev g, const double* __restrict__ C,
                                                        const double* __restrict__ mdot, double coef,
                                                        double* __restrict__ s, double* __restrict__ nx,
                                                        double* __restrict__ ny, double* __restrict__ nz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= g.nx) return;
  const size_t t = ((size_t)k * g.ny + j) * g.nx + i;
  if (!VOFP_IN(t, ncells(g), CHK_CELL_STORE)) return;
  double3 n;
  const double m = geometry_at(g, C, i, j, k, MODE, n);
  s[t] = __ldg(mdot + t) * coef * m;
  if (nx) {
    nx[t] = n.x;
    ny[t] = n.y;
    nz[t] = n.z;
  }
}
// The same geometry for reduced-precision plans (central differences): the C differences are taken in FP64,
// everything after them -- scaling, |grad C|^2, the reciprocal square root (FP32 seed and one FP32-pair
// Newton step), s and n -- in FP32 pairs, with integer-pipe conversions; FP64 work per cell drops from some
// 25 operations to 9.  Results agree with the FP64 kernel to about 1e-14 relative.
static __global__ void __launch_bounds__(256) k_geometry_ff(GridDev g, const double* __restrict__ C,
                                                           const double* __restrict__ mdot, double coef,
                                                           double* __restrict__ s, double* __restrict__ nx,
                                                           double* __restrict__ ny, double* __restrict__ nz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= g.nx) return;
  const size_t t = ((size_t)k * g.ny + j) * g.nx + i;
  if (!VOFP_IN(t, ncells(g), CHK_CELL_STORE)) return;
  const ff gx = ff_split(cval(g, C, i + 1, j, k) - cval(g, C, i - 1, j, k)) * ff_split(g.hrdx);
  const ff gy = ff_split(cval(g, C, i, j + 1, k) - cval(g, C, i, j - 1, k)) * ff_split(g.hrdy);
  const ff gz = ff_split(cval(g, C, i, j, k + 1) - cval(g, C, i, j, k - 1)) * ff_split(__ldg(g.rzc + k));
  const ff m2 = gx * gx + gy * gy + gz * gz;
  double sv = 0.0, n0 = 0.0, n1 = 0.0, n2 = 0.0;
  if (m2.hi > 0.0f) {
    const float y0 = rsqrtf(m2.hi);
    const ff y(y0, 0.0f);
    const ff r = y * (ff(1.5f, 0.0f) - ff(0.5f, 0.0f) * (m2 * y * y));  // one Newton step for 1/sqrt(m2)
    sv = wide_of(ff_split(__ldg(mdot + t) * coef) * (m2 * r));
    const double c = __ldg(C + t);
    if (fmin(c, 1.0 - c) >= 1e-8) {
      n0 = wide_of(-(gx * r));
      n1 = wide_of(-(gy * r));
      n2 = wide_of(-(gz * r));
    }
  }
  s[t] = sv;
  if (nx) {
    nx[t] = n0;
    ny[t] = n1;
    nz[t] = n2;
  }
}

inline dim3 cell_grid(const GridDev& g, int threads) {
  return dim3((unsigned)((g.nx + threads - 1) / threads), (unsigned)g.ny, (unsigned)g.nz);
}

// Twice the mean of a cell array over the cells adjacent to face (axis, i, j, k): the sum of the two
// neighbours, or twice the one adjacent cell on a bounded axis' end face.
__device__ __forceinline__ double face_sum_arr(const GridDev& g, const double* __restrict__ q, int axis, int i,
                                                int j, int k) {
  int n, bc, f;
  size_t st;
  const size_t plane = (size_t)g.nx * g.ny;
  size_t base;
  if (axis == 0) {
    n = g.nx, bc = g.bcx, f = i, st = 1, base = (size_t)k * plane + (size_t)j * g.nx;
  } else if (axis == 1) {
    n = g.ny, bc = g.bcy, f = j, st = g.nx, base = (size_t)k * plane + i;
  } else {
    n = g.nz, bc = g.bcz, f = k, st = plane, base = (size_t)j * g.nx + i;
  }
  int lo = f - 1, hi = f;
  if (bc == VOFP_BC_P) {
    if (lo < 0) lo += n;
  } else {
    if (lo < 0) lo = 0;
    if (hi >= n) hi = n - 1;
  }
  if (!line_in(g, axis, i, j, k)) return 0.0;
  return __ldg(q + base + lo * st) + __ldg(q + base + hi * st);
}

struct ExtArgs {
  GridDev g;
  const double* phi;
  const double* u;
  const double* v;
  const double* w;
  const double* mdot;
  const double* n[3];  // stored cell normals
  double quarter_inv_rho1;  // 1 / (4 rho1)
  double* ue;
  double* ve;
  double* we;
  double* ug;
  double* vg;
  double* wg;
};

static __global__ void __launch_bounds__(256) k_extend_epi(ExtArgs a) {
  const GridDev& g = a.g;
  int axis, i, j, k;
  size_t off;
  if (!face_coord(g, axis, i, j, k, off)) return;
  const double* U = axis == 0 ? a.u : (axis == 1 ? a.v : a.w);
  double d;
  const int e = face_diff_axis(g, a.phi, axis, i, j, k, d);
  const double ue = e < 0 ? __ldg(U + off) : fma(-face_rdist(g, axis, k, e), d, __ldg(U + off));
  (axis == 0 ? a.ue : (axis == 1 ? a.ve : a.we))[off] = ue;
  if (a.ug) {
    // (mean mdot)(mean n) / rho1 = (sum mdot)(sum n) / (4 rho1)
    const double md = face_sum_arr(g, a.mdot, axis, i, j, k);
    const double nf = face_sum_arr(g, a.n[axis], axis, i, j, k);
    (axis == 0 ? a.ug : (axis == 1 ? a.vg : a.wg))[off] = fma(-a.quarter_inv_rho1 * md, nf, ue);
  }
}

// Variable-density pressure splitting (§3.2, Eq. lap_p and the update after it): u* -= dt (1/rho_f - 1/rho0)
// G p_hat on every face, p_hat = (1 + r) p^n - r p^{n-1} (p^n alone when pm is NULL), rho_f = rho2 + (rho1 -
// rho2) C_f with C_f the mean of C over the face's two cells (its one cell at a bounded end); N faces carry no
// flux.  The constant-coefficient projection of the result with dt/rho0 completes the step.
struct VdArgs {
  GridDev g;
  const double* pn;
  const double* pm;
  double opr, r;        // 1 + dt/dt_prev, dt/dt_prev
  const double* C;
  double half_drho;     // (rho1 - rho2) / 2
  double rho2;
  double dt;
  double dt_over_rho0;
  double* u;
  double* v;
  double* w;
};
static __global__ void __launch_bounds__(256) k_vd_predict(VdArgs a) {
  const GridDev& g = a.g;
  int axis, i, j, k;
  size_t off;
  if (!face_coord(g, axis, i, j, k, off)) return;
  double d;
  const int e = face_diff_axis(g, a.pn, axis, i, j, k, d);
  if (e < 0) return;  // N face: no flux
  if (a.pm) {
    double dm;
    face_diff_axis(g, a.pm, axis, i, j, k, dm);
    d = fma(a.opr, d, -a.r * dm);  // the difference of p_hat
  }
  const double h = face_rdist(g, axis, k, e);  // 1 / distance between the values differenced
  const double rho_f = fma(a.half_drho, face_sum_arr(g, a.C, axis, i, j, k), a.rho2);
  const double c = h * fma(a.dt, recip_newton(rho_f), -a.dt_over_rho0);  // dt (1/rho_f - 1/rho0) / distance
  double* F = axis == 0 ? a.u : (axis == 1 ? a.v : a.w);
  F[off] = fma(-c, d, F[off]);
}

}  // namespace vofp
