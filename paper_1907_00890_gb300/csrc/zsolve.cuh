// z pass: for every (x, y) spectral pair (q, r) solve
//     a_k p_{k-1} + (b_k + lx_q + ly_r) p_k + c_k p_{k+1} = scale * S_k      (k = 0..nz-1)
// where scale = 1/(nx ny) undoes the unnormalised x and y transforms.  The rows carry the z boundary
// conditions (§3.2 homogeneous conditions: N folds the outer coupling into the diagonal, D subtracts it,
// periodic wraps).  The singular mean mode (no D end anywhere, q = r = 0) first removes the volume-weighted
// mean of its right-hand side (the compatibility defect, reported), pins p_0 = 0, solves rows 1..nz-1 and
// finally shifts to zero volume-weighted mean.  A block stages `ti` neighbouring systems of one y index in
// shared memory so that global loads and stores are row-coalesced; one thread then runs each system's
// recurrence.  The mixed-precision path runs the bulk of the systems in FP32 and its low-eigenvalue
// systems (ill-conditioned in z) in FP64 through k_zlow64.
#pragma once

#include "vofp_internal.cuh"

namespace vofp {

struct ZArgs {
  int nx, ny, nz, bcz;
  int ti;
  int singular;
  double scale;
  double lz;  // sum of dz
  const double* lamx;
  const double* lamy;
  const double* za;
  const double* zb;
  const double* zc;
  const double* dz;
  vofp_devinfo* info;
  void* S;          // spectrum (double or float)
  double lowthr;    // mixed: systems with |lx + ly| <= lowthr are left to k_zlow64 (< 0: none)
  const double* skip_conv;  // mixed: skip the launch when conv[3 + skip_k] <= tol2 * conv[0]
  int skip_k;
  double tol2;
};

// Strided view of one system's column.
template <typename T>
struct Col {
  T* p;
  int s;
  __device__ __forceinline__ T& operator[](int k) const { return p[(size_t)k * s]; }
};

// Thomas elimination on rows k0..k1 with the first row's sub-diagonal and the last row's super-diagonal
// dropped, `add0` / `add1` added to the first / last diagonal.  d: right-hand side in, solution out.
template <typename TA>
__device__ __forceinline__ void thomas_col(Col<TA> d, Col<TA> cp, int k0, int k1, TA lam,
                                           const double* __restrict__ za, const double* __restrict__ zb,
                                           const double* __restrict__ zc, TA add0, TA add1) {
  TA den = (TA)__ldg(zb + k0) + lam + add0 + (k0 == k1 ? add1 : (TA)0);
  TA m = (TA)1 / den;
  TA cprev = (k0 < k1 ? (TA)__ldg(zc + k0) : (TA)0) * m;
  TA dprev = d[k0] * m;
  cp[k0] = cprev;
  d[k0] = dprev;
  for (int k = k0 + 1; k <= k1; ++k) {
    const TA ak = (TA)__ldg(za + k);
    den = (TA)__ldg(zb + k) + lam + (k == k1 ? add1 : (TA)0) - ak * cprev;
    m = (TA)1 / den;
    cprev = (k < k1 ? (TA)__ldg(zc + k) : (TA)0) * m;
    dprev = (d[k] - ak * dprev) * m;
    cp[k] = cprev;
    d[k] = dprev;
  }
  TA x = dprev;
  for (int k = k1 - 1; k >= k0; --k) {
    x = d[k] - cp[k] * x;
    d[k] = x;
  }
}

// Solve the system of spectral pair (iq, jq) whose scaled-by-nothing right-hand side is in d (in place).
template <typename TA>
__device__ void solve_column(const ZArgs& a, int iq, int jq, Col<TA> d, Col<TA> cp, Col<TA> zv) {
  const int nz = a.nz;
  const TA lam = (TA)(__ldg(a.lamx + iq) + __ldg(a.lamy + jq));
  for (int k = 0; k < nz; ++k) d[k] = d[k] * (TA)a.scale;
  const bool per = a.bcz == VOFP_BC_P;
  if (a.singular && iq == 0 && jq == 0) {
    TA s = 0;
    for (int k = 0; k < nz; ++k) s += (TA)__ldg(a.dz + k) * d[k];
    const TA defect = s / (TA)a.lz;
    for (int k = 0; k < nz; ++k) d[k] -= defect;
    if (a.info) a.info->compat_defect = (double)defect;
    d[0] = 0;
    if (nz > 1) {
      Col<TA> d1 = {&d[1], d.s}, c1 = {&cp[1], cp.s};
      thomas_col<TA>(d1, c1, 0, nz - 2, (TA)0, a.za + 1, a.zb + 1, a.zc + 1, (TA)0, (TA)0);
    }
    TA mean = 0;
    for (int k = 0; k < nz; ++k) mean += (TA)__ldg(a.dz + k) * d[k];
    mean /= (TA)a.lz;
    for (int k = 0; k < nz; ++k) d[k] -= mean;
  } else if (!per) {
    thomas_col<TA>(d, cp, 0, nz - 1, lam, a.za, a.zb, a.zc, (TA)0, (TA)0);
  } else if (nz == 1) {
    d[0] = d[0] / lam;
  } else if (nz == 2) {
    const TA m00 = (TA)__ldg(a.zb) + lam, m01 = (TA)(__ldg(a.za) + __ldg(a.zc));
    const TA m10 = (TA)(__ldg(a.za + 1) + __ldg(a.zc + 1)), m11 = (TA)__ldg(a.zb + 1) + lam;
    const TA det = m00 * m11 - m01 * m10;
    const TA r0 = d[0], r1 = d[1];
    d[0] = (m11 * r0 - m01 * r1) / det;
    d[1] = (m00 * r1 - m10 * r0) / det;
  } else {
    // cyclic: A = T + u v^T, u = (gamma, 0, .., beta), v = (1, 0, .., alpha / gamma)
    const TA alpha = (TA)__ldg(a.za), beta = (TA)__ldg(a.zc + nz - 1);
    const TA gamma = -((TA)__ldg(a.zb) + lam);
    for (int k = 0; k < nz; ++k) zv[k] = 0;
    zv[0] = gamma;
    zv[nz - 1] = beta;
    const TA add0 = -gamma, add1 = -alpha * beta / gamma;
    // both eliminations share the factors: run the z-vector with its own copy of cp
    thomas_col<TA>(d, cp, 0, nz - 1, lam, a.za, a.zb, a.zc, add0, add1);
    thomas_col<TA>(zv, cp, 0, nz - 1, lam, a.za, a.zb, a.zc, add0, add1);
    const TA vy = d[0] + alpha / gamma * d[nz - 1];
    const TA vz = zv[0] + alpha / gamma * zv[nz - 1];
    const TA f = vy / ((TA)1 + vz);
    for (int k = 0; k < nz; ++k) d[k] -= f * zv[k];
  }
  if (a.info) {
    bool bad = false;
    for (int k = 0; k < nz; ++k) bad |= !isfinite((double)d[k]);
    if (bad) atomicOr(&a.info->nonfinite, 1u);
  }
}

// One block: `ti` neighbouring x indices of one y index, staged [nz][ti] in shared memory.
template <typename TS, typename TA>
__device__ __forceinline__ void zsolve_block(const ZArgs& a, int bx, int by, unsigned char* smem_raw) {
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const int TI = a.ti, nz = a.nz;
  TA* d = reinterpret_cast<TA*>(smem_raw);
  TA* cp = d + (size_t)nz * TI;
  TA* zv = cp + (size_t)nz * TI;  // periodic z only
  const int i0 = bx * TI;
  const int jq = by;
  const size_t plane = (size_t)a.nx * a.ny;
  const size_t col0 = (size_t)jq * a.nx + i0;
  TS* S = reinterpret_cast<TS*>(a.S);
  for (int t = threadIdx.x; t < nz * TI; t += blockDim.x) {
    const int k = t / TI, c = t - k * TI;
    d[t] = (i0 + c < a.nx) ? (TA)S[k * plane + col0 + c] : (TA)0;
  }
  __syncthreads();
  const int c = threadIdx.x;
  bool mine = c < TI && i0 + c < a.nx;
  if (mine && a.lowthr >= 0) {
    const double lam = __ldg(a.lamx + i0 + c) + __ldg(a.lamy + jq);
    if (fabs(lam) <= a.lowthr) mine = false;  // solved in FP64 by k_zlow64
  }
  if (mine) {
    Col<TA> dd = {d + c, TI}, cc = {cp + c, TI}, zz = {zv + c, TI};
    solve_column<TA>(a, i0 + c, jq, dd, cc, zz);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nz * TI; t += blockDim.x) {
    const int k = t / TI, cc2 = t - k * TI;
    if (i0 + cc2 < a.nx) {
      bool low = false;
      if (a.lowthr >= 0) low = fabs(__ldg(a.lamx + i0 + cc2) + __ldg(a.lamy + jq)) <= a.lowthr;
      if (!low) S[k * plane + col0 + cc2] = (TS)d[t];
    }
  }
}

template <typename TS, typename TA>
__global__ void __launch_bounds__(128) k_zsolve(ZArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zsolve_block<TS, TA>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// Mixed path: the low-eigenvalue systems (listed at plan time) solved in FP64 on their reduced-precision
// spectrum.  Bounded z: plan-time Thomas factors (lowtab[k * nlow + t] = (c'_k, 1/den_k), the singular mean
// mode pinned), so the recurrence has no division; scratch columns are k-major so that consecutive systems
// touch consecutive addresses.  Periodic z: the general column solver on three scratch columns per system.
static __global__ void k_zfactor_low(ZArgs a, const int2* __restrict__ modes, int nlow, double2* tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlow) return;
  const int2 md = modes[t];
  const double lam = a.lamx[md.x] + a.lamy[md.y];
  const bool sing = a.singular && md.x == 0 && md.y == 0;
  const int k0 = sing ? 1 : 0;
  if (sing) tab[t] = make_double2(0.0, 0.0);
  double cprev = 0.0;
  for (int k = k0; k < a.nz; ++k) {
    const double den = a.zb[k] + lam - (k > k0 ? a.za[k] * cprev : 0.0);
    const double m = 1.0 / den;
    const double c = (k < a.nz - 1 ? a.zc[k] : 0.0) * m;
    tab[(size_t)k * nlow + t] = make_double2(c, m);
    cprev = c;
  }
}

template <typename TS>
__device__ __forceinline__ void zlow_system(const ZArgs& a, int2 md, int t, int nlow, const double2* __restrict__ tab,
                                            double* __restrict__ scratch) {
  const int nz = a.nz;
  const size_t plane = (size_t)a.nx * a.ny;
  TS* S = reinterpret_cast<TS*>(a.S);
  const size_t col = (size_t)md.y * a.nx + md.x;
  if (!tab) {
    double* d = scratch + (size_t)t * 3 * nz;
    for (int k = 0; k < nz; ++k) d[k] = (double)S[k * plane + col];
    Col<double> dd = {d, 1}, cc = {d + nz, 1}, zz = {d + 2 * nz, 1};
    solve_column<double>(a, md.x, md.y, dd, cc, zz);
    for (int k = 0; k < nz; ++k) S[k * plane + col] = (TS)d[k];
    return;
  }
  Col<double> d = {scratch + t, nlow};
  const double sc = a.scale;
  for (int k = 0; k < nz; ++k) d[k] = (double)S[k * plane + col] * sc;
  int k0 = 0;
  if (a.singular && md.x == 0 && md.y == 0) {
    double s = 0;
    for (int k = 0; k < nz; ++k) s += __ldg(a.dz + k) * d[k];
    const double defect = s / a.lz;
    if (a.info) a.info->compat_defect = defect;
    for (int k = 0; k < nz; ++k) d[k] -= defect;
    d[0] = 0.0;
    k0 = 1;
  }
  double dprev = 0.0;
  for (int k = k0; k < nz; ++k) {
    const double2 f = __ldg(tab + (size_t)k * nlow + t);
    dprev = (d[k] - (k > k0 ? __ldg(a.za + k) * dprev : 0.0)) * f.y;
    d[k] = dprev;
  }
  double x = dprev;
  for (int k = nz - 2; k >= k0; --k) {
    const double2 f = __ldg(tab + (size_t)k * nlow + t);
    x = fma(-f.x, x, d[k]);
    d[k] = x;
  }
  if (k0 == 1) {
    double mean = 0;
    for (int k = 0; k < nz; ++k) mean += __ldg(a.dz + k) * d[k];
    mean /= a.lz;
    for (int k = 0; k < nz; ++k) d[k] -= mean;
  }
  for (int k = 0; k < nz; ++k) S[k * plane + col] = (TS)d[k];
}

template <typename TS>
__global__ void k_zlow64(ZArgs a, const int2* __restrict__ modes, int nlow, const double2* __restrict__ tab,
                         double* scratch) {
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlow) return;
  zlow_system<TS>(a, modes[t], t, nlow, tab, scratch);
}

// ---- factorisation tables (bounded z, FP64 path) -------------------------------------------------------
// The z matrix of a spectral pair depends only on lx + ly, and the periodic half-complex packing gives the
// real and imaginary parts of one Fourier mode the same eigenvalue, so the Thomas factors (c'_k, 1/den_k) are
// computed once per distinct eigenvalue pair at plan time: table[(k * Uy + uy) * Ux + ux] = (c'_k, m_k).
// The singular mean mode stores the factors of its pinned system (rows 1..nz-1, p_0 = 0).

__device__ __forceinline__ int distinct_index(int q, int bc) { return bc == VOFP_BC_P ? (q + 1) >> 1 : q; }

struct ZTabArgs {
  int Ux, Uy;
  int bcx, bcy;
  const double2* tab;
};

static __global__ void k_zfactor64(ZArgs a, ZTabArgs zt, double2* tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= zt.Ux * zt.Uy) return;
  const int ux = t % zt.Ux, uy = t / zt.Ux;
  const int qx = zt.bcx == VOFP_BC_P ? (ux ? 2 * ux - 1 : 0) : ux;
  const int qy = zt.bcy == VOFP_BC_P ? (uy ? 2 * uy - 1 : 0) : uy;
  const double lam = a.lamx[qx] + a.lamy[qy];
  const bool sing = a.singular && ux == 0 && uy == 0;
  const int k0 = sing ? 1 : 0;
  const size_t stride = (size_t)zt.Ux * zt.Uy;
  if (sing) tab[t] = make_double2(0.0, 0.0);
  double cprev = 0.0;
  for (int k = k0; k < a.nz; ++k) {
    const double den = a.zb[k] + lam - (k > k0 ? a.za[k] * cprev : 0.0);
    const double m = 1.0 / den;
    const double c = (k < a.nz - 1 ? a.zc[k] : 0.0) * m;
    tab[k * stride + t] = make_double2(c, m);
    cprev = c;
  }
}

// Bounded-z solve with precomputed factors: forward d_k = (r_k - a_k d_{k-1}) m_k, back x_k = d_k - c'_k x_{k+1}.
static __global__ void __launch_bounds__(128) k_zsolve64_tab(ZArgs a, ZTabArgs zt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TI = a.ti, nz = a.nz;
  // the recurrences read only shared memory: factors [nz][TI] (double2) and right-hand sides [nz][TI]
  double2* ft = reinterpret_cast<double2*>(smem_raw);
  double* d = reinterpret_cast<double*>(ft + (size_t)nz * TI);
  const int i0 = blockIdx.x * TI;
  const int jq = blockIdx.y;
  const size_t plane = (size_t)a.nx * a.ny;
  const size_t col0 = (size_t)jq * a.nx + i0;
  const size_t stride = (size_t)zt.Ux * zt.Uy;
  const double2* Trow = zt.tab + (size_t)distinct_index(jq, zt.bcy) * zt.Ux;
  double* S = reinterpret_cast<double*>(a.S);
  for (int t = threadIdx.x; t < nz * TI; t += blockDim.x) {
    const int k = t / TI, c = t - k * TI;
    const bool in = i0 + c < a.nx;
    d[t] = in ? S[k * plane + col0 + c] : 0.0;
    ft[t] = in ? __ldg(Trow + k * stride + distinct_index(i0 + c, zt.bcx)) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < TI && i0 + c < a.nx) {
    const int iq = i0 + c;
    const double2* T = ft + c;
    const size_t stride = TI;  // shadows the table stride: factors are now staged [nz][TI]
    const double sc = a.scale;
    int k0 = 0;
    if (a.singular && iq == 0 && jq == 0) {
      double s = 0;
      for (int k = 0; k < nz; ++k) s += __ldg(a.dz + k) * d[k * TI + c];
      const double defect = s * sc / a.lz;
      if (a.info) a.info->compat_defect = defect;
      for (int k = 0; k < nz; ++k) d[k * TI + c] = d[k * TI + c] * sc - defect;
      d[c] = 0.0;
      k0 = 1;
      double dprev = 0.0;
      for (int k = 1; k < nz; ++k) {
        const double2 f = T[k * stride];
        dprev = (d[k * TI + c] - (k > 1 ? __ldg(a.za + k) * dprev : 0.0)) * f.y;
        d[k * TI + c] = dprev;
      }
    } else {
      double dprev = 0.0;
#pragma unroll 4
      for (int k = 0; k < nz; ++k) {
        const double2 f = T[k * stride];
        dprev = fma(d[k * TI + c], sc, -__ldg(a.za + k) * dprev) * f.y;
        d[k * TI + c] = dprev;
      }
    }
    double x = d[(nz - 1) * TI + c];
#pragma unroll 4
    for (int k = nz - 2; k >= k0; --k) {
      const double2 f = T[k * stride];
      x = fma(-f.x, x, d[k * TI + c]);
      d[k * TI + c] = x;
    }
    if (k0 == 1) {
      double mean = 0;
      for (int k = 0; k < nz; ++k) mean += __ldg(a.dz + k) * d[k * TI + c];
      mean /= a.lz;
      for (int k = 0; k < nz; ++k) d[k * TI + c] -= mean;
    }
    if (a.info) {
      bool bad = false;
      for (int k = 0; k < nz; ++k) bad |= !isfinite(d[k * TI + c]);
      if (bad) atomicOr(&a.info->nonfinite, 1u);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nz * TI; t += blockDim.x) {
    const int k = t / TI, cc = t - k * TI;
    if (i0 + cc < a.nx) S[k * plane + col0 + cc] = d[t];
  }
}

}  // namespace vofp
