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
    d[t] = (i0 + c < a.nx && VOFP_IN(col0 + c, plane, CHK_Z_COLUMN)) ? (TA)S[k * plane + col0 + c] : (TA)0;
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
    if (i0 + cc2 < a.nx && VOFP_IN(col0 + cc2, plane, CHK_Z_COLUMN)) {
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
  if (!VOFP_IN(md.x, a.nx, CHK_Z_TABLE) || !VOFP_IN(md.y, a.ny, CHK_Z_TABLE)) return;
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
  if (!VOFP_IN(col, plane, CHK_Z_COLUMN) || !VOFP_IN(md.x, a.nx, CHK_Z_COLUMN)) return;
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

// ---- factorisation tables (bounded z) -------------------------------------------------------------------
// The z matrix of a spectral pair depends only on lx + ly, and the periodic half-complex packing gives the
// real and imaginary parts of one Fourier mode the same eigenvalue, so the Thomas factors (c'_k, 1/den_k) are
// computed once per distinct eigenvalue pair at plan time (in FP64, stored in the plan's arithmetic type):
// table[(k * Uy + uy) * Ux + ux] = (c'_k, m_k).  The singular mean mode stores the factors of its pinned
// system (rows 1..nz-1, p_0 = 0).

__device__ __forceinline__ int distinct_index(int q, int bc) { return bc == VOFP_BC_P ? (q + 1) >> 1 : q; }

struct ZTabArgs {
  int Ux, Uy;
  int bcx, bcy;
  const void* tab;     // [nz][Uy][Ux] factor pairs in the plan's arithmetic type
  const void* za;      // a_k in the same type
  const int* lowcut;   // refinement plans: column i of row j is a low mode iff i < lowcut[j]; NULL: none
};

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ ff fma_t(ff a, ff b, ff c) { return a * b + c; }

// Factor-table element: c' = c'_k (back substitution), ms = s m_k (forward, with the transform scale s of the
// z pass folded in), al = alpha_k = -a_k m_k (0 on the first eliminated row).  Forward: d_k = al d_{k-1} +
// ms r_k; back: x_k = d_k - c' x_{k+1}; x is the scaled solution.
template <typename T>
struct ZF {
  T c, ms, al;
};

__device__ __forceinline__ ZF<double> make_factor(double c, double ms, double al, ZF<double>*) { return {c, ms, al}; }
__device__ __forceinline__ ZF<float> make_factor(double c, double ms, double al, ZF<float>*) {
  return {(float)c, (float)ms, (float)al};
}
__device__ __forceinline__ ZF<ff> make_factor(double c, double ms, double al, ZF<ff>*) {
  return {ff(c), ff(ms), ff(al)};
}

template <typename TT>
static __global__ void k_zfactor(ZArgs a, ZTabArgs zt, TT* tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= zt.Ux * zt.Uy) return;
  const int ux = t % zt.Ux, uy = t / zt.Ux;
  const int qx = zt.bcx == VOFP_BC_P ? (ux ? 2 * ux - 1 : 0) : ux;
  const int qy = zt.bcy == VOFP_BC_P ? (uy ? 2 * uy - 1 : 0) : uy;
  if (!VOFP_IN(qx, a.nx, CHK_Z_TABLE) || !VOFP_IN(qy, a.ny, CHK_Z_TABLE)) return;
  const double lam = a.lamx[qx] + a.lamy[qy];
  const bool sing = a.singular && ux == 0 && uy == 0;
  const int k0 = sing ? 1 : 0;
  const size_t stride = (size_t)zt.Ux * zt.Uy;
  if (sing) tab[t] = make_factor(0.0, 0.0, 0.0, (TT*)nullptr);
  double cprev = 0.0;
  for (int k = k0; k < a.nz; ++k) {
    const double den = a.zb[k] + lam - (k > k0 ? a.za[k] * cprev : 0.0);
    const double m = 1.0 / den;
    const double c = (k < a.nz - 1 ? a.zc[k] : 0.0) * m;
    tab[k * stride + t] = make_factor(c, a.scale * m, k > k0 ? -a.za[k] * m : 0.0, (TT*)nullptr);
    cprev = c;
  }
}

// Bounded-z solve with precomputed factors, one thread per system, `blockDim.x` neighbouring x indices of one
// y index per block: forward d_k = (r_k - a_k d_{k-1}) m_k, back x_k = d_k - c'_k x_{k+1}, x scaled on the
// way out.  Right-hand sides are read and solutions written row by row (coalesced across the warp); the
// forward values d_k are kept in shared memory ([nz][blockDim.x], SMEM) or in place in the spectrum.  Written
// as d_k = alpha_k d_{k-1} + beta_k (alpha_k = -a_k m_k, beta_k = s r_k m_k, both off the chain) and
// x_k = d_k - c'_k x_{k+1}, each recurrence has one dependent multiply-add per row (FP64 latency is some 64
// cycles on this GPU); the loads of rows k + 1 .. k + 8 are issued before row k is used (a register ring).
template <typename T, typename TT, bool SMEM>
__device__ __forceinline__ bool ztab_sweep(T* __restrict__ col, T* __restrict__ dsm, size_t plane, int TI,
                                           const TT* __restrict__ F, size_t ts, const T* __restrict__ za, int nz,
                                           T sc, bool check) {
  constexpr int U = 8;
  T rb[U];
  TT fb[U];  // ZF<T>
#pragma unroll
  for (int u = 0; u < U; ++u)
    if (u < nz) {
      rb[u] = col[u * plane];
      fb[u] = F[u * ts];
    }
  T dprev = (T)0;
  for (int k0 = 0; k0 < nz; k0 += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      if (k < nz) {
        const T al = fb[u].al, be = rb[u] * fb[u].ms;  // off the dependent chain
        if (k + U < nz) {
          rb[u] = col[(k + U) * plane];
          fb[u] = F[(k + U) * ts];
        }
        dprev = fma_t(al, dprev, be);
        if (SMEM)
          dsm[k * TI] = dprev;
        else
          col[k * plane] = dprev;
      }
    }
  }
  bool bad = false;
  T x = dprev;
  col[(size_t)(nz - 1) * plane] = x;
  if (check) bad |= !isfinite((double)x);
  T db[U], cb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int k = nz - 2 - u;
    if (k >= 0) {
      db[u] = SMEM ? dsm[k * TI] : col[k * plane];
      cb[u] = F[k * ts].c;
    }
  }
  for (int k0 = nz - 2; k0 >= 0; k0 -= U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 - u;
      if (k >= 0) {
        const T d = db[u], c = cb[u];
        if (k - U >= 0) {
          db[u] = SMEM ? dsm[(k - U) * TI] : col[(k - U) * plane];
          cb[u] = F[(k - U) * ts].c;
        }
        x = fma_t(-c, x, d);
        col[k * plane] = x;
        if (check) bad |= !isfinite((double)x);
      }
    }
  }
  return bad;
}

// The pinned mean mode (singular operator, q = r = 0): remove the volume-weighted mean of its right-hand
// side (the compatibility defect), fix p_0 = 0, eliminate rows 1..nz-1 (the table holds the pinned system's
// factors), back-substitute, shift to zero volume-weighted mean.  One thread; `dcol` / `ds` is its
// forward-value column.
template <typename T, typename TT>
__device__ bool ztab_singular(const ZArgs& a, T* col, T* dcol, size_t ds, size_t plane, const TT* F, size_t ts) {
  const int nz = a.nz;
  T s = (T)0;
  for (int k = 0; k < nz; ++k) s += (T)__ldg(a.dz + k) * col[k * plane];
  const T defect = s / (T)a.lz;  // of the unscaled right-hand side
  if (a.info) a.info->compat_defect = (double)defect * a.scale;
  T dp = (T)0;
  for (int k = 1; k < nz; ++k) {
    const TT f = F[k * ts];
    dp = fma_t(f.al, dp, (col[k * plane] - defect) * f.ms);
    dcol[k * ds] = dp;
  }
  T x = dp;
  for (int k = nz - 2; k >= 1; --k) {
    x = dcol[k * ds] - F[k * ts].c * x;
    dcol[k * ds] = x;
  }
  dcol[0] = (T)0;
  T mean = (T)0;
  for (int k = 0; k < nz; ++k) mean += (T)__ldg(a.dz + k) * dcol[k * ds];
  mean = mean / (T)a.lz;
  bool bad = false;
  for (int k = 0; k < nz; ++k) {
    const T o = dcol[k * ds] - mean;
    col[k * plane] = o;
    bad |= !isfinite((double)o);
  }
  return bad;
}

template <typename T, typename TT>
__device__ __forceinline__ void ztab_block(const ZArgs& a, const ZTabArgs& zt, int smem_d, int bx, int by,
                                           unsigned char* smem_raw) {
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const int TI = blockDim.x, nz = a.nz;
  const int c = threadIdx.x;
  const int i = bx * TI + c, j = by;
  if (i >= a.nx) return;
  if (zt.lowcut && i < __ldg(zt.lowcut + j)) return;  // solved in FP64 by the low-mode kernel
  const size_t plane = (size_t)a.nx * a.ny;
  T* col = reinterpret_cast<T*>(a.S) + (size_t)j * a.nx + i;
  T* dsm = reinterpret_cast<T*>(smem_raw) + c;
  const size_t ts = (size_t)zt.Ux * zt.Uy;
  if (!VOFP_IN((size_t)j * a.nx + i, plane, CHK_Z_COLUMN) ||
      !VOFP_IN((size_t)distinct_index(j, zt.bcy) * zt.Ux + distinct_index(i, zt.bcx), ts, CHK_Z_TABLE))
    return;
  const TT* F = reinterpret_cast<const TT*>(zt.tab) + (size_t)distinct_index(j, zt.bcy) * zt.Ux +
                distinct_index(i, zt.bcx);
  const T* za = reinterpret_cast<const T*>(zt.za);
  bool bad;
  if (a.singular && i == 0 && j == 0)
    bad = smem_d ? ztab_singular<T, TT>(a, col, dsm, TI, plane, F, ts)
                 : ztab_singular<T, TT>(a, col, col, plane, plane, F, ts);
  else if (smem_d)
    bad = ztab_sweep<T, TT, true>(col, dsm, plane, TI, F, ts, za, nz, (T)a.scale, a.info != nullptr);
  else
    bad = ztab_sweep<T, TT, false>(col, nullptr, plane, TI, F, ts, za, nz, (T)a.scale, a.info != nullptr);
  if (bad && a.info) atomicOr(&a.info->nonfinite, 1u);
}

template <typename T, typename TT>
static __global__ void __launch_bounds__(128) k_ztab(ZArgs a, ZTabArgs zt, int smem_d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ztab_block<T, TT>(a, zt, smem_d, blockIdx.x, blockIdx.y, smem_raw);
}

// Launch shape of k_ztab: threads (= systems) per block and whether the forward values fit in shared memory
// (at most 96 KB per block, so that two blocks share an SM).
struct ZTabShape {
  int threads;
  int smem_d;
  size_t smem;
};
inline ZTabShape ztab_shape(int ti, int nz, size_t elem) {
  ZTabShape s;
  s.threads = ti < 32 ? 32 : (ti > 128 ? 128 : ti);
  const size_t need = (size_t)s.threads * nz * elem;
  s.smem_d = need <= 96 * 1024;
  s.smem = s.smem_d ? need : 0;
  return s;
}

// ---- one system per warp: affine scans ---------------------------------------------------------------
// Both Thomas sweeps with plan-time factors are first-order affine recurrences, d_k = alpha_k d_{k-1} + beta_k
// with alpha_k = -a_k m_k, beta_k = m_k r_k, then x_k = -c'_k x_{k+1} + d_k.  Each lane composes the affine maps
// of a contiguous run of rows, an inclusive warp scan of the composed maps (five shuffle steps) gives every
// lane its incoming value, and the lane then re-applies its rows from it.  Used where a system's serial chain
// would dominate: the low-eigenvalue systems of refinement plans (FP64) and the pinned mean mode.
__device__ __forceinline__ double shfl_up_t(double v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down_t(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor_t(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ ff shfl_up_t(ff v, int o) {
  return ff(__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ ff shfl_down_t(ff v, int o) {
  return ff(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ ff shfl_xor_t(ff v, int o) {
  return ff(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

template <typename T>
__device__ __forceinline__ void affine_scan_up(T& A, T& B, int lane) {
  // inclusive scan over lanes 0..lane of maps x -> A x + B, later lanes applied after earlier ones
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T pa = shfl_up_t(A, o);
    const T pb = shfl_up_t(B, o);
    if (lane >= o) {
      B = fma_t(A, pb, B);
      A = A * pa;
    }
  }
}
template <typename T>
__device__ __forceinline__ void affine_scan_down(T& A, T& B, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T pa = shfl_down_t(A, o);
    const T pb = shfl_down_t(B, o);
    if (lane + o < 32) {
      B = fma_t(A, pb, B);
      A = A * pa;
    }
  }
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor_t(v, o);
  return v;
}

// Uniform view of a factor entry: plan tables hold ZF already; the low-mode tables hold (c'_k, m_k).
__device__ __forceinline__ ZF<double> fac_view(const double2& f, double za_k, double sc) {
  return {f.x, sc * f.y, -za_k * f.y};
}
template <typename T>
__device__ __forceinline__ ZF<T> fac_view(const ZF<T>& f, T, T) {
  return f;
}

// One bounded-z system by one warp, arithmetic in T.  col: the system's column in the spectrum (stride plane,
// storage TS); F: its factor pairs (c'_k, m_k) at stride fs; scr: nz forward values at stride ss.  sing: the
// pinned mean mode (defect removed, p_0 = 0, zero volume-weighted mean; its factors are the pinned system's).
template <typename T, typename TS, typename TT>
__device__ void zscan_system(const ZArgs& a, TS* col, size_t plane, const TT* F, size_t fs, T* scr, size_t ss,
                             const T* za, bool sing, int lane) {
  const int nz = a.nz;
  const T sc = (T)a.scale;
  const int R = (nz + 31) >> 5;
  const int k0 = lane * R < nz ? lane * R : nz;
  const int k1 = k0 + R < nz ? k0 + R : nz;
  T defect = (T)0;  // of the unscaled right-hand side
  if (sing) {
    T s = (T)0;
    for (int k = k0; k < k1; ++k) s += (T)__ldg(a.dz + k) * (T)col[k * plane];
    defect = warp_sum(s) / (T)a.lz;
    if (lane == 0 && a.info) a.info->compat_defect = (double)defect * a.scale;
  }
  const int kb = sing ? 1 : 0;  // first eliminated row (p_0 = 0 pinned in the singular mode)
  const int ks = k0 > kb ? k0 : kb;
  // forward: compose this lane's rows, scan, re-apply
  T A = (T)1, B = (T)0;
  for (int k = ks; k < k1; ++k) {
    const ZF<T> f = fac_view(F[k * fs], za[k], sc);
    const T al = k > kb ? f.al : (T)0;
    const T be = ((T)col[k * plane] - defect) * f.ms;
    B = fma_t(al, B, be);
    A = al * A;
  }
  affine_scan_up(A, B, lane);
  T d = shfl_up_t(B, 1);
  if (lane == 0) d = (T)0;
  for (int k = ks; k < k1; ++k) {
    const ZF<T> f = fac_view(F[k * fs], za[k], sc);
    const T al = k > kb ? f.al : (T)0;
    const T be = ((T)col[k * plane] - defect) * f.ms;
    d = fma_t(al, d, be);
    scr[k * ss] = d;
  }
  // backward: x_k = -c'_k x_{k+1} + d_k from the last row down
  A = (T)1;
  B = (T)0;
  for (int k = k1 - 1; k >= ks; --k) {
    const T g = -fac_view(F[k * fs], za[k], sc).c;
    B = fma_t(g, B, scr[k * ss]);
    A = g * A;
  }
  affine_scan_down(A, B, lane);
  T x = shfl_down_t(B, 1);
  if (lane == 31) x = (T)0;
  T msum = (T)0;
  for (int k = k1 - 1; k >= ks; --k) {
    const T g = -fac_view(F[k * fs], za[k], sc).c;
    x = fma_t(g, x, scr[k * ss]);
    scr[k * ss] = x;
    if (sing) msum += (T)__ldg(a.dz + k) * x;
  }
  T mean = (T)0;
  if (sing) mean = warp_sum(msum) / (T)a.lz;  // row 0 holds 0
  bool bad = false;
  for (int k = k0; k < k1; ++k) {
    const T v = (k < kb ? (T)0 : scr[k * ss]) - mean;
    col[k * plane] = (TS)v;
    if (a.info) bad |= !isfinite((double)v);
  }
  if (bad) atomicOr(&a.info->nonfinite, 1u);
}

// Refinement plans: the low-eigenvalue systems (listed at plan time) in FP64, one warp each; factors k-major
// (tab[k * nlow + t]), forward values in `scratch` ([nz][nlow]).
template <typename TS>
__device__ __forceinline__ void zlow_scan_system(const ZArgs& a, int2 md, int t, int nlow,
                                                 const double2* __restrict__ tab, double* __restrict__ scratch,
                                                 int lane) {
  TS* col = reinterpret_cast<TS*>(a.S) + (size_t)md.y * a.nx + md.x;
  if (!VOFP_IN((size_t)md.y * a.nx + md.x, (size_t)a.nx * a.ny, CHK_Z_COLUMN) || !VOFP_IN(md.x, a.nx, CHK_Z_COLUMN))
    return;  // (uniform per warp)
  zscan_system<double, TS, double2>(a, col, (size_t)a.nx * a.ny, tab + t, (size_t)nlow, scratch + t, (size_t)nlow,
                                    a.za, a.singular && md.x == 0 && md.y == 0, lane);
}

template <typename TS>
static __global__ void __launch_bounds__(128) k_zlow_scan(ZArgs a, const int2* __restrict__ modes, int nlow,
                                                          const double2* __restrict__ tab, double* scratch) {
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nlow) return;  // uniform per warp
  zlow_scan_system<TS>(a, modes[w], w, nlow, tab, scratch, threadIdx.x & 31);
}

// ---- small grids: systems staged in shared memory -----------------------------------------------------
// With few systems (nx * ny small) one thread per system leaves most of each SM idle, and an FP64 recurrence
// is then bound by its 64-cycle dependent latency.  This kernel stages a tile of 32 systems ([nz][32]) in
// shared memory with all 128 threads, computing alpha_k, beta_k (scaled) and c'_k on the way in; warp 0 runs
// the two one-multiply-add recurrences from shared memory; warp 1 solves the pinned mean mode (if it is in
// the tile) by affine scans; all threads store the tile.  Shared memory: nz * 32 * 3 values + nz scratch.
constexpr int kZStagedTI = 32;
template <typename T>
struct Pair {
  T x, y;
};
inline size_t ztab_staged_smem(int nz, size_t elem) { return (size_t)nz * (3 * kZStagedTI + 1) * elem; }
// Staged kernel for FP64 / FP32-pair arithmetic when the grid has fewer than 152 * 256 systems (too few to
// hide the recurrences' latency one thread each) and the tile fits in shared memory.
inline bool ztab_use_staged(int nx, int ny, int nz, size_t elem) {
  return (size_t)nx * ny < (size_t)152 * 256 && ztab_staged_smem(nz, elem) <= 200 * 1024;
}

template <typename T, typename TT>
static __global__ void __launch_bounds__(128) k_ztab_staged(ZArgs a, ZTabArgs zt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  constexpr int TI = kZStagedTI;
  const int nz = a.nz;
  const int i0 = blockIdx.x * TI, j = blockIdx.y;
  Pair<T>* ab = reinterpret_cast<Pair<T>*>(smem_raw);  // [nz][TI] (alpha_k, beta_k), then d_k / x_k in .y
  T* cp = reinterpret_cast<T*>(ab + (size_t)nz * TI);  // [nz][TI] c'_k
  T* scr = cp + (size_t)nz * TI;                        // [nz] pinned-mode scratch
  const size_t plane = (size_t)a.nx * a.ny;
  T* S = reinterpret_cast<T*>(a.S) + (size_t)j * a.nx + i0;
  const TT* F = reinterpret_cast<const TT*>(zt.tab) + (size_t)distinct_index(j, zt.bcy) * zt.Ux;
  const size_t ts = (size_t)zt.Ux * zt.Uy;
  const T* za = reinterpret_cast<const T*>(zt.za);
  const T sc = (T)a.scale;
  const int cut = zt.lowcut ? __ldg(zt.lowcut + j) : 0;
  const bool sing_here = a.singular && j == 0 && i0 == 0;  // the pinned mode is column 0 of this tile
  const int ncol = a.nx - i0 < TI ? a.nx - i0 : TI;
  if (!VOFP_IN(i0, a.nx, CHK_Z_COLUMN) || !VOFP_IN((size_t)j * a.nx + i0 + ncol - 1, plane, CHK_Z_COLUMN) ||
      !VOFP_IN((size_t)distinct_index(j, zt.bcy) * zt.Ux + distinct_index(i0 + ncol - 1, zt.bcx), ts, CHK_Z_TABLE))
    return;  // (uniform per block)
  // tile load: eight rows per thread in flight (all loads issued before any is used)
  constexpr int UL = 8;
  for (int t0 = threadIdx.x; t0 < nz * TI; t0 += UL * blockDim.x) {
    T rv[UL];
    TT fv[UL];
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int t = t0 + u * blockDim.x;
      const int k = t / TI, c = t - k * TI;
      if (t < nz * TI && c < ncol && i0 + c >= cut) {
        fv[u] = F[k * ts + distinct_index(i0 + c, zt.bcx)];
        rv[u] = S[k * plane + c];
      }
    }
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int t = t0 + u * blockDim.x;
      const int k = t / TI, c = t - k * TI;
      if (t < nz * TI && c < ncol && i0 + c >= cut) {
        Pair<T> v;
        v.x = fv[u].al;
        v.y = rv[u] * fv[u].ms;
        ab[t] = v;
        cp[t] = fv[u].c;
      }
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    const int c = lane, i = i0 + c;
    if (c < ncol && i >= cut && !(sing_here && c == 0)) {
      // the shared-memory operands of rows k + 1 .. k + 8 are read before row k is used (a register ring),
      // so each row costs one dependent multiply-add and no load latency
      constexpr int U = 8;
      Pair<T> rb[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (u < nz) rb[u] = ab[u * TI + c];
      T d = (T)0;
      for (int k0 = 0; k0 < nz; k0 += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + u;
          if (k < nz) {
            const Pair<T> v = rb[u];
            if (k + U < nz) rb[u] = ab[(k + U) * TI + c];
            d = fma_t(v.x, d, v.y);
            ab[k * TI + c].y = d;
          }
        }
      }
      T x = d;
      T db[U], cb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = nz - 2 - u;
        if (k >= 0) {
          db[u] = ab[k * TI + c].y;
          cb[u] = cp[k * TI + c];
        }
      }
      for (int k0 = nz - 2; k0 >= 0; k0 -= U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 - u;
          if (k >= 0) {
            const T dk = db[u], ck = cb[u];
            if (k - U >= 0) {
              db[u] = ab[(k - U) * TI + c].y;
              cb[u] = cp[(k - U) * TI + c];
            }
            x = fma_t(-ck, x, dk);
            ab[k * TI + c].y = x;
          }
        }
      }
    }
  } else if (warp == 1 && sing_here && cut == 0) {
    zscan_system<T, T, TT>(a, S, plane, F, ts, scr, 1, za, true, lane);
  }
  __syncthreads();
  bool bad = false;
  for (int t = threadIdx.x; t < nz * TI; t += blockDim.x) {
    const int k = t / TI, c = t - k * TI;
    const int i = i0 + c;
    if (c < ncol && i >= cut && !(sing_here && c == 0)) {
      const T x = ab[t].y;
      S[k * plane + c] = x;
      if (a.info) bad |= !isfinite((double)x);
    }
  }
  if (bad) atomicOr(&a.info->nonfinite, 1u);
}

// ---- segmented tiles: every warp on the recurrences ---------------------------------------------------
// The staged kernel leaves three of its four warps idle while warp 0 runs 32 recurrences of nz rows each, so
// a tile costs 2 nz dependent multiply-adds of latency.  Here a tile of 32 systems is cut into 8 row
// segments, one warp each, and every recurrence d_k = alpha_k d_{k-1} + beta_k (then x_k = g_k x_{k+1} + d_k,
// g_k = -c'_k) is an affine map composed in two levels: each warp composes its segment's rows into one map
// (A, B), each warp folds the maps of the segments before it (at most 7) into its carry-in, then re-runs its
// rows from that carry.  Latency per sweep: 2 nz / 8 + 7 steps instead of nz; work: about 2.5 multiply-adds
// per row and sweep instead of 1.  Used where the arithmetic is cheap: FP32 and FP32 pairs (FP64 keeps the
// staged and streaming kernels: its narrow FP64 pipe makes the extra multiply-adds cost more than the
// latency they hide).
//
// Two layouts of the tile in shared memory ([nz][32] each array):
//   full: alpha_k, beta_k and c'_k staged as the tile is loaded (three values per cell);
//   lean: beta_k only (overwritten by d_k, then x_k); alpha_k and c'_k are re-read from the factor table
//         (the tile's entries, some 100 KB at nz = 512, come from DRAM once and from L2 after).
// A kernel that holds the SM alone stops the SM's memory traffic during its recurrences, so the plan takes
// the full layout while two blocks still fit per SM (FP32 up to nz = 279, FP32 pairs up to 134), else the
// lean one (FP32 up to nz = 822, FP32 pairs up to 395; the z passes of a 512^3 FP32 + refinement solve, three
// working launches: 3.52 -> 2.46 ms, 2.14 ms with the loops below), else the streaming kernel.  The full layout is the faster one where both fit twice
// (128^3 FP32: 13.4 against 14.9 us).  The loops keep each lane on its column with strided pointers and let
// lanes without a system skip them: ncu had the lean kernel issue-bound at some 160 instructions per cell.
constexpr int kZSegTI = 32, kZSegW = 8;
inline size_t ztab_seg_smem(int nz, size_t elem, bool lean) {
  return ((size_t)nz * ((lean ? 1 : 3) * kZSegTI + 1) + (size_t)4 * kZSegW * kZSegTI) * elem;
}
// plan code of the segmented kernel for a reduced-precision plan: -1 full, -2 lean, 0 neither (two blocks per
// SM must fit: 110 KB each)
inline int ztab_seg_code(int nz, size_t elem) {
  if (ztab_seg_smem(nz, elem, false) <= 110 * 1024) return -1;
  if (ztab_seg_smem(nz, elem, true) <= 110 * 1024) return -2;
  return 0;
}

// Block body (kZSegW warps): tile bx of row by.
template <typename T, typename TT, bool LEAN>
__device__ __forceinline__ void ztab_seg_block(const ZArgs& a, const ZTabArgs& zt, int bx, int by,
                                               unsigned char* smem_raw) {
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  constexpr int TI = kZSegTI, W = kZSegW;
  const int nz = a.nz;
  const int i0 = bx * TI, j = by;
  T* yv = reinterpret_cast<T*>(smem_raw);            // [nz][TI] beta_k, then d_k, then x_k
  T* alv = yv + (LEAN ? 0 : (size_t)nz * TI);         // [nz][TI] alpha_k (full layout)
  T* cpv = alv + (LEAN ? 0 : (size_t)nz * TI);        // [nz][TI] c'_k (full layout)
  T* fA = (LEAN ? yv : cpv) + (size_t)nz * TI;        // [W][TI] segment maps: forward A, B, backward A, B
  T* fB = fA + W * TI;
  T* bA = fB + W * TI;
  T* bB = bA + W * TI;
  T* scr = bB + W * TI;  // [nz] pinned-mode scratch
  const size_t plane = (size_t)a.nx * a.ny;
  T* S = reinterpret_cast<T*>(a.S) + (size_t)j * a.nx + i0;
  const TT* F = reinterpret_cast<const TT*>(zt.tab) + (size_t)distinct_index(j, zt.bcy) * zt.Ux;
  const size_t ts = (size_t)zt.Ux * zt.Uy;
  const T* za = reinterpret_cast<const T*>(zt.za);
  const int cut = zt.lowcut ? __ldg(zt.lowcut + j) : 0;
  const bool sing_here = a.singular && j == 0 && i0 == 0;  // the pinned mode is column 0 of this tile
  const int ncol = a.nx - i0 < TI ? a.nx - i0 : TI;
  if (!VOFP_IN(i0, a.nx, CHK_Z_COLUMN) || !VOFP_IN((size_t)j * a.nx + i0 + ncol - 1, plane, CHK_Z_COLUMN) ||
      !VOFP_IN((size_t)distinct_index(j, zt.bcy) * zt.Ux + distinct_index(i0 + ncol - 1, zt.bcx), ts, CHK_Z_TABLE))
    return;  // (uniform per block)
  // Lane c of every warp works on column c of the tile (32 consecutive x indices: coalesced rows), warp w on rows
  // w, w + W, ... for the load and the store and on the segment [k0, k1) for the recurrences.  Lanes without a
  // system of their own (past the row's end, low modes, the pinned mode) skip the loads, the recurrences and the
  // stores; their segment maps are never read by a live lane.
  const int w = threadIdx.x >> 5, c = threadIdx.x & 31;
  const bool mine = c < ncol && i0 + c >= cut;           // column c is solved by this kernel...
  const bool live = mine && !(sing_here && c == 0);      // ... by the recurrences below (not the pinned mode)
  const TT* Fl = F + (mine ? distinct_index(i0 + c, zt.bcx) : 0);  // this column's factors (stride ts)
  T* yc = yv + c;                                         // this column of the tile (stride TI)
  // tile load: eight rows per thread in flight (four with the full layout's three values per row, which keeps
  // the registers at four blocks per SM); beta_k = m_k r_k (scaled)
  constexpr int UL = LEAN ? 8 : 4;
  if (mine) {
    const T* Sc = S + c;
    for (int kb = w; kb < nz; kb += UL * W) {
      T rv[UL];
      TT fv[UL];
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        const int k = kb + u * W;
        if (k < nz) {
          if (LEAN)
            fv[u].ms = Fl[(size_t)k * ts].ms;
          else
            fv[u] = Fl[(size_t)k * ts];
          rv[u] = Sc[(size_t)k * plane];
        }
      }
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        const int k = kb + u * W;
        if (k < nz) {
          yc[k * TI] = rv[u] * fv[u].ms;
          if (!LEAN) {
            alv[k * TI + c] = fv[u].al;
            cpv[k * TI + c] = fv[u].c;
          }
        }
      }
    }
  }
  __syncthreads();
  const int L = (nz + W - 1) / W;
  const int k0 = w * L < nz ? w * L : nz;
  const int k1 = k0 + L < nz ? k0 + L : nz;
  // unrolling of the recurrence loops: the lean FP32 layout reads alpha_k / c'_k from L2 in them (ncu: stalled
  // on those loads), and 16 rows of them in flight took the z passes of a 512^3 solve from 2.11 to 1.94 ms
  // (FP32 pairs, with twice the registers per value, measured no better)
  constexpr int UR = (LEAN && sizeof(T) == 4) ? 16 : 4;
  // factors of row k of this column: alpha_k and c'_k from the staged tile (full) or the table (lean)
  const T* ac = alv + c;
  const T* cc = cpv + c;
  {  // forward: this segment's rows as one map d_out = A d_in + B
    T A = (T)1, B = (T)0;
    if (live) {
      const TT* f = Fl + (size_t)k0 * ts;
#pragma unroll (UR)
      for (int k = k0; k < k1; ++k, f += ts) {
        const T al = LEAN ? f->al : ac[k * TI];
        B = fma_t(al, B, yc[k * TI]);
        A = al * A;
      }
    }
    fA[w * TI + c] = A;
    fB[w * TI + c] = B;
  }
  __syncthreads();
  if (live) {
    T d = (T)0;
    for (int sg = 0; sg < w; ++sg) d = fma_t(fA[sg * TI + c], d, fB[sg * TI + c]);
    const TT* f = Fl + (size_t)k0 * ts;
#pragma unroll (UR)
    for (int k = k0; k < k1; ++k, f += ts) {
      d = fma_t(LEAN ? f->al : ac[k * TI], d, yc[k * TI]);
      yc[k * TI] = d;
    }
  }
  __syncthreads();
  // backward: x_{nz-1} = d_{nz-1}, x_k = -c'_k x_{k+1} + d_k (the last row peeled off: it has no c'_k term)
  const int kt = k1 == nz ? nz - 2 : k1 - 1;  // first row of the segment with a c'_k term
  {
    T A = (T)1, B = (T)0;
    if (live) {
      if (k1 == nz && k0 < k1) {
        B = yc[(nz - 1) * TI];
        A = (T)0;
      }
      const TT* f = Fl + (size_t)kt * ts;
#pragma unroll (UR)
      for (int k = kt; k >= k0; --k, f -= ts) {
        const T g = -(LEAN ? f->c : cc[k * TI]);
        B = fma_t(g, B, yc[k * TI]);
        A = g * A;
      }
    }
    bA[w * TI + c] = A;
    bB[w * TI + c] = B;
  }
  __syncthreads();
  if (live) {
    T x = (T)0;
    for (int sg = W - 1; sg > w; --sg) x = fma_t(bA[sg * TI + c], x, bB[sg * TI + c]);
    if (k1 == nz && k0 < k1) x = yc[(nz - 1) * TI];  // (stored already: x_{nz-1} = d_{nz-1})
    const TT* f = Fl + (size_t)kt * ts;
#pragma unroll (UR)
    for (int k = kt; k >= k0; --k, f -= ts) {
      x = fma_t(-(LEAN ? f->c : cc[k * TI]), x, yc[k * TI]);
      yc[k * TI] = x;
    }
  }
  if (w == 0 && sing_here && cut == 0) zscan_system<T, T, TT>(a, S, plane, F, ts, scr, 1, za, true, c);
  __syncthreads();
  bool bad = false;
  if (live) {
    T* Sc = S + c;
    for (int k = w; k < nz; k += W) {
      const T x = yc[k * TI];
      Sc[(size_t)k * plane] = x;
      if (a.info) bad |= !isfinite((double)x);
    }
  }
  if (bad) atomicOr(&a.info->nonfinite, 1u);
}

template <typename T, typename TT, bool LEAN>
static __global__ void __launch_bounds__(256) k_ztab_seg(ZArgs a, ZTabArgs zt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ztab_seg_block<T, TT, LEAN>(a, zt, blockIdx.x, blockIdx.y, smem_raw);
}

}  // namespace vofp
