// z pass: for every (x, y) spectral pair (q, r) solve
//     a_k p_{k-1} + (b_k + lx_q + ly_r) p_k + c_k p_{k+1} = scale * S_k      (k = 0..nz-1)
// where scale = 1/(nx ny) undoes the unnormalised x and y transforms.  The rows carry the z boundary
// conditions (§3.2; §8 of the design notes: N folds, D subtracts, periodic wraps).  The singular mean mode
// (no D end anywhere, q = r = 0) first removes the volume-weighted mean of its right-hand side (the
// compatibility defect, reported), pins p_0 = 0, solves rows 1..nz-1 and finally shifts to zero
// volume-weighted mean.  A block stages `ti` neighbouring systems of one y index in shared memory so that
// global loads and stores are row-coalesced; one thread then runs each system's recurrence.
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
  double* S;
};

// Thomas elimination on column `c` of the [nz][ti] shared tiles, rows k0..k1 (inclusive), off-diagonals of
// the first and last row dropped.  On entry d holds the right-hand side, on exit the solution.
__device__ __forceinline__ void thomas_smem(double* d, double* cp, int ti, int c, int k0, int k1, double lam,
                                            const double* __restrict__ za, const double* __restrict__ zb,
                                            const double* __restrict__ zc, double diag0_add, double diag1_add) {
  double den = __ldg(zb + k0) + lam + diag0_add;
  double m = 1.0 / den;
  double cprev = (k0 < k1 ? __ldg(zc + k0) : 0.0) * m;
  double dprev = d[k0 * ti + c] * m;
  cp[k0 * ti + c] = cprev;
  d[k0 * ti + c] = dprev;
  for (int k = k0 + 1; k <= k1; ++k) {
    const double ak = __ldg(za + k);
    den = __ldg(zb + k) + lam + (k == k1 ? diag1_add : 0.0) - ak * cprev;
    m = 1.0 / den;
    cprev = (k < k1 ? __ldg(zc + k) : 0.0) * m;
    dprev = (d[k * ti + c] - ak * dprev) * m;
    cp[k * ti + c] = cprev;
    d[k * ti + c] = dprev;
  }
  double x = dprev;
  for (int k = k1 - 1; k >= k0; --k) {
    x = d[k * ti + c] - cp[k * ti + c] * x;
    d[k * ti + c] = x;
  }
}

__global__ void __launch_bounds__(128) k_zsolve64(ZArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TI = a.ti, nz = a.nz;
  double* d = reinterpret_cast<double*>(smem_raw);
  double* cp = d + (size_t)nz * TI;
  double* zv = cp + (size_t)nz * TI;  // periodic z only
  const int i0 = blockIdx.x * TI;
  const int jq = blockIdx.y;
  const size_t plane = (size_t)a.nx * a.ny;
  const size_t col0 = (size_t)jq * a.nx + i0;
  for (int t = threadIdx.x; t < nz * TI; t += blockDim.x) {
    const int k = t / TI, c = t - k * TI;
    d[t] = (i0 + c < a.nx) ? a.S[k * plane + col0 + c] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < TI && i0 + c < a.nx) {
    const int iq = i0 + c;
    const double lam = __ldg(a.lamx + iq) + __ldg(a.lamy + jq);
    for (int k = 0; k < nz; ++k) d[k * TI + c] *= a.scale;
    const bool per = a.bcz == VOFP_BC_P;
    if (a.singular && iq == 0 && jq == 0) {
      double s = 0;
      for (int k = 0; k < nz; ++k) s += __ldg(a.dz + k) * d[k * TI + c];
      const double defect = s / a.lz;
      for (int k = 0; k < nz; ++k) d[k * TI + c] -= defect;
      if (a.info) a.info->compat_defect = defect;
      d[c] = 0.0;
      if (nz > 1) thomas_smem(d, cp, TI, c, 1, nz - 1, 0.0, a.za, a.zb, a.zc, 0.0, 0.0);
      double mean = 0;
      for (int k = 0; k < nz; ++k) mean += __ldg(a.dz + k) * d[k * TI + c];
      mean /= a.lz;
      for (int k = 0; k < nz; ++k) d[k * TI + c] -= mean;
    } else if (!per) {
      thomas_smem(d, cp, TI, c, 0, nz - 1, lam, a.za, a.zb, a.zc, 0.0, 0.0);
    } else if (nz == 1) {
      d[c] = d[c] / lam;
    } else if (nz == 2) {
      const double m00 = __ldg(a.zb) + lam, m01 = __ldg(a.za) + __ldg(a.zc);
      const double m10 = __ldg(a.za + 1) + __ldg(a.zc + 1), m11 = __ldg(a.zb + 1) + lam;
      const double det = m00 * m11 - m01 * m10;
      const double r0 = d[c], r1 = d[TI + c];
      d[c] = (m11 * r0 - m01 * r1) / det;
      d[TI + c] = (m00 * r1 - m10 * r0) / det;
    } else {
      // cyclic: A = T + u v^T, u = (gamma, 0, .., beta), v = (1, 0, .., alpha / gamma)
      const double alpha = __ldg(a.za), beta = __ldg(a.zc + nz - 1);
      const double gamma = -(__ldg(a.zb) + lam);
      for (int k = 0; k < nz; ++k) zv[k * TI + c] = 0.0;
      zv[c] = gamma;
      zv[(nz - 1) * TI + c] = beta;
      // y: T y = rhs ; z: T z = u (same factorisation, so run both eliminations together)
      const double add0 = -gamma, add1 = -alpha * beta / gamma;
      double den = __ldg(a.zb) + lam + add0;
      double m = 1.0 / den;
      double cprev = __ldg(a.zc) * m;
      double dy = d[c] * m, dz2 = zv[c] * m;
      cp[c] = cprev;
      d[c] = dy;
      zv[c] = dz2;
      for (int k = 1; k < nz; ++k) {
        const double ak = __ldg(a.za + k);
        den = __ldg(a.zb + k) + lam + (k == nz - 1 ? add1 : 0.0) - ak * cprev;
        m = 1.0 / den;
        cprev = (k < nz - 1 ? __ldg(a.zc + k) : 0.0) * m;
        dy = (d[k * TI + c] - ak * dy) * m;
        dz2 = (zv[k * TI + c] - ak * dz2) * m;
        cp[k * TI + c] = cprev;
        d[k * TI + c] = dy;
        zv[k * TI + c] = dz2;
      }
      double xy = dy, xz = dz2;
      for (int k = nz - 2; k >= 0; --k) {
        xy = d[k * TI + c] - cp[k * TI + c] * xy;
        xz = zv[k * TI + c] - cp[k * TI + c] * xz;
        d[k * TI + c] = xy;
        zv[k * TI + c] = xz;
      }
      const double vy = d[c] + alpha / gamma * d[(nz - 1) * TI + c];
      const double vz = zv[c] + alpha / gamma * zv[(nz - 1) * TI + c];
      const double f = vy / (1.0 + vz);
      for (int k = 0; k < nz; ++k) d[k * TI + c] -= f * zv[k * TI + c];
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
    if (i0 + cc < a.nx) a.S[k * plane + col0 + cc] = d[t];
  }
}

}  // namespace vofp
