// Internal declarations of the vofp library: plan layout, launch descriptors and the shared-memory FFT
// engine used by every transform pass.
//
// Transform conventions (per axis of n cells; every forward/inverse pair multiplies by n):
//   periodic  : X[m] = sum_j x[j] e^{-2 pi i m j / n}, stored half-complex and interleaved:
//               r[0] = Re X[0], r[2m-1] = Re X[m], r[2m] = Im X[m] (1 <= m < n/2), r[n-1] = Re X[n/2] (n even);
//               eigenvalue of r[q]: -(4/h^2) sin^2(pi ((q+1)/2) / n).
//   NN        : DCT-II, X[m] = sum_j x[j] cos(pi m (j+1/2) / n); eigenvalue -(4/h^2) sin^2(pi m / (2n)).
//   DD        : DST-II, X[m] = sum_j x[j] sin(pi (m+1)(j+1/2) / n); eigenvalue -(4/h^2) sin^2(pi (m+1) / (2n)).
// Each is evaluated for two real lines at once through one complex FFT of length n (a + i b): DFT split by
// Hermitian symmetry; DCT-II via the even/odd reordering v[j/2] = x[j] (j even), v[n-1-(j-1)/2] = x[j]
// (j odd) followed by a quarter-wave twiddle; DST-II as the DCT-II of (-1)^j x[j] read in reverse order.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>
#include <stdint.h>

#include "checked.cuh"
#include "ffloat.cuh"
#include "vofp.h"

#define VOFP_MAX_STAGES 24
#define VOFP_CONV_SLOTS 32

namespace vofp {

// ---- small complex helpers ---------------------------------------------------------------------------

template <typename R>
struct Cplx;
template <>
struct Cplx<double> {
  typedef double2 T;
};
template <>
struct Cplx<float> {
  typedef float2 T;
};

template <typename C>
__device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) {
  C r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  return cmk<C>(a.x + b.x, a.y + b.y);
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  return cmk<C>(a.x - b.x, a.y - b.y);
}
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i
template <typename C>
__device__ __forceinline__ C cmi(C a) {
  return cmk<C>(a.y, -a.x);
}

// Sign flip by the sign bit (integer pipe; no FP64 multiply on a narrow FP64 unit).
__device__ __forceinline__ double neg_if(double x, bool f) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)f << 63));
}
__device__ __forceinline__ float neg_if(float x, bool f) {
  return __int_as_float(__float_as_int(x) ^ ((int)f << 31));
}
__device__ __forceinline__ ff neg_if(ff x, bool f) { return ff(neg_if(x.hi, f), neg_if(x.lo, f)); }

// ---- mixed-precision refinement: device-side convergence test ---------------------------------------
// Slots: conv[0] = ||f||^2, conv[1] = sum f V, conv[2] = sum |f| V,
//        conv[VOFP_CONV_RES + j] = ||r_j||^2, r_j = f - fbar - L p_j the residual after j corrections,
//        conv[VOFP_CONV_DEL + j] = ||delta_j||^2 (delta_0 = the initial FP32 solve, delta_j the j-th
//        correction), conv[VOFP_CONV_MEAN] = sum of delta dz over all of them (the gauge of p),
//        conv[VOFP_CONV_FINAL] = ||r||^2 of the returned p (reporting pass),
//        conv[VOFP_CONV_EST] = ||S(r)||^2, the reduced-precision solve of that residual (not applied): the
//        error left in p, reported as the error estimate.
// Correction m (m >= 1) is a residual pass R_m (r_{m-1} = f - fbar - L p_{m-1}, its squared norm into
// conv[VOFP_CONV_RES + m - 1]), a reduced-precision solve S_m and the inverse pass X_m (p_m = p_{m-1} +
// delta_m, ||delta_m||^2 into conv[VOFP_CONV_DEL + m]).  F_k ("done after correction k - 1"): the residual
// after it is small, ||r_{k-1}||^2 <= tol^2 ||f||^2, AND the error left after it is estimated small, from the
// correction itself: ||delta_{k-1}|| <= (tol/10) ||delta_0||, or -- the corrections contracting by rho =
// ||delta_{k-1}|| / ||delta_{k-2}|| <= 1/4 -- rho ||delta_{k-1}|| <= (tol/10) ||delta_0||.  (A residual test
// alone is blind to errors in the smoothest modes, whose residual is smaller by their eigenvalue.)  R_m is
// skipped when F_{m-1} holds, S_m and X_m when F_m holds, so the refinement stops right after the residual
// pass that shows convergence.
#define VOFP_CONV_RES 3
#define VOFP_CONV_DEL 16
#define VOFP_CONV_EST 29
#define VOFP_CONV_MEAN 30
#define VOFP_CONV_FINAL 31
#define VOFP_MAX_REFINE 12
__host__ __device__ __forceinline__ bool refine_err_ok(const double* c, int j, double tol2) {
  if (j < 1) return false;  // no estimate from the first solve alone
  const double d0 = c[VOFP_CONV_DEL], dj = c[VOFP_CONV_DEL + j], dp = c[VOFP_CONV_DEL + j - 1];
  if (dj <= 0.01 * tol2 * d0) return true;
  return dj <= 0.0625 * dp && dj * dj <= 0.01 * tol2 * d0 * dp;
}
__host__ __device__ __forceinline__ bool refine_done(const double* c, int k, double tol2) {
  if (k < 1) return false;
  return c[VOFP_CONV_RES + k - 1] <= tol2 * c[0] && refine_err_ok(c, k - 1, tol2);
}
// j <= -2: always skipped (a correction beyond an instance's own limit in a batch); j <= 0: never; j >= 1:
// skipped when F_j holds.  Every block reads the same values.
__device__ __forceinline__ bool launch_skipped(const double* conv, int j, double tol2) {
  if (j <= -2) return true;
  if (!conv || j <= 0) return false;
  return refine_done(conv, j, tol2);
}

// Most line pairs per block of an x pass (the plan's default takes at most 16, the tuner at most 32).
constexpr int kMaxPB = 32;

// ---- FFT descriptor ----------------------------------------------------------------------------------

struct FftDesc {
  int n;
  int nst;
  int radix[VOFP_MAX_STAGES];
  // Bluestein (chirp-z) form, used when n has a prime factor above 13 and the plan supplies its tables: the
  // length-n DFT as a cyclic convolution of length bm (the least c * 2^k >= 2n - 1, c in {1, 3, 5, 15}) done
  // with bm-point FFTs.
  int bm;  // 0: n's own stages only
  int bst;
  int bradix[VOFP_MAX_STAGES];
};

// Points per shared-memory line of a transform: n, or bm when the Bluestein form runs (tables present).
__host__ __device__ __forceinline__ int fft_span(const FftDesc& fd, const void* blu) {
  return (blu && fd.bm) ? fd.bm : fd.n;
}

// Per-axis tables on the device.
struct AxisDev {
  int n;
  int bc;
  FftDesc fd;
  const double2* tw64;    // e^{-2 pi i k / n}, k < n
  const double2* quart64; // e^{-i pi k / (2 n)}, k < n
  const float2* tw32;
  const float2* quart32;
  const cff* twff;     // float-float twiddles (FP32-pair precision)
  const cff* quartff;
  const double2* blu64;  // Bluestein tables (see fft_smem), NULL when n needs none
  const float2* blu32;
  const cff* bluff;
  const double* lam; // eigenvalue of packed spectral index q, q < n
};

// Host-side factorisation of n into radices (8, 4, then 2, 3, 5, then 7, 11, 13 and any remaining prime).
void factor_radices(int n, FftDesc* fd);

// ---- shared-memory Stockham FFT ----------------------------------------------------------------------
// Batched forward complex DFT (exponent -2 pi i / n) of `batch` sequences of length n held in shared memory
// buffer `a` with line stride `ld` >= n; `b` is a second buffer of the same size.  Returns the buffer that holds the
// result.  All threads of the block must call it; it ends with __syncthreads().

template <typename C, int RAD>
__device__ __forceinline__ void dft_small(C* v) {
  typedef decltype(C::x) R;
  if (RAD == 2) {
    C t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  } else if (RAD == 3) {
    const R h = (R)0.86602540378443864676;  // sin(2 pi / 3)
    C s = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C m = cmk<C>(v[0].x - (R)0.5 * s.x, v[0].y - (R)0.5 * s.y);
    C r = cmk<C>(h * d.y, -h * d.x);  // -i h d
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  } else if (RAD == 4) {
    C a0 = cadd(v[0], v[2]);
    C a1 = csub(v[0], v[2]);
    C b0 = cadd(v[1], v[3]);
    C b1 = cmi(csub(v[1], v[3]));
    v[0] = cadd(a0, b0);
    v[2] = csub(a0, b0);
    v[1] = cadd(a1, b1);
    v[3] = csub(a1, b1);
  } else if (RAD == 5) {
    const R c1 = (R)0.30901699437494742410;   // cos(2 pi / 5)
    const R c2 = (R)-0.80901699437494742410;  // cos(4 pi / 5)
    const R s1 = (R)0.95105651629515357212;   // sin(2 pi / 5)
    const R s2 = (R)0.58778525229247312917;   // sin(4 pi / 5)
    C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    C m1 = cmk<C>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    C m2 = cmk<C>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    C t1 = cmk<C>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
    C t2 = cmk<C>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
    v[0] = cmk<C>(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
    v[1] = cadd(m1, cmi(t1));
    v[4] = csub(m1, cmi(t1));
    v[2] = cadd(m2, cmi(t2));
    v[3] = csub(m2, cmi(t2));
  } else if (RAD == 8) {
    const R r2 = (R)0.70710678118654752440;
    // two radix-4 transforms on even and odd samples
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<C, 4>(e);
    dft_small<C, 4>(o);
    // twiddles W8^k, k = 1..3 with W8 = e^{-i pi / 4}
    C o1 = cmk<C>(r2 * (o[1].x + o[1].y), r2 * (o[1].y - o[1].x));
    C o2 = cmi(o[2]);
    C o3 = cmk<C>(r2 * (o[3].y - o[3].x), -r2 * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
}

template <typename C, int RAD>
__device__ __forceinline__ void fft_stage(const C* __restrict__ src, C* __restrict__ dst, int batch, int n, int Ns,
                                          const C* __restrict__ tw, int ld) {
  const int NR = n / RAD;
  const int twstep = n / (Ns * RAD);
  const int total = batch * NR;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = t / NR;
    const int j = t - bi * NR;
    const C* s = src + bi * ld;
    C* d = dst + bi * ld;
    const int k = j % Ns;
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = s[j + r * NR];
    if (k != 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[r * k * twstep]);
    }
    dft_small<C, RAD>(v);
    const int base = (j - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) d[base + r * Ns] = v[r];
  }
}

// Stage of an odd prime radix R >= 7 (a runtime value; no hand-written butterfly).  The twiddles are applied in
// place first (src is scratch once a stage has run), then every butterfly is split into H + 1 work items
// (H = (R - 1) / 2): item 0 sums the inputs, item m >= 1 forms the output pair (m, R - m) from the input pairs
// a_r = v_r + v_{R-r}, b_r = v_r - v_{R-r} (r = 1..H) as X_m = v_0 + sum_r a_r cos(2 pi r m / R)
// - i sum_r b_r sin(2 pi r m / R), X_{R-m} the same with +i.  That is H complex-by-real multiply-add pairs
// per output pair, without per-output twiddles, and the loops stay rolled (few registers: the kernels that
// hold every stage keep their register count).  cos and sin of 2 pi q / R come from the n-point twiddle
// table, entry q n / R.
template <typename C>
__device__ __forceinline__ void fft_stage_odd(C* __restrict__ src, C* __restrict__ dst, int batch, int n, int Ns,
                                              int RAD, const C* __restrict__ tw, int ld) {
  typedef decltype(C::x) R;
  const int NR = n / RAD;
  const int H = (RAD - 1) / 2;
  if (Ns > 1) {
    const int twstep = n / (Ns * RAD);
#pragma unroll 1
    for (int t = threadIdx.x; t < batch * n; t += blockDim.x) {
      const int bi = t / n;
      const int e = t - bi * n;  // e = j + r NR
      const int r = e / NR;
      const int k = (e - r * NR) % Ns;
      if (r != 0 && k != 0) {
        C* p = src + bi * ld + e;
        *p = cmul(*p, tw[r * k * twstep]);
      }
    }
    __syncthreads();
  }
  const int per = NR * (H + 1);
#pragma unroll 1
  for (int t = threadIdx.x; t < batch * per; t += blockDim.x) {
    const int bi = t / per;
    const int rem = t - bi * per;
    const int m = rem / NR;  // item-major: a warp shares m and reads consecutive j
    const int j = rem - m * NR;
    const int k = j % Ns;
    const C* s = src + bi * ld;
    C* d = dst + bi * ld + (j - k) * RAD + k;
    const C v0 = s[j];
    if (m == 0) {
      C x = v0;
#pragma unroll 1
      for (int r = 1; r < RAD; ++r) x = cadd(x, s[j + r * NR]);
      d[0] = x;
      continue;
    }
    R ax = v0.x, ay = v0.y, bx = (R)0, by = (R)0;
    int q = m;  // r m mod R
#pragma unroll 1
    for (int r = 1; r <= H; ++r) {
      const C lo = s[j + r * NR], hi = s[j + (RAD - r) * NR];
      const bool up = q > H;  // past half a turn: cos(2 pi q / R) = cos(2 pi (R - q) / R), sin flips sign
      const C w = tw[(up ? RAD - q : q) * NR];  // e^{-2 pi i q' / R} = cos - i sin
      const R c = w.x, sq = up ? w.y : -w.y;
      ax += (lo.x + hi.x) * c;
      ay += (lo.y + hi.y) * c;
      bx += (lo.x - hi.x) * sq;
      by += (lo.y - hi.y) * sq;
      q += m;
      if (q >= RAD) q -= RAD;
    }
    d[m * Ns] = cmk<C>(ax + by, ay - bx);
    d[(RAD - m) * Ns] = cmk<C>(ax - by, ay + bx);
  }
}

// The same stage for a power-of-two n: every index is a shift or a mask of the thread's item number (no
// integer division by a runtime length, which costs the reduced-precision passes more issue slots than their
// butterflies).
template <typename C, int RAD>
__device__ __forceinline__ void fft_stage_p2(const C* __restrict__ src, C* __restrict__ dst, int batch, int lgn,
                                             int lgNs, const C* __restrict__ tw, int ld) {
  constexpr int lgR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
  const int lgNR = lgn - lgR;
  const int mNR = (1 << lgNR) - 1;
  const int mNs = (1 << lgNs) - 1;
  const int lgtw = lgn - lgNs - lgR;  // twiddle step n / (Ns RAD)
  const int total = batch << lgNR;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = t >> lgNR;
    const int j = t & mNR;
    const C* s = src + bi * ld;
    C* d = dst + bi * ld;
    const int k = j & mNs;
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = s[j + (r << lgNR)];
    if (k != 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[(r * k) << lgtw]);
    }
    dft_small<C, RAD>(v);
    const int base = ((j - k) << lgR) + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) d[base + (r << lgNs)] = v[r];
  }
}

template <typename C>
__device__ C* fft_stages(C* a, C* b, int batch, int n, int nst, const int* radix, const C* __restrict__ tw, int ld) {
  if constexpr (!std::is_same<C, double2>::value) {
    if ((n & (n - 1)) == 0) {  // radices 8, 4, 2 only: the shift-and-mask stages
      const int lgn = 31 - __clz(n);
      int lgNs = 0;
      for (int s = 0; s < nst; ++s) {
        const int R = radix[s];
        if (R == 8) fft_stage_p2<C, 8>(a, b, batch, lgn, lgNs, tw, ld);
        else if (R == 4) fft_stage_p2<C, 4>(a, b, batch, lgn, lgNs, tw, ld);
        else fft_stage_p2<C, 2>(a, b, batch, lgn, lgNs, tw, ld);
        __syncthreads();
        C* t = a;
        a = b;
        b = t;
        lgNs += R == 8 ? 3 : (R == 4 ? 2 : 1);
      }
      return a;
    }
  }
  int Ns = 1;
  for (int s = 0; s < nst; ++s) {
    const int R = radix[s];
    switch (R) {
      case 2: fft_stage<C, 2>(a, b, batch, n, Ns, tw, ld); break;
      case 3: fft_stage<C, 3>(a, b, batch, n, Ns, tw, ld); break;
      case 4: fft_stage<C, 4>(a, b, batch, n, Ns, tw, ld); break;
      case 5: fft_stage<C, 5>(a, b, batch, n, Ns, tw, ld); break;
      case 8: fft_stage<C, 8>(a, b, batch, n, Ns, tw, ld); break;
      default: fft_stage_odd<C>(a, b, batch, n, Ns, R, tw, ld); break;  // an odd prime >= 7
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// Complex conjugate.
template <typename C>
__device__ __forceinline__ C cconj(C a) {
  return cmk<C>(a.x, -a.y);
}

// `blu`: the plan's Bluestein tables for this axis in the precision of C -- chirp w_j = e^{-i pi j^2 / n}
// (n entries), then Bh = FFT_bm(h) / bm with h_m = conj(w_|m|) placed cyclically (bm entries), then the
// bm-point twiddles (bm entries) -- or NULL.  With them, X_k = w_k * y_k, y = the cyclic convolution of
// (x_j w_j) with h, computed as conj(FFT(conj(FFT(x w) * Bh))).  Lines need a stride ld >= bm then.
// FP64 transforms read their twiddles from a shared-memory copy of the table of the stages that run (the
// n-point table, or the bm-point one of a Bluestein length; up to kTwSmem points): the scattered
// per-butterfly twiddle loads then go to shared memory instead of queueing on the texture/L1 path, the top
// stall of these FP64-pipe-bound passes (measured 6-10% faster per pass at 128^3).
// The reduced-precision passes keep the table in global memory (no gain there, and the copy's registers cost
// the FP32-pair x pass a block per SM).
constexpr int kTwSmem = 1024;
// The Bluestein convolution of fft_smem with the bm-point twiddles twM.
template <typename C>
__device__ __forceinline__ C* blu_conv(C* a, C* b, int batch, const FftDesc& fd, const C* __restrict__ blu,
                                       const C* __restrict__ twM, int ld) {
  const int n = fd.n, M = fd.bm;
  const C* __restrict__ w = blu;
  const C* __restrict__ Bh = blu + n;
  for (int t = threadIdx.x; t < batch * M; t += blockDim.x) {
    const int bi = t / M, j = t - bi * M;
    C* p = a + bi * ld + j;
    *p = j < n ? cmul(*p, w[j]) : cmk<C>((decltype(C::x))0, (decltype(C::x))0);
  }
  __syncthreads();
  C* r = fft_stages(a, b, batch, M, fd.bst, fd.bradix, twM, ld);
  C* o = r == a ? b : a;
  for (int t = threadIdx.x; t < batch * M; t += blockDim.x) {
    const int bi = t / M, j = t - bi * M;
    C* p = r + bi * ld + j;
    *p = cconj(cmul(*p, Bh[j]));
  }
  __syncthreads();
  C* r2 = fft_stages(r, o, batch, M, fd.bst, fd.bradix, twM, ld);
  for (int t = threadIdx.x; t < batch * n; t += blockDim.x) {
    const int bi = t / n, k = t - bi * n;
    C* p = r2 + bi * ld + k;
    *p = cmul(cconj(*p), w[k]);
  }
  __syncthreads();
  return r2;
}

template <typename C>
__device__ C* fft_smem(C* a, C* b, int batch, const FftDesc& fd, const C* __restrict__ tw, int ld,
                       const C* __restrict__ blu) {
  const bool bl = blu && fd.bm != 0;
  if constexpr (std::is_same<C, double2>::value) {
    const int m = bl ? fd.bm : fd.n;
    if (m <= kTwSmem) {
      // the shared copy is passed on as a shared-memory pointer in both branches (a pointer that may be
      // either would compile to generic loads, which queue on the same path as global ones)
      __shared__ C tws[kTwSmem];
      const C* src = bl ? blu + fd.n + fd.bm : tw;
      for (int t = threadIdx.x; t < m; t += blockDim.x) tws[t] = src[t];
      __syncthreads();
      if (bl) return blu_conv(a, b, batch, fd, blu, (const C*)tws, ld);
      return fft_stages(a, b, batch, fd.n, fd.nst, fd.radix, (const C*)tws, ld);
    }
  }
  // (the reduced-precision types keep this code shape: their register allocation is sensitive to it)
  if (!bl) return fft_stages(a, b, batch, fd.n, fd.nst, fd.radix, tw, ld);
  const int n = fd.n, M = fd.bm;
  const C* __restrict__ w = blu;
  const C* __restrict__ Bh = blu + n;
  const C* __restrict__ twM = blu + n + M;
  for (int t = threadIdx.x; t < batch * M; t += blockDim.x) {
    const int bi = t / M, j = t - bi * M;
    C* p = a + bi * ld + j;
    *p = j < n ? cmul(*p, w[j]) : cmk<C>((decltype(C::x))0, (decltype(C::x))0);
  }
  __syncthreads();
  C* r = fft_stages(a, b, batch, M, fd.bst, fd.bradix, twM, ld);
  C* o = r == a ? b : a;
  for (int t = threadIdx.x; t < batch * M; t += blockDim.x) {
    const int bi = t / M, j = t - bi * M;
    C* p = r + bi * ld + j;
    *p = cconj(cmul(*p, Bh[j]));
  }
  __syncthreads();
  C* r2 = fft_stages(r, o, batch, M, fd.bst, fd.bradix, twM, ld);
  for (int t = threadIdx.x; t < batch * n; t += blockDim.x) {
    const int bi = t / n, k = t - bi * n;
    C* p = r2 + bi * ld + k;
    *p = cmul(cconj(*p), w[k]);
  }
  __syncthreads();
  return r2;
}

// ---- pre/post-processing of the real-to-real transforms ----------------------------------------------

// Shared-memory line stride of the column (y) passes: odd, so that the lines a warp touches at one sample
// index fall in different banks.
__host__ __device__ __forceinline__ int y_ld(int n) { return n | 1; }

// Position of sample j in the reordered sequence used by DCT-II / DST-II (and DCT-IV / DST-IV).
__device__ __forceinline__ int dct_perm(int j, int n) { return (j & 1) ? (n - 1 - (j >> 1)) : (j >> 1); }

// ND / DN on a transformed axis: the quarter-wave transforms DCT-IV / DST-IV, X[m] = sum_j x[j] cos (resp.
// sin) (pi (2m+1)(2j+1) / (4n)).  With the DCT-II reordering and the odd samples negated (v), X[m] =
// Re(e^{-i pi (2m+1)/(4n)} W[m]), W the length-n DFT of v_k e^{-i pi k/n}; for real v, W[n-1-m] =
// conj(W[m]), so two packed lines split about n-1.  DST-IV is the DCT-IV of the reversed line with signs
// (-1)^m.  Both are their own inverses up to n/2.  The axis' quart table then holds the pre-twiddles
// e^{-i pi k/n} (k < n) followed by the post-twiddles e^{-i pi (2m+1)/(4n)}.
__host__ __device__ __forceinline__ bool quarter_bc(int bc) { return bc == VOFP_BC_ND || bc == VOFP_BC_DN; }

// Place sample i of two packed lines (a, b) for a quarter-wave transform: position, value (pre-twiddled).
template <typename C>
__device__ __forceinline__ void quarter_load(int i, int n, int bc, decltype(C::x) a, decltype(C::x) b,
                                             const C* __restrict__ quart, int& pos, C& v) {
  const int s = bc == VOFP_BC_ND ? i : n - 1 - i;
  pos = dct_perm(s, n);
  const bool neg = s & 1;
  v = cmul(cmk<C>(neg_if(a, neg), neg_if(b, neg)), quart[pos]);
}

// Split the FFT Z of (a + i b) at index m into the spectra of a and b: A = (Z[m] + conj Z[n-m]) / 2,
// B = (Z[m] - conj Z[n-m]) / (2 i).
template <typename C>
__device__ __forceinline__ void split_two(const C* Z, int n, int m, C& A, C& B) {
  typedef decltype(C::x) R;
  const C P = Z[m];
  const C Q = Z[m == 0 ? 0 : n - m];
  A = cmk<C>((R)0.5 * (P.x + Q.x), (R)0.5 * (P.y - Q.y));
  B = cmk<C>((R)0.5 * (P.y + Q.y), (R)-0.5 * (P.x - Q.x));
}

// Forward post-processing: spectral output q of both lines from the FFT result Z, returned TWICE the
// transform (2A, 2B of split_two without the halving; the z pass folds the factor into its scale).
// `es`: element stride of the line in Z (1: contiguous; the TMA y pass keeps its lines element-major).
template <typename C>
__device__ __forceinline__ void fwd_post(const C* Z, int n, int bc, int q, const C* __restrict__ quart,
                                         decltype(C::x)& oa, decltype(C::x)& ob, int es = 1) {
  if (quarter_bc(bc)) {
    // 2 W_a = Z[q] + conj Z[n-1-q], 2 W_b = (Z[q] - conj Z[n-1-q]) / i; outputs Re(w 2W) with the post-twiddle
    const C P = Z[q * es];
    const C Q = Z[(n - 1 - q) * es];
    const C w = quart[n + q];
    oa = w.x * (P.x + Q.x) - w.y * (P.y - Q.y);
    ob = w.x * (P.y + Q.y) - w.y * (Q.x - P.x);
    if (bc == VOFP_BC_DN && (q & 1)) {
      oa = -oa;
      ob = -ob;
    }
  } else if (bc == VOFP_BC_P) {
    const int m = (q + 1) >> 1;
    const C P = Z[m * es];
    const C Q = Z[(m == 0 ? 0 : n - m) * es];
    if ((q == 0) || (q & 1)) {  // real parts
      oa = P.x + Q.x;
      ob = P.y + Q.y;
    } else {  // imaginary parts
      oa = P.y - Q.y;
      ob = Q.x - P.x;
    }
  } else {
    const int m = (bc == VOFP_BC_DD) ? (n - 1 - q) : q;
    const C P = Z[m * es];
    const C Q = Z[(m == 0 ? 0 : n - m) * es];
    const C w = quart[m];
    // Re(w * 2A) and Re(w * 2B)
    oa = w.x * (P.x + Q.x) - w.y * (P.y - Q.y);
    ob = w.x * (P.y + Q.y) - w.y * (Q.x - P.x);
  }
}

// Half-complex unpacking: spectrum value X[m] (0 <= m < n) of a packed periodic line r.
template <typename C, typename LOAD>
__device__ __forceinline__ C unpack_hc(LOAD r, int n, int m) {
  typedef decltype(C::x) R;
  if (m == 0) return cmk<C>(r(0), (R)0);
  const bool conj = 2 * m > n;
  const int mm = conj ? n - m : m;
  if (2 * mm == n) return cmk<C>(r(n - 1), (R)0);
  C v = cmk<C>(r(2 * mm - 1), r(2 * mm));
  if (conj) v.y = -v.y;
  return v;
}

// Inverse pre-processing: complex input (already conjugated for the forward engine) at FFT index m for
// two packed spectral lines ra, rb.  After the forward FFT of this input, Y = conj(n (a + i b)) at the
// reordered positions.
template <typename C, typename LA, typename LB>
__device__ __forceinline__ C inv_pre(LA ra, LB rb, int n, int bc, int m, const C* __restrict__ quart) {
  typedef decltype(C::x) R;
  C Z;
  if (bc == VOFP_BC_P) {
    const C A = unpack_hc<C>(ra, n, m);
    const C B = unpack_hc<C>(rb, n, m);
    Z = cmk<C>(A.x - B.y, A.y + B.x);
  } else {
    // V[m] = e^{+i pi m / (2n)} (X[m] - i X[n-m]), X[n] = 0; DD reads X in reverse order
    R xa, xb, ya = 0, yb = 0;
    if (bc == VOFP_BC_DD) {
      xa = ra(n - 1 - m);
      xb = rb(n - 1 - m);
      if (m > 0) {
        ya = ra(m - 1);
        yb = rb(m - 1);
      }
    } else {
      xa = ra(m);
      xb = rb(m);
      if (m > 0) {
        ya = ra(n - m);
        yb = rb(n - m);
      }
    }
    const C w = quart[m];  // (c, -s)
    const R c = w.x, s = -w.y;
    const C Va = cmk<C>(c * xa + s * ya, s * xa - c * ya);
    const C Vb = cmk<C>(c * xb + s * yb, s * xb - c * yb);
    Z = cmk<C>(Va.x - Vb.y, Va.y + Vb.x);
  }
  return cmk<C>(Z.x, -Z.y);
}

}  // namespace vofp

// ---- plan ---------------------------------------------------------------------------------------------

struct vofp_devinfo {
  double compat_defect;
  double abs_sum;  // sum |f| V over the grid (for the incompatibility warning)
  double res2;     // mixed: ||f - L p||^2
  double f2;       // mixed: ||f||^2
  unsigned int nonfinite;
  unsigned int timeout;  // a bounded device wait (TMA tile load) gave up
};

struct vofp_plan {
  int n[3];
  int bc[3];
  double dx, dy;
  double* dz_host;
  vofp_opts opts;
  int device;
  int singular;
  double volume;  // total volume
  vofp::AxisDev ax[2];
  // z tables
  double* za;  // coefficient of p_{k-1} in row k (wraps for periodic z)
  double* zb;  // diagonal
  double* zc;  // coefficient of p_{k+1}
  double* dz;  // widths
  double* hz;  // centre distance across face k (k = 0..nz; ghost distances at the ends)
  double* rdz;   // 1/dz
  double* rhz;   // 1/hz
  double* rzc;   // 1/(hz[k] + hz[k+1])
  double* kz;    // per plane k: cell volume, then the residual stencil's z coefficients czp, czm, czc
                 // (4 arrays of nz)
  float* volf;   // cell volume per plane, FP32
  vofp::ff* dzff;  // dz per plane, FP32 pair
  double* conv;  // mixed path: FP64 reduction slots (norms, means) per solve
  double* G;     // interface geometry: s, n_x, n_y, n_z (4 * cells)
  void* hstep;   // device fields, streams and events of the host-buffer step (allocated on first use)
  void* ztab;    // bounded z: Thomas factors per distinct eigenvalue pair in the plan's arithmetic type
                 // (double2, float2 or cff; NULL: periodic z)
  const void* zaT;     // z sub-diagonal a_k in the same type
  int* lowcut;         // refinement plans: spectral x index i of row j is a low mode iff i < lowcut[j]
  int Ux, Uy;    // distinct eigenvalue counts in x, y
  // mixed path
  double lowthr;       // |lx + ly| at or below which a z system is solved in FP64
  int nlow;            // number of such systems
  int2* lowmodes;      // their (x, y) spectral indices
  double* lowscratch;  // FP64 columns for them (3 nz each)
  double2* lowtab;     // bounded z: their Thomas factors (k-major), NULL for periodic z
  void* low_block;     // allocation holding lowmodes and lowscratch
  int ytx32, zti32;    // launch shapes of the FP32 y and z passes
  int radix_order;     // bit a set: the FFT stages of axis a (0 = x, 1 = y) run in reverse order (autotuned)
  // TMA-staged y pass of the reduced-precision spectra (set up on first use): state 0 = not yet examined,
  // 1 = in use, -1 = not applicable (or switched off by VOFP_Y_TMA=0); its tile width, persistent grid and the
  // encoded tensor map (a CUtensorMap, kept as bytes)
  int ytma_state, ytma_lgB, ytma_grid;
  unsigned char ytma_map[128];
  // the same for the TMA-staged inverse x pass (power-of-two nx of 128, 256 or 512)
  int xtma_state, xtma_grid;
  unsigned char xtma_map[128];
  // tensor-core x passes of FP32 refinement plans: the forward and inverse x transform matrices (TF32 hi / lo,
  // MMA operand layout) in the plan's memory, NULL when not used; persistent grid (0 = not yet sized)
  float* xtc_fwd;
  float* xtc_inv;
  int xtc_grid;
  // workspace
  double* S;   // spectrum, nx*ny*nz (FP64 path)
  double* P;   // potential scratch when the caller passes none
  float* S32;  // spectrum (mixed path)
  double* F;   // mixed: right-hand side kept in FP64
  double* R;   // mixed: residual
  vofp_devinfo* info;
  void* table_block;  // one allocation for all tables
  size_t bytes;
  // launch shapes
  int xpb;  // line pairs per block, x pass
  int ytx;  // columns per block, y pass
  int zti;  // systems per block, z pass (table kernel: threads per block)
};
