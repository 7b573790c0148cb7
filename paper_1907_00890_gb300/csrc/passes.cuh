// Transform and tridiagonal passes of the direct Poisson solve (device code, templated on precision).
//
//   x pass (forward) : right-hand side (given, divergence stencil, Stefan source or FP64 residual) fused with
//                      the real-to-real x transform of two grid lines per complex FFT;
//   y pass           : the same transform along y on column tiles of one z plane;
//   z pass           : one tridiagonal system per (x, y) spectral pair (Thomas; Sherman-Morrison around it
//                      for periodic z; gauge-fixed solve of the singular mean mode);
//   y pass (inverse), x pass (inverse) : back to cell values.
// The spectrum S is stored [z][y][x] like the fields, one real number per cell.
#pragma once

#include <type_traits>

#include "stencil.cuh"
#include "vofp_internal.cuh"

namespace vofp {

enum RhsMode { RHS_F = 0, RHS_DIV = 1, RHS_STEFAN = 2, RHS_RESID = 3, RHS_DIV_STEFAN = 4 };

struct XArgs {
  GridDev g;
  FftDesc fd;
  const void* tw;     // complex twiddles of the compute precision
  const void* quart;
  const void* blu;  // Bluestein tables of the x axis (NULL: direct stages)  // quarter-wave twiddles
  int pb;             // line pairs per block
  // right-hand side inputs
  const double* f;    // RHS_F: f;  RHS_RESID: f (FP64)
  const double* u;
  const double* v;
  const double* w;
  const double* src;  // RHS_DIV: optional source
  const double* C;
  const double* mdot;
  const double* p;    // RHS_RESID: current potential
  double scale;       // multiplies the right-hand side (RHS_F, RHS_DIV)
  double coef;        // RHS_STEFAN: 1/rho2 - 1/rho1
  int grad_mode;
  double* fsave;      // if non-null, the FP64 right-hand side is stored here (mixed path)
  vofp_devinfo* info; // if non-null, accumulate sum |f| V into info->abs_sum
  double* sq_out;     // if non-null, accumulate sum f^2 here
  double* fv_out;     // if non-null, accumulate sum f V here
  double* abs_out;    // if non-null, accumulate sum |f| V here
  const double* skip_conv;  // mixed refinement: skip when conv[3 + skip_k] <= tol2 conv[0]
  int skip_k;
  double tol2;
  const double* defect_sum; // RHS_RESID on a singular operator: subtract (*defect_sum) * inv_volume
  double inv_volume;
  void* S;            // spectrum output
};

// base - L p at a cell, L the 7-point operator with the ghost rules of the MAC grid, as a weighted sum of the
// neighbours with per-plane coefficients (rdx2, rdy2, czp, czm, and czc for the centre) subtracted from `base`
// in one multiply-add chain: two additions and five multiply-adds in FP64.
__device__ __forceinline__ double resid_at(const GridDev& g, const double* __restrict__ p, int i, int j, int k,
                                           double base) {
  const size_t plane = (size_t)g.nx * g.ny;
  const size_t c = k * plane + (size_t)j * g.nx + i;
  if (!VOFP_IN(c, ncells(g), CHK_CELL_LOAD)) return base;
  const double pc = __ldg(p + c);
  double xs, ys, zlo, zhi;
  {
    double lo, hi;
    // ghosts: wrapped (P), copied at an N end, negated at a D end (low end D for DD, DN; high end for DD, ND)
    if (i > 0) lo = __ldg(p + c - 1);
    else lo = g.bcx == VOFP_BC_P ? __ldg(p + c + g.nx - 1) : neg_if(pc, g.bcx == VOFP_BC_DD || g.bcx == VOFP_BC_DN);
    if (i < g.nx - 1) hi = __ldg(p + c + 1);
    else hi = g.bcx == VOFP_BC_P ? __ldg(p + c - (g.nx - 1)) : neg_if(pc, g.bcx == VOFP_BC_DD || g.bcx == VOFP_BC_ND);
    xs = hi + lo;
  }
  {
    double lo, hi;
    if (j > 0) lo = __ldg(p + c - g.nx);
    else lo = g.bcy == VOFP_BC_P ? __ldg(p + c + (size_t)(g.ny - 1) * g.nx)
                                 : neg_if(pc, g.bcy == VOFP_BC_DD || g.bcy == VOFP_BC_DN);
    if (j < g.ny - 1) hi = __ldg(p + c + g.nx);
    else hi = g.bcy == VOFP_BC_P ? __ldg(p + c - (size_t)(g.ny - 1) * g.nx)
                                 : neg_if(pc, g.bcy == VOFP_BC_DD || g.bcy == VOFP_BC_ND);
    ys = hi + lo;
  }
  {
    const bool lowN = g.bcz == VOFP_BC_NN || g.bcz == VOFP_BC_ND;
    const bool highN = g.bcz == VOFP_BC_NN || g.bcz == VOFP_BC_DN;
    if (k > 0) zlo = __ldg(p + c - plane);
    else zlo = g.bcz == VOFP_BC_P ? __ldg(p + c + (size_t)(g.nz - 1) * plane) : neg_if(pc, !lowN);
    if (k < g.nz - 1) zhi = __ldg(p + c + plane);
    else zhi = g.bcz == VOFP_BC_P ? __ldg(p + c - (size_t)(g.nz - 1) * plane) : neg_if(pc, !highN);
  }
  return fma(-g.rdx2, xs,
             fma(-g.rdy2, ys, fma(-__ldg(g.czc + k), pc, fma(-__ldg(g.czp + k), zhi, fma(-__ldg(g.czm + k), zlo, base)))));
}

template <int MODE>
__device__ __forceinline__ double rhs_at(const XArgs& a, int i, int j, int k, double fbar) {
  const size_t c = ((size_t)k * a.g.ny + j) * a.g.nx + i;
  if (!VOFP_IN(c, ncells(a.g), CHK_CELL_LOAD)) return 0.0;
  double f;
  if (MODE == RHS_F) {
    f = __ldg(a.f + c);
    if (a.scale != 1.0) f *= a.scale;
  } else if (MODE == RHS_DIV) {
    f = divergence_at(a.g, a.u, a.v, a.w, i, j, k, a.src ? -__ldg(a.src + c) : 0.0) * a.scale;
  } else if (MODE == RHS_STEFAN) {
    const double3 gc = grad_c_at(a.g, a.C, i, j, k, a.grad_mode);
    f = __ldg(a.mdot + c) * a.coef * sqrt(gc.x * gc.x + gc.y * gc.y + gc.z * gc.z);
  } else if (MODE == RHS_DIV_STEFAN) {
    const double3 gc = grad_c_at(a.g, a.C, i, j, k, a.grad_mode);
    const double s = __ldg(a.mdot + c) * a.coef * sqrt(gc.x * gc.x + gc.y * gc.y + gc.z * gc.z);
    f = divergence_at(a.g, a.u, a.v, a.w, i, j, k, -s) * a.scale;
  } else {
    // (fbar = 0 unless the operator is singular: no subtraction then)
    f = resid_at(a.g, a.p, i, j, k, a.defect_sum ? __ldg(a.f + c) - fbar : __ldg(a.f + c));
  }
  return f;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  }
  return s;
}

// Item t of a block's (line pair, sample) loop: pair t / n, sample t % n -- by shift and mask for a
// power-of-two n (lgn >= 0), else by division.
__device__ __forceinline__ void split_item(int t, int n, int lgn, int& pb, int& i) {
  if (lgn >= 0) {
    pb = t >> lgn;
    i = t & (n - 1);
  } else {
    pb = t / n;
    i = t - pb * n;
  }
}
__device__ __forceinline__ int pow2_log(int n) { return (n & (n - 1)) == 0 ? 31 - __clz(n) : -1; }

// x pass, forward: RHS + transform of line pairs (2p, 2p+1) of the flattened (k, j) line index.
// Block body: `bx` is the block's index within this grid's launch (batched launches pass a local index).
template <typename T, typename C, int MODE>
__device__ __forceinline__ void xfwd_block(const XArgs& a, int bx, unsigned char* smem_raw, double* red) {
  typedef decltype(C::x) R;
  C* b0 = reinterpret_cast<C*>(smem_raw);
  const int n = a.g.nx;
  const int PB = a.pb;
  const int ld = fft_span(a.fd, a.blu);
  C* b1 = b0 + PB * ld;
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const long nlines = (long)a.g.ny * a.g.nz;
  const long pair0 = (long)bx * PB;
  const int bc = a.g.bcx;
  const int lgn = pow2_log(n);
  // (k, j) of the block's 2 PB lines, computed once instead of a 64-bit division per sample
  __shared__ int lk[2 * kMaxPB], lj[2 * kMaxPB];
  if (threadIdx.x < 2 * PB) {
    const long l = 2 * pair0 + threadIdx.x;
    lk[threadIdx.x] = (int)(l / a.g.ny);
    lj[threadIdx.x] = (int)(l - (long)lk[threadIdx.x] * a.g.ny);
  }
  __syncthreads();
  const bool stats = a.info || a.sq_out || a.fv_out || a.abs_out;
  // FP64 plans keep every sum in FP64; reduced-precision plans keep only sum f V (the compatibility defect)
  // in FP64 and accumulate the norms, which feed thresholds only, in FP32
  constexpr bool f64 = std::is_same<T, double>::value;
  const double fbar = (MODE == RHS_RESID && a.defect_sum) ? *a.defect_sum * a.inv_volume : 0.0;
  double acc_abs = 0, acc_sq = 0, acc_fv = 0;
  float accf_abs = 0.0f, accf_sq = 0.0f;
  for (int t = threadIdx.x; t < PB * n; t += blockDim.x) {
    int pb, i;
    split_item(t, n, lgn, pb, i);
    const long l0 = 2 * (pair0 + pb), l1 = l0 + 1;
    R fa = (R)0, fb = (R)0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long l = h ? l1 : l0;
      if (l < nlines) {
        const int k = lk[2 * pb + h], j = lj[2 * pb + h];
        const double f = rhs_at<MODE>(a, i, j, k, fbar);
        const R fr = red_of(f, (R*)nullptr);  // integer-pipe conversion in reduced-precision plans
        if (a.fsave && VOFP_IN(l * n + i, nlines * n, CHK_XFWD_STORE)) a.fsave[l * n + i] = f;
        if (stats) {
          if (f64) {
            const double vol = __ldg(a.g.vol + k);
            acc_abs = fma(fabs(f), vol, acc_abs);
            acc_sq = fma(f, f, acc_sq);
            acc_fv = fma(f, vol, acc_fv);
          } else {
            const float fs = lead(fr);
            accf_abs = fmaf(fabsf(fs), __ldg(a.g.volf + k), accf_abs);
            accf_sq = fmaf(fs, fs, accf_sq);
            if (a.fv_out) acc_fv = fma(f, __ldg(a.g.vol + k), acc_fv);
          }
        }
        if (h)
          fb = fr;
        else
          fa = fr;
      }
    }
    if (quarter_bc(bc)) {
      int pos;
      C v;
      quarter_load<C>(i, n, bc, fa, fb, reinterpret_cast<const C*>(a.quart), pos, v);
      b0[pb * ld + pos] = v;
      continue;
    }
    int idx = i;
    bool fl = false;
    if (bc != VOFP_BC_P) {
      idx = dct_perm(i, n);
      fl = bc == VOFP_BC_DD && (i & 1);
    }
    b0[pb * ld + idx] = cmk<C>(neg_if(fa, fl), neg_if(fb, fl));
  }
  if (!f64) {
    acc_abs = accf_abs;
    acc_sq = accf_sq;
  }
  if (a.info || a.abs_out) {
    const double s1 = block_sum(acc_abs, red);
    if (threadIdx.x == 0 && s1 != 0) {
      if (a.info) atomicAdd(&a.info->abs_sum, s1);
      if (a.abs_out) atomicAdd(a.abs_out, s1);
    }
  }
  if (a.sq_out) {
    const double s2 = block_sum(acc_sq, red);
    if (threadIdx.x == 0 && s2 != 0) atomicAdd(a.sq_out, s2);
  }
  if (a.fv_out) {
    const double s3 = block_sum(acc_fv, red);
    if (threadIdx.x == 0 && s3 != 0) atomicAdd(a.fv_out, s3);
  }
  __syncthreads();
  const C* Z = fft_smem<C>(b0, b1, PB, a.fd, reinterpret_cast<const C*>(a.tw), ld,
                           reinterpret_cast<const C*>(a.blu));
  const C* quart = reinterpret_cast<const C*>(a.quart);
  T* S = reinterpret_cast<T*>(a.S);
  for (int t = threadIdx.x; t < PB * n; t += blockDim.x) {
    int pb, q;
    split_item(t, n, lgn, pb, q);
    const long l0 = 2 * (pair0 + pb), l1 = l0 + 1;
    R oa, ob;
    fwd_post<C>(Z + pb * ld, n, bc, q, quart, oa, ob);
    if (l0 < nlines && VOFP_IN(l0 * n + q, nlines * n, CHK_XFWD_STORE)) S[l0 * n + q] = (T)oa;
    if (l1 < nlines && VOFP_IN(l1 * n + q, nlines * n, CHK_XFWD_STORE)) S[l1 * n + q] = (T)ob;
  }
}

template <typename T, typename C, int MODE>
__global__ void __launch_bounds__(256) k_xfwd(XArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  xfwd_block<T, C, MODE>(a, blockIdx.x, smem_raw, red);
}

// Number of blocks of the x pass for one grid.
__host__ __device__ __forceinline__ int xpass_blocks(int ny, int nz, int pb) {
  const long npairs = ((long)ny * nz + 1) / 2;
  return (int)((npairs + pb - 1) / pb);
}

struct YArgs {
  int nx, ny, nz, bc;
  FftDesc fd;
  const void* tw;
  const void* quart;
  const void* blu;
  int tx;  // columns per block (even)
  void* S;
  const double* skip_conv;
  int skip_k;
  double tol2;
};

// y pass on a tile of `tx` columns (pairs of columns share one complex FFT) of plane k = by.
template <typename T, typename C, bool INV>
__device__ __forceinline__ void ypass_block(const YArgs& a, int bx, int by, unsigned char* smem_raw) {
  typedef decltype(C::x) R;
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const int n = a.ny;
  const int B = a.tx >> 1;
  C* b0 = reinterpret_cast<C*>(smem_raw);
  const int ld = y_ld(fft_span(a.fd, a.blu));
  C* b1 = b0 + B * ld;
  const int i0 = bx * a.tx;
  const size_t base = (size_t)by * a.ny * a.nx;
  [[maybe_unused]] const size_t cells = (size_t)a.nx * a.ny * a.nz;  // (bounds-checked builds)
  T* S = reinterpret_cast<T*>(a.S);
  const int bc = a.bc;
  const C* quart = reinterpret_cast<const C*>(a.quart);
  if (!INV) {
    for (int t = threadIdx.x; t < B * n; t += blockDim.x) {
      const int c = t % B, j = t / B;
      const int i = i0 + 2 * c;
      const size_t o = base + (size_t)j * a.nx + i;
      const R va = i < a.nx && VOFP_IN(o, cells, CHK_Y_PASS) ? (R)S[o] : (R)0;
      const R vb = i + 1 < a.nx && VOFP_IN(o + 1, cells, CHK_Y_PASS) ? (R)S[o + 1] : (R)0;
      if (quarter_bc(bc)) {
        int pos;
        C v;
        quarter_load<C>(j, n, bc, va, vb, quart, pos, v);
        b0[c * ld + pos] = v;
        continue;
      }
      int idx = j;
      bool fl = false;
      if (bc != VOFP_BC_P) {
        idx = dct_perm(j, n);
        fl = bc == VOFP_BC_DD && (j & 1);
      }
      b0[c * ld + idx] = cmk<C>(neg_if(va, fl), neg_if(vb, fl));
    }
    __syncthreads();
    const C* Z = fft_smem<C>(b0, b1, B, a.fd, reinterpret_cast<const C*>(a.tw), ld,
                             reinterpret_cast<const C*>(a.blu));
    for (int t = threadIdx.x; t < B * n; t += blockDim.x) {
      const int c = t % B, q = t / B;
      const int i = i0 + 2 * c;
      R oa, ob;
      fwd_post<C>(Z + c * ld, n, bc, q, quart, oa, ob);
      const size_t o = base + (size_t)q * a.nx + i;
      if (i < a.nx && VOFP_IN(o, cells, CHK_Y_PASS)) S[o] = (T)oa;
      if (i + 1 < a.nx && VOFP_IN(o + 1, cells, CHK_Y_PASS)) S[o + 1] = (T)ob;
    }
  } else {
    // stage the tile column-major in b1: column col holds the packed line of length n
    R* st = reinterpret_cast<R*>(b1);
    for (int t = threadIdx.x; t < B * n; t += blockDim.x) {
      const int c = t % B, q = t / B;
      const int i = i0 + 2 * c;
      const size_t o = base + (size_t)q * a.nx + i;
      st[(2 * c) * n + q] = i < a.nx && VOFP_IN(o, cells, CHK_Y_PASS) ? (R)S[o] : (R)0;
      st[(2 * c + 1) * n + q] = i + 1 < a.nx && VOFP_IN(o + 1, cells, CHK_Y_PASS) ? (R)S[o + 1] : (R)0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < B * n; t += blockDim.x) {
      const int c = t / n, m = t - c * n;
      const R* ra = st + (2 * c) * n;
      const R* rb = st + (2 * c + 1) * n;
      if (quarter_bc(bc)) {  // the inverse is the same transform: spectral index m placed as a sample
        int pos;
        C v;
        quarter_load<C>(m, n, bc, ra[m], rb[m], quart, pos, v);
        b0[c * ld + pos] = v;
        continue;
      }
      b0[c * ld + m] = inv_pre<C>([&](int q) { return ra[q]; }, [&](int q) { return rb[q]; }, n, bc, m, quart);
    }
    __syncthreads();
    const C* Y = fft_smem<C>(b0, b1, B, a.fd, reinterpret_cast<const C*>(a.tw), ld,
                             reinterpret_cast<const C*>(a.blu));
    for (int t = threadIdx.x; t < B * n; t += blockDim.x) {
      const int c = t % B, j = t / B;
      const int i = i0 + 2 * c;
      const size_t o = base + (size_t)j * a.nx + i;
      if (quarter_bc(bc)) {  // the transform again (twice it, as every pass): a forward-inverse pair gives 2n x
        R oa, ob;
        fwd_post<C>(Y + c * ld, n, bc, j, quart, oa, ob);
        if (i < a.nx && VOFP_IN(o, cells, CHK_Y_PASS)) S[o] = (T)oa;
        if (i + 1 < a.nx && VOFP_IN(o + 1, cells, CHK_Y_PASS)) S[o + 1] = (T)ob;
        continue;
      }
      int idx = j;
      bool fl = false;
      if (bc != VOFP_BC_P) {
        idx = dct_perm(j, n);
        fl = bc == VOFP_BC_DD && (j & 1);
      }
      const C y = Y[c * ld + idx];
      if (i < a.nx && VOFP_IN(o, cells, CHK_Y_PASS)) S[o] = (T)neg_if(y.x, fl);
      if (i + 1 < a.nx && VOFP_IN(o + 1, cells, CHK_Y_PASS)) S[o + 1] = (T)neg_if(y.y, !fl);
    }
  }
}

template <typename T, typename C, bool INV>
__global__ void __launch_bounds__(256) k_ypass(YArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ypass_block<T, C, INV>(a, blockIdx.x, blockIdx.y, smem_raw);
}

struct XInvArgs {
  int nx, ny, nz, bc;
  FftDesc fd;
  const void* tw;
  const void* quart;
  const void* blu;
  int pb;
  const void* S;
  double* p;
  int accumulate;  // 0: p = value, 1: p += value
  const double* skip_conv;
  int skip_k;
  double tol2;
  const double* dz;   // with mean_out: accumulate sum value * dz[k] (the gauge of the result)
  double* mean_out;
  double* d2_out;     // if non-null: accumulate sum value^2 (size of this correction)
  const ff* dzff;     // dz as FP32 pairs (reduced-precision plans' gauge sum)
};

// x pass, inverse: two packed lines per complex FFT, result written (or added) to the FP64 cell array p.
template <typename T, typename C>
__device__ __forceinline__ void xinv_block(const XInvArgs& a, int bx, unsigned char* smem_raw, double* red) {
  typedef decltype(C::x) R;
  if (launch_skipped(a.skip_conv, a.skip_k, a.tol2)) return;
  const int n = a.nx;
  const int PB = a.pb;
  const int ld = fft_span(a.fd, a.blu);
  C* b0 = reinterpret_cast<C*>(smem_raw);
  C* b1 = b0 + PB * ld;
  const long nlines = (long)a.ny * a.nz;
  const long pair0 = (long)bx * PB;
  const T* S = reinterpret_cast<const T*>(a.S);
  const int bc = a.bc;
  const C* quart = reinterpret_cast<const C*>(a.quart);
  R* st = reinterpret_cast<R*>(b1);
  const int lgn = pow2_log(n);
  // z plane of each of the block's 2 PB lines (the gauge sum's dz), computed once instead of a 64-bit
  // division per sample
  __shared__ int lplane[2 * kMaxPB];
  if (threadIdx.x < 2 * PB) lplane[threadIdx.x] = (int)((2 * pair0 + threadIdx.x) / a.ny);
  {
    // the block's lines are consecutive: one contiguous run of the spectrum
    const long lim = (nlines - 2 * pair0) * n;
    const T* src = S + 2 * pair0 * n;
    for (int t = threadIdx.x; t < 2 * PB * n; t += blockDim.x)
      st[t] = t < lim && VOFP_IN(2 * pair0 * n + t, nlines * n, CHK_XINV) ? (R)src[t] : (R)0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < PB * n; t += blockDim.x) {
    int pb, m;
    split_item(t, n, lgn, pb, m);
    const R* ra = st + (2 * pb) * n;
    const R* rb = st + (2 * pb + 1) * n;
    if (quarter_bc(bc)) {  // the inverse is the same transform: spectral index m placed as a sample
      int pos;
      C v;
      quarter_load<C>(m, n, bc, ra[m], rb[m], quart, pos, v);
      b0[pb * ld + pos] = v;
      continue;
    }
    b0[pb * ld + m] = inv_pre<C>([&](int q) { return ra[q]; }, [&](int q) { return rb[q]; }, n, bc, m, quart);
  }
  __syncthreads();
  const C* Y = fft_smem<C>(b0, b1, PB, a.fd, reinterpret_cast<const C*>(a.tw), ld,
                           reinterpret_cast<const C*>(a.blu));
  // FP64 plans sum in FP64.  Reduced-precision plans: the correction's size (a threshold) in FP32 and its
  // gauge sum (subtracted from p at the end, so it must be exact to well below the tolerance) in FP32 pairs
  // of FP32 products -- no FP64 arithmetic per cell beyond the addition into p.
  constexpr bool f64 = std::is_same<T, double>::value;
  double acc = 0, acc2 = 0;
  ff accm(0.0f, 0.0f);
  float acc2f = 0.0f;
  for (int t = threadIdx.x; t < PB * n; t += blockDim.x) {
    int pb, i;
    split_item(t, n, lgn, pb, i);
    const long l0 = 2 * (pair0 + pb), l1 = l0 + 1;
    R ya, yb;
    if (quarter_bc(bc)) {  // the transform again (twice it, as every pass): a forward-inverse pair gives 2n x
      fwd_post<C>(Y + pb * ld, n, bc, i, quart, ya, yb);
    } else {
      int idx = i;
      bool fl = false;
      if (bc != VOFP_BC_P) {
        idx = dct_perm(i, n);
        fl = bc == VOFP_BC_DD && (i & 1);
      }
      const C y = Y[pb * ld + idx];
      ya = neg_if(y.x, fl);
      yb = neg_if(y.y, !fl);
    }
    const double va = wide_of(ya), vb = wide_of(yb);  // integer-pipe widening (one FP64 add for a pair)
    if (!a.p) {
      // norm only (the error estimate of a refinement plan): the transform's output is not stored
    } else if (a.accumulate) {
      if (l0 < nlines && VOFP_IN(l0 * n + i, nlines * n, CHK_XINV)) a.p[l0 * n + i] += va;
      if (l1 < nlines && VOFP_IN(l1 * n + i, nlines * n, CHK_XINV)) a.p[l1 * n + i] += vb;
    } else {
      if (l0 < nlines && VOFP_IN(l0 * n + i, nlines * n, CHK_XINV)) a.p[l0 * n + i] = va;
      if (l1 < nlines && VOFP_IN(l1 * n + i, nlines * n, CHK_XINV)) a.p[l1 * n + i] = vb;
    }
    if (f64) {
      if (a.mean_out) {
        if (l0 < nlines) acc = fma(va, __ldg(a.dz + lplane[2 * pb]), acc);
        if (l1 < nlines) acc = fma(vb, __ldg(a.dz + lplane[2 * pb + 1]), acc);
      }
      if (a.d2_out) {
        if (l0 < nlines) acc2 = fma(va, va, acc2);
        if (l1 < nlines) acc2 = fma(vb, vb, acc2);
      }
    } else {
      if (a.mean_out) {
        if (l0 < nlines) accm += ff_of(ya) * a.dzff[lplane[2 * pb]];
        if (l1 < nlines) accm += ff_of(yb) * a.dzff[lplane[2 * pb + 1]];
      }
      if (a.d2_out) {
        const float fa = lead(ya), fb = lead(yb);
        if (l0 < nlines) acc2f = fmaf(fa, fa, acc2f);
        if (l1 < nlines) acc2f = fmaf(fb, fb, acc2f);
      }
    }
  }
  if (!f64) {
    acc = (double)accm;
    acc2 = acc2f;
  }
  if (a.mean_out) {
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0 && s != 0) atomicAdd(a.mean_out, s);
  }
  if (a.d2_out) {
    const double s = block_sum(acc2, red);
    if (threadIdx.x == 0 && s != 0) atomicAdd(a.d2_out, s);
  }
}

template <typename T, typename C>
__global__ void __launch_bounds__(256) k_xinv(XInvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  xinv_block<T, C>(a, blockIdx.x, smem_raw, red);
}

// The FP32 passes with their registers capped at 48 (five 256-thread blocks per SM; left alone the compiler
// takes 58 for the x passes and drops that to four).  The FP32 x pass that also evaluates the Stefan source
// keeps the plain kernel: it spills under the cap.
template <int MODE>
__global__ void __launch_bounds__(256, 4) k_xfwd_f32(XArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  xfwd_block<float, float2, MODE>(a, blockIdx.x, smem_raw, red);
}
template <bool INV>
__global__ void __launch_bounds__(256, 4) k_ypass_f32(YArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ypass_block<float, float2, INV>(a, blockIdx.x, blockIdx.y, smem_raw);
}
template <int UNUSED>
__global__ void __launch_bounds__(256, 4) k_xinv_f32(XInvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  xinv_block<float, float2>(a, blockIdx.x, smem_raw, red);
}

// The FP64 passes capped at 64 registers (four 256-thread blocks per SM instead of three): they are bound by
// the FP64 pipe, which more resident warps keep busier.
template <int MODE>
__global__ void __launch_bounds__(256, 4) k_xfwd_f64(XArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  xfwd_block<double, double2, MODE>(a, blockIdx.x, smem_raw, red);
}
template <bool INV>
__global__ void __launch_bounds__(256, 4) k_ypass_f64(YArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ypass_block<double, double2, INV>(a, blockIdx.x, blockIdx.y, smem_raw);
}
template <int UNUSED>
__global__ void __launch_bounds__(256, 4) k_xinv_f64(XInvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  xinv_block<double, double2>(a, blockIdx.x, smem_raw, red);
}

typedef void (*XFwdKernel)(XArgs);
typedef void (*YPassKernel)(YArgs);
typedef void (*XInvKernel)(XInvArgs);

// The kernel that runs a pass for spectrum type T.
template <typename T, typename C, int MODE>
inline XFwdKernel xfwd_kernel() {
  if constexpr (std::is_same<T, float>::value && MODE != RHS_DIV_STEFAN) return k_xfwd_f32<MODE>;
  else return k_xfwd<T, C, MODE>;
}
template <typename T, typename C, bool INV>
inline YPassKernel ypass_kernel() {
  if constexpr (std::is_same<T, float>::value) return k_ypass_f32<INV>;
  else return k_ypass<T, C, INV>;
}
template <typename T, typename C>
inline XInvKernel xinv_kernel() {
  if constexpr (std::is_same<T, float>::value) return k_xinv_f32<0>;
  else return k_xinv<T, C>;
}

}  // namespace vofp
