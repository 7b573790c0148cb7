// y transform on column tiles staged by the Tensor Memory Accelerator (FP64, FP32 and FP32-pair spectra).
//
// The y pass (A3 forward, A5 inverse) transforms every column of each z plane.  A column tile -- tx = 2B
// adjacent columns, all ny rows of one plane -- is one box of the spectrum viewed as a (ny nz) x nx matrix, and
// a 2-D TMA load copies it into shared memory row after row.  Element j of the complex line c (the packed
// columns 2c, 2c + 1) then sits at tile[j B + c]: the lines are element-major, and the 32 threads of a warp,
// taking consecutive lines at every butterfly, read and write consecutive complex words -- the tile is never
// transposed.  The CTAs are persistent and double-buffered: while one tile is transformed, the load of the next
// one is in flight.  Power-of-two ny only (radix 8 / 4 / 2 stages indexed by shifts and masks); the other
// lengths keep the gather kernel of passes.cuh.  The loads read this GPU's own memory only (no multicast).
//
// Every wait on a tile load is bounded (2^31 clock cycles, about a second): on expiry the CTA records a timeout
// in the plan's device info, waits (bounded) for its other load in flight, and returns.
#pragma once

#include <cuda.h>

#include "passes.cuh"

namespace vofp {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of `bar`; false once 2^31 clock cycles have passed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}
// Order this thread's (and, after a barrier, the CTA's) generic accesses of shared memory before the async
// proxy's next write into it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 2-D tile load of the box at element coordinates (x, y) into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Stockham stage on element-major lines (element e of line b at buf[(e << lgB) + b], 2^lgB lines) of
// power-of-two length 2^lgn; thread items run over the lines fastest.
template <typename C, int RAD>
__device__ __forceinline__ void fft_stage_em(const C* __restrict__ src, C* __restrict__ dst, int lgB, int lgn,
                                             int lgNs, const C* __restrict__ tw) {
  constexpr int lgR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
  const int lgNR = lgn - lgR;
  const int mB = (1 << lgB) - 1;
  const int mNs = (1 << lgNs) - 1;
  const int lgtw = lgn - lgNs - lgR;
  const int total = 1 << (lgB + lgNR);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = t & mB;
    const int j = t >> lgB;
    const int k = j & mNs;
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[((j + (r << lgNR)) << lgB) + bi];
    if (k != 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[(r * k) << lgtw]);
    }
    dft_small<C, RAD>(v);
    const int base = ((j - k) << lgR) + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[((base + (r << lgNs)) << lgB) + bi] = v[r];
  }
}

// All stages of fd (radices 8, 4, 2) on element-major lines; returns the buffer holding the result.
template <typename C>
__device__ C* fft_em(C* a, C* b, int lgB, int lgn, const FftDesc& fd, const C* __restrict__ tw) {
  int lgNs = 0;
  for (int s = 0; s < fd.nst; ++s) {
    const int R = fd.radix[s];
    if (R == 8) fft_stage_em<C, 8>(a, b, lgB, lgn, lgNs, tw);
    else if (R == 4) fft_stage_em<C, 4>(a, b, lgB, lgn, lgNs, tw);
    else fft_stage_em<C, 2>(a, b, lgB, lgn, lgNs, tw);
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
    lgNs += R == 8 ? 3 : (R == 4 ? 2 : 1);
  }
  return a;
}

// The same transform with the length (2^LGN), the lines per tile (2^LGB) and the block size (NT) known at
// compile time: every index becomes an immediate offset, the loops unroll.  Radix sequence as the plan's
// factorisation of a power of two (a leading 2, 4 or 4 x 4, then 8s).
__host__ __device__ constexpr int p2_nstages(int lgn) {
  return lgn % 3 == 1 ? (lgn / 3 > 0 ? lgn / 3 + 1 : 1) : (lgn % 3 == 2 ? lgn / 3 + 1 : lgn / 3);
}
__host__ __device__ constexpr int p2_radix(int lgn, int s) {
  return lgn % 3 == 1 ? (lgn / 3 > 0 ? (s < 2 ? 4 : 8) : 2) : (lgn % 3 == 2 ? (s == 0 ? 4 : 8) : 8);
}
template <typename C, int RAD, int LGB, int LGN, int LGNS, int NT>
__device__ __forceinline__ void fft_stage_emc(const C* __restrict__ src, C* __restrict__ dst,
                                              const C* __restrict__ tw) {
  constexpr int lgR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
  constexpr int LGNR = LGN - lgR;
  constexpr int TOTAL = 1 << (LGB + LGNR);
#pragma unroll
  for (int t0 = 0; t0 < TOTAL; t0 += NT) {
    const int t = t0 + (int)threadIdx.x;
    if (TOTAL % NT != 0 && t >= TOTAL) break;
    const int bi = t & ((1 << LGB) - 1);
    const int j = t >> LGB;
    const int k = j & ((1 << LGNS) - 1);
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[((j + (r << LGNR)) << LGB) + bi];
    if (LGNS > 0 && k != 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[(r * k) << (LGN - LGNS - lgR)]);
    }
    dft_small<C, RAD>(v);
    const int base = ((j - k) << lgR) + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[((base + (r << LGNS)) << LGB) + bi] = v[r];
  }
}
template <typename C, int LGB, int LGN, int NT, int S = 0, int LGNS = 0>
__device__ __forceinline__ C* fft_emc(C* a, C* b, const C* __restrict__ tw) {
  if constexpr (S == p2_nstages(LGN)) {
    return a;
  } else {
    constexpr int R = p2_radix(LGN, S);
    fft_stage_emc<C, R, LGB, LGN, LGNS, NT>(a, b, tw);
    __syncthreads();
    return fft_emc<C, LGB, LGN, NT, S + 1, LGNS + (R == 8 ? 3 : (R == 4 ? 2 : 1))>(b, a, tw);
  }
}

template <typename T>
struct CplxOf;
template <>
struct CplxOf<float> {
  typedef float2 C;
};
template <>
struct CplxOf<ff> {
  typedef cff C;
};
template <>
struct CplxOf<double> {
  typedef double2 C;
};

struct YTmaArgs {
  YArgs y;             // sizes, boundary condition, tables, spectrum, convergence skip
  int lgB;             // 2^lgB complex lines (2^(lgB+1) columns) per tile
  int tiles_x;         // tiles per plane
  vofp_devinfo* info;  // timeout flag (NULL: not recorded)
};

// Shared memory of one CTA: two tile buffers, one work buffer, the n-point twiddles, alignment slack.
__host__ __device__ __forceinline__ size_t ytma_smem_bytes(int n, int lgB, size_t csize) {
  return 3 * ((size_t)n << lgB) * csize + (size_t)n * csize + 128;
}

// Threads per CTA of the TMA y pass.
constexpr int kYTmaThreads = 512;

// LGN > 0: ny = 2^LGN and 2^LGB lines per tile fixed at compile time; LGN = 0: both read from the arguments.
template <typename T, bool INV, int LGN = 0, int LGB = 0>
__global__ void __launch_bounds__(kYTmaThreads) k_ypass_tma(const YTmaArgs a, const __grid_constant__ CUtensorMap tm) {
  typedef typename CplxOf<T>::C C;
  constexpr bool CT = LGN > 0;
  const YArgs& y = a.y;
  if (launch_skipped(y.skip_conv, y.skip_k, y.tol2)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long bar[2];
  const int n = CT ? (1 << LGN) : y.ny, lgn = CT ? LGN : 31 - __clz(n);
  const int lgB = CT ? LGB : a.lgB, B = 1 << lgB, tx = 2 * B;
  const int items = n << lgB;  // complex words per tile
  unsigned char* base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  C* const buf0 = reinterpret_cast<C*>(base);
  C* const buf1 = buf0 + items;
  C* W = buf0 + 2 * items;
  C* tws = W + items;
  const int ntiles = a.tiles_x * y.nz;
  const unsigned tile_bytes = (unsigned)((size_t)items * sizeof(C));
  const int boxr = n < 256 ? n : 256;
  auto issue = [&](int tile, int which) {
    const int k = tile / a.tiles_x, bx = tile - k * a.tiles_x;
    mbar_expect_tx(&bar[which], tile_bytes);
    for (int r0 = 0; r0 < n; r0 += boxr)
      tma_load_2d(reinterpret_cast<T*>(which ? buf1 : buf0) + (size_t)r0 * tx, &tm, bx * tx, k * n + r0,
                  &bar[which]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  const C* twg = reinterpret_cast<const C*>(y.tw);
  for (int t = threadIdx.x; t < n; t += kYTmaThreads) tws[t] = twg[t];
  __syncthreads();
  int tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) issue(tile, 0);
  T* S = reinterpret_cast<T*>(y.S);
  const C* quart = reinterpret_cast<const C*>(y.quart);
  const int bc = y.bc;
  const int nx = y.nx;
  [[maybe_unused]] const size_t cells = (size_t)nx * y.ny * y.nz;  // (bounds-checked builds)
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int cur = it & 1;
    const int nxt = tile + gridDim.x;
    if (threadIdx.x == 0 && nxt < ntiles) {
      fence_proxy_async_smem();
      issue(nxt, cur ^ 1);
    }
    const bool ok = mbar_wait_bounded(&bar[cur], (it >> 1) & 1);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        if (a.info) atomicOr(&a.info->timeout, 1u);
        if (nxt < ntiles) mbar_wait_bounded(&bar[cur ^ 1], ((it + 1) >> 1) & 1);
      }
      return;
    }
    C* In = cur ? buf1 : buf0;
    const int k = tile / a.tiles_x, bx = tile - k * a.tiles_x;
    const int i0 = bx * tx;
    const size_t pbase = (size_t)k * n * nx;
    if (!INV) {
      C* X = In;
      C* Y2 = W;
      if (bc != VOFP_BC_P) {  // reordered (and pre-twiddled) copy: DCT-II / DST-II, DCT-IV / DST-IV
        for (int t = threadIdx.x; t < items; t += kYTmaThreads) {
          const int c = t & (B - 1), j = t >> lgB;
          const C v = In[t];
          if (quarter_bc(bc)) {
            int pos;
            C w;
            quarter_load<C>(j, n, bc, v.x, v.y, quart, pos, w);
            W[(pos << lgB) + c] = w;
          } else {
            const bool fl = bc == VOFP_BC_DD && (j & 1);
            W[(dct_perm(j, n) << lgB) + c] = cmk<C>(neg_if(v.x, fl), neg_if(v.y, fl));
          }
        }
        __syncthreads();
        X = W;
        Y2 = In;
      }
      const C* Z;
      if constexpr (CT)
        Z = fft_emc<C, LGB, LGN, kYTmaThreads>(X, Y2, tws);
      else
        Z = fft_em(X, Y2, lgB, lgn, y.fd, tws);
      for (int t = threadIdx.x; t < items; t += kYTmaThreads) {
        const int c = t & (B - 1), q = t >> lgB;
        const int i = i0 + 2 * c;
        T oa, ob;
        fwd_post<C>(Z + c, n, bc, q, quart, oa, ob, B);
        const size_t o = pbase + (size_t)q * nx + i;
        if (i < nx && VOFP_IN(o, cells, CHK_Y_TMA)) S[o] = oa;
        if (i + 1 < nx && VOFP_IN(o + 1, cells, CHK_Y_TMA)) S[o + 1] = ob;
      }
    } else {
      for (int t = threadIdx.x; t < items; t += kYTmaThreads) {
        const int c = t & (B - 1), m = t >> lgB;
        const C* col = In + c;
        if (quarter_bc(bc)) {  // the inverse is the same transform: spectral index m placed as a sample
          int pos;
          C v;
          const C s = col[m << lgB];
          quarter_load<C>(m, n, bc, s.x, s.y, quart, pos, v);
          W[(pos << lgB) + c] = v;
          continue;
        }
        W[(m << lgB) + c] = inv_pre<C>([&](int q) { return col[q << lgB].x; },
                                       [&](int q) { return col[q << lgB].y; }, n, bc, m, quart);
      }
      __syncthreads();
      const C* Yv;
      if constexpr (CT)
        Yv = fft_emc<C, LGB, LGN, kYTmaThreads>(W, In, tws);
      else
        Yv = fft_em(W, In, lgB, lgn, y.fd, tws);
      for (int t = threadIdx.x; t < items; t += kYTmaThreads) {
        const int c = t & (B - 1), j = t >> lgB;
        const int i = i0 + 2 * c;
        const size_t o = pbase + (size_t)j * nx + i;
        T oa, ob;
        if (quarter_bc(bc)) {  // the transform again (twice it, as every pass)
          fwd_post<C>(Yv + c, n, bc, j, quart, oa, ob, B);
        } else {
          int idx = j;
          bool fl = false;
          if (bc != VOFP_BC_P) {
            idx = dct_perm(j, n);
            fl = bc == VOFP_BC_DD && (j & 1);
          }
          const C v = Yv[(idx << lgB) + c];
          oa = neg_if(v.x, fl);
          ob = neg_if(v.y, !fl);
        }
        if (i < nx && VOFP_IN(o, cells, CHK_Y_TMA)) S[o] = oa;
        if (i + 1 < nx && VOFP_IN(o + 1, cells, CHK_Y_TMA)) S[o + 1] = ob;
      }
    }
    __syncthreads();  // this tile's buffers are free again
  }
}

}  // namespace vofp
