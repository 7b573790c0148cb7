// Inverse x transform of the reduced-precision spectra on line tiles staged by the Tensor Memory Accelerator.
//
// The inverse x pass (A6) reads 2B consecutive spectral lines (rows of the spectrum), forms B complex lines
// from them (two real lines per complex FFT, as every pass), transforms, and writes or adds the result into the
// FP64 potential, summing the correction's size and (FP32 spectra of a singular operator) its gauge.  Here the
// lines arrive as one TMA box into shared memory (a 3-D view {min(n, 256), n / min(n, 256), lines} of the
// spectrum, so that a 512-sample line lands as one row), the CTAs are persistent and
// double-buffered (the next tile's load is in flight while this one is transformed, as in the TMA y pass), and
// the FFT of a power-of-two length 128, 256 or 512 runs with its length and stage sequence compiled in, line-
// major (a warp's threads on consecutive samples of a line).  When the pass adds into the potential, the tile's
// rows of p are fetched by a second TMA load issued as the tile starts, so they arrive while it is transformed
// (read one by one after the FFT, they stalled the pass).  Every wait on a tile load is bounded: on expiry the
// CTA records a timeout in the plan's device info, waits (bounded) for its other load in flight, and returns.
#pragma once

#include "ypass_tma.cuh"

namespace vofp {

// 3-D tile load of the box at element coordinates (x, y, z) into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Stockham stage on line-major lines (line b at buf[b << LGN], contiguous samples), length 2^LGN known at
// compile time, `batch` lines.
template <typename C, int RAD, int LGN, int LGNS, int NT>
__device__ __forceinline__ void fft_stage_lmc(const C* __restrict__ src, C* __restrict__ dst, int batch,
                                              const C* __restrict__ tw) {
  constexpr int lgR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
  constexpr int LGNR = LGN - lgR;
  const int total = batch << LGNR;
  for (int t = threadIdx.x; t < total; t += NT) {
    const int bi = t >> LGNR;
    const int j = t & ((1 << LGNR) - 1);
    const int k = j & ((1 << LGNS) - 1);
    const C* s = src + (bi << LGN);
    C* d = dst + (bi << LGN);
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = s[j + (r << LGNR)];
    if (LGNS > 0 && k != 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[(r * k) << (LGN - LGNS - lgR)]);
    }
    dft_small<C, RAD>(v);
    const int base = ((j - k) << lgR) + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) d[base + (r << LGNS)] = v[r];
  }
}
template <typename C, int LGN, int NT, int S = 0, int LGNS = 0>
__device__ __forceinline__ C* fft_lmc(C* a, C* b, int batch, const C* __restrict__ tw) {
  if constexpr (S == p2_nstages(LGN)) {
    return a;
  } else {
    constexpr int R = p2_radix(LGN, S);
    fft_stage_lmc<C, R, LGN, LGNS, NT>(a, b, batch, tw);
    __syncthreads();
    return fft_lmc<C, LGN, NT, S + 1, LGNS + (R == 8 ? 3 : (R == 4 ? 2 : 1))>(b, a, batch, tw);
  }
}

constexpr int kXTmaThreads = 512;

struct XTmaArgs {
  XInvArgs xi;         // sizes, boundary condition, tables, spectrum in, potential out, sums, skip
  int lgB;             // 2^lgB complex lines (2^(lgB+1) spectral lines) per tile
  vofp_devinfo* info;  // timeout flag (NULL: not recorded)
};

// Shared memory: two staged tiles (2B lines of T), two FFT buffers (B complex lines), the twiddles, the tile's
// rows of the potential (accumulating passes), slack.
__host__ __device__ __forceinline__ size_t xtma_smem_bytes(int n, int lgB, size_t rsize, bool acc) {
  return 2 * ((size_t)n << (lgB + 1)) * rsize + 2 * ((size_t)n << lgB) * 2 * rsize + (size_t)n * 2 * rsize +
         (acc ? ((size_t)n << (lgB + 1)) * sizeof(double) : 0) + 128;
}

// tm: the spectrum {min(n, 256), n / min(n, 256), lines} (T); tp: the potential, the same view (FP64), used when
// the pass accumulates into it.
template <typename T, int LGN, int LGB>
__global__ void __launch_bounds__(kXTmaThreads) k_xinv_tma(const XTmaArgs a, const __grid_constant__ CUtensorMap tm,
                                                           const __grid_constant__ CUtensorMap tp) {
  typedef typename CplxOf<T>::C C;
  const XInvArgs& x = a.xi;
  if (launch_skipped(x.skip_conv, x.skip_k, x.tol2)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long bar[3];  // the two spectrum tiles, the potential's rows
  __shared__ double red[32];
  constexpr int n = 1 << LGN, B = 1 << LGB, R2 = 2 * B;  // samples per line, complex lines, spectral lines
  __shared__ int lplane[R2];                             // z plane of each line of the tile
  unsigned char* base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  T* const st0 = reinterpret_cast<T*>(base);
  T* const st1 = st0 + R2 * n;
  C* const w0 = reinterpret_cast<C*>(st1 + R2 * n);
  C* const w1 = w0 + B * n;
  C* const tws = w1 + B * n;
  double* const pt = reinterpret_cast<double*>(tws + n);  // the tile's rows of p (accumulating passes)
  const bool acc = x.p && x.accumulate;
  const long nlines = (long)x.ny * x.nz;
  const long ntiles = (nlines + R2 - 1) / R2;
  const unsigned tile_bytes = (unsigned)(R2 * n * sizeof(T));
  auto issue = [&](long tile, int which) {
    mbar_expect_tx(&bar[which], tile_bytes);
    tma_load_3d(which ? st1 : st0, &tm, 0, 0, (int)(tile * R2), &bar[which]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    mbar_init_fence();
  }
  const C* twg = reinterpret_cast<const C*>(x.tw);
  for (int t = threadIdx.x; t < n; t += kXTmaThreads) tws[t] = twg[t];
  __syncthreads();
  long tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) issue(tile, 0);
  const int bc = x.bc;
  const C* quart = reinterpret_cast<const C*>(x.quart);
  float acc2f = 0.0f;
  ff accm(0.0f, 0.0f);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int cur = it & 1;
    const long nxt = tile + gridDim.x;
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
    const T* st = cur ? st1 : st0;
    const long l0 = tile * R2;
    if (threadIdx.x < R2) lplane[threadIdx.x] = (int)((l0 + threadIdx.x) / x.ny);
    if (acc && threadIdx.x == 0) {  // this tile's rows of p: in flight while the tile is transformed
      fence_proxy_async_smem();
      mbar_expect_tx(&bar[2], (unsigned)(R2 * n * sizeof(double)));
      tma_load_3d(pt, &tp, 0, 0, (int)l0, &bar[2]);
    }
    // (the box rows past the last line read zeros: those lines are computed and never stored)
    for (int t = threadIdx.x; t < (B << LGN); t += kXTmaThreads) {
      const int pb = t >> LGN, m = t & (n - 1);
      const T* ra = st + (2 * pb) * n;
      const T* rb = st + (2 * pb + 1) * n;
      if (quarter_bc(bc)) {
        int pos;
        C v;
        quarter_load<C>(m, n, bc, ra[m], rb[m], quart, pos, v);
        w0[(pb << LGN) + pos] = v;
        continue;
      }
      w0[(pb << LGN) + m] = inv_pre<C>([&](int q) { return ra[q]; }, [&](int q) { return rb[q]; }, n, bc, m, quart);
    }
    __syncthreads();
    const C* Y = fft_lmc<C, LGN, kXTmaThreads>(w0, w1, B, tws);
    if (acc) {
      const bool okp = mbar_wait_bounded(&bar[2], it & 1);
      if (__syncthreads_or(!okp)) {
        if (threadIdx.x == 0) {
          if (a.info) atomicOr(&a.info->timeout, 1u);
          if (nxt < ntiles) mbar_wait_bounded(&bar[cur ^ 1], ((it + 1) >> 1) & 1);
        }
        return;
      }
    }
    for (int t = threadIdx.x; t < (B << LGN); t += kXTmaThreads) {
      const int pb = t >> LGN, i = t & (n - 1);
      const long la = l0 + 2 * pb, lb = la + 1;
      T ya, yb;
      if (quarter_bc(bc)) {
        fwd_post<C>(Y + (pb << LGN), n, bc, i, quart, ya, yb);
      } else {
        int idx = i;
        bool fl = false;
        if (bc != VOFP_BC_P) {
          idx = dct_perm(i, n);
          fl = bc == VOFP_BC_DD && (i & 1);
        }
        const C y = Y[(pb << LGN) + idx];
        ya = neg_if(y.x, fl);
        yb = neg_if(y.y, !fl);
      }
      const double va = wide_of(ya), vb = wide_of(yb);
      if (x.p) {
        if (x.accumulate) {
          if (la < nlines && VOFP_IN(la * n + i, nlines * n, CHK_X_TMA)) x.p[la * n + i] = pt[(2 * pb) * n + i] + va;
          if (lb < nlines && VOFP_IN(lb * n + i, nlines * n, CHK_X_TMA))
            x.p[lb * n + i] = pt[(2 * pb + 1) * n + i] + vb;
        } else {
          if (la < nlines && VOFP_IN(la * n + i, nlines * n, CHK_X_TMA)) x.p[la * n + i] = va;
          if (lb < nlines && VOFP_IN(lb * n + i, nlines * n, CHK_X_TMA)) x.p[lb * n + i] = vb;
        }
      }
      if (x.mean_out) {
        if (la < nlines) accm += ff_of(ya) * x.dzff[lplane[2 * pb]];
        if (lb < nlines) accm += ff_of(yb) * x.dzff[lplane[2 * pb + 1]];
      }
      if (x.d2_out) {
        const float fa = lead(ya), fb = lead(yb);
        if (la < nlines) acc2f = fmaf(fa, fa, acc2f);
        if (lb < nlines) acc2f = fmaf(fb, fb, acc2f);
      }
    }
    __syncthreads();  // this tile's buffers are free again
  }
  if (x.mean_out) {
    const double s = block_sum((double)accm, red);
    if (threadIdx.x == 0 && s != 0) atomicAdd(x.mean_out, s);
  }
  if (x.d2_out) {
    const double s = block_sum((double)acc2f, red);
    if (threadIdx.x == 0 && s != 0) atomicAdd(x.d2_out, s);
  }
}

}  // namespace vofp
