// x transforms of the FP32 refinement plans on the tensor cores (tcgen05), as dense transform-matrix
// products.
//
// Every x transform of a line -- half-complex DFT (periodic), DCT-II / DST-II, DCT-IV / DST-IV, forward or
// inverse, with the factors the FFT passes apply -- is a linear map of the line, out = T in.  T (n x n, one
// per direction) is built once per plan by running the plan's own FP64 x passes on the identity lines, so it
// carries exactly their conventions; it is split into TF32 high and low parts and laid out as the MMA's A
// operand.  A pass then computes, for a tile of 64 lines, D[q][line] = sum_j T[q][j] X[line][j] with the
// tile X as the B operand (each line is contiguous in memory: the K-major layout the tf32 MMA needs, no
// transpose), in three TF32 products (T_hi X_hi + T_hi X_lo + T_lo X_hi, about FP32 accuracy; the
// refinement corrects the rest) accumulated in FP32 in tensor memory, 128 outputs per MMA block.  Lengths
// up to 512 (any length: no Bluestein form), at O(n) tensor-core work per value instead of O(log n) FP32
// butterflies.  The right-hand side (divergence, FP64 residual) is formed in FP64 while the tile is staged,
// and the inverse adds into the FP64 potential, as in the FFT passes.
//
// Pipeline per CTA (persistent over line tiles): K is cut into chunks; for chunk c the T chunk arrives by one
// bulk copy while the threads stage the data chunk (FP64 -> FP32 -> TF32 split) into shared memory in the
// tensor cores' core-matrix order, then one thread issues the chunk's MMAs and commits them to the stage's
// barrier; two stages alternate.  After the last chunk the 4 lane quarters of tensor memory are read back
// (tcgen05.ld) and written out, consecutive outputs of a line to consecutive lanes (coalesced).  Every wait is
// bounded (2^31 clock cycles): on expiry the CTA records a timeout in the plan's device info, waits (bounded)
// for its copies and products in flight, frees its tensor memory and returns.
#include <cmath>
#include <cstring>

#include "passes.cuh"
#include "solve_internal.h"
#include "ypass_tma.cuh"

namespace vofp {

constexpr int kXtcLines = 64;     // lines per tile (the MMA's N)
constexpr int kXtcThreads = 256;  // 8 warps: two per tensor-memory lane quarter in the read-back
constexpr int kXtcMaxN = 512;     // longest x axis (TMEM columns: 128-row output blocks x 64 lines <= 256)

// ---- tcgen05 / bulk-copy primitives ------------------------------------------------------------------------
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Shared-memory operand descriptor: K-major, no swizzle, 8-row x 16-byte core matrices; lbo = byte step between
// core matrices along K, sbo = along the rows.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// D (FP32, tensor memory) (+)= A B^T, kind::tf32, M = 128, N = 64, K = 8.
__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long ad, unsigned long long bd, unsigned idesc,
                                       unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_ld8(unsigned taddr, float* v) {
  unsigned r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}
// Nearest TF32 value of x (an FP32 value with the low 13 significand bits zero).
__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Table geometry for an x axis of n cells.
struct XtcGeom {
  int nmb;  // 128-row output blocks
  int kc;   // K chunk (columns of T per pipeline stage)
  int nch;  // chunks
};
__host__ __device__ __forceinline__ XtcGeom xtc_geom(int n) {
  XtcGeom g;
  g.nmb = (n + 127) / 128;
  g.kc = g.nmb <= 2 ? 32 : 16;
  g.nch = (n + g.kc - 1) / g.kc;
  return g;
}
// floats of one direction's table: chunks x {hi, lo} x output blocks x (128 x kc)
__host__ __device__ __forceinline__ size_t xtc_floats(const XtcGeom& g) {
  return (size_t)g.nch * 2 * g.nmb * 128 * g.kc;
}
// Tiles in shared memory (and the table chunks) are K-major core-matrix order: element (row r, column k) of a
// rows x kc tile at byte ((r / 8) (kc / 4) + k / 4) 128 + (r % 8) 16 + (k % 4) 4 -- i.e. position e of the
// tile's linear order is row (e / 32 / (kc/4)) 8 + (e % 32) / 4, column (e / 32 % (kc/4)) 4 + e % 4.

// ---- table construction -------------------------------------------------------------------------------------
__global__ void k_xtc_identity(double* P, int n) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < (size_t)n * n) P[t] = (t / n == t % n) ? 1.0 : 0.0;
}
// out[j][q] (the transform of identity line j) = T[q][j]: split into TF32 hi / lo in the A-operand layout.
__global__ void k_xtc_pack(const double* __restrict__ out, int n, XtcGeom g, float* __restrict__ T) {
  const size_t per = (size_t)128 * g.kc;
  const size_t total = xtc_floats(g);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t blk = t / per;
    const int e = (int)(t - blk * per);
    const int mb = (int)(blk % g.nmb);
    const int h = (int)((blk / g.nmb) % 2);
    const int c = (int)(blk / (2 * (size_t)g.nmb));
    // position e of the tile in core-matrix order -> (row, column)
    const int cmi = e >> 5, within = e & 31;
    const int r = (cmi / (g.kc >> 2)) * 8 + (within >> 2);
    const int kk = (cmi % (g.kc >> 2)) * 4 + (within & 3);
    const int q = mb * 128 + r, j = c * g.kc + kk;
    const double v = (q < n && j < n) ? out[(size_t)j * n + q] : 0.0;
    const float hi = tf32_rna((float)v);
    T[t] = h ? tf32_rna((float)(v - (double)hi)) : hi;
  }
}

// ---- the passes ----------------------------------------------------------------------------------------------
struct XtcArgs {
  int n;           // x cells
  int ny;          // lines per plane
  long nlines;     // ny * nz
  XtcGeom geo;
  const float* T;  // this direction's table
  XArgs xa;        // forward: right-hand side inputs, stats, spectrum out
  XInvArgs xi;     // inverse: spectrum in, potential out, sums
  vofp_devinfo* info;
};

__host__ __device__ __forceinline__ size_t xtc_stage_bytes(const XtcGeom& g) {
  return (size_t)2 * g.nmb * 128 * g.kc * 4 + (size_t)2 * kXtcLines * g.kc * 4;
}
__host__ __device__ __forceinline__ size_t xtc_smem_bytes(const XtcGeom& g) { return 2 * xtc_stage_bytes(g) + 128; }
__host__ __device__ __forceinline__ unsigned xtc_tmem_cols(const XtcGeom& g) {
  const int c = g.nmb * kXtcLines;
  return c <= 64 ? 64u : (c <= 128 ? 128u : (c <= 256 ? 256u : 512u));
}

// Bounded wait of every thread on `bar`'s phase `parity`; true on success (a CTA-uniform answer).
__device__ __forceinline__ bool cta_wait(unsigned long long* bar, unsigned parity) {
  const bool ok = mbar_wait_bounded(bar, parity);
  return !__syncthreads_or(!ok);
}

// DIR 0: forward (MODE = RHS_F, RHS_DIV or RHS_RESID), DIR 1: inverse.
template <int DIR, int MODE>
__global__ void __launch_bounds__(kXtcThreads) k_xtc(const XtcArgs a) {
  if (DIR == 0 ? launch_skipped(a.xa.skip_conv, a.xa.skip_k, a.xa.tol2)
               : launch_skipped(a.xi.skip_conv, a.xi.skip_k, a.xi.tol2))
    return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long tl[2], md[2];
  __shared__ unsigned tmem_slot;
  __shared__ int lk[kXtcLines], lj[kXtcLines];
  __shared__ double red[32];
  const XtcGeom g = a.geo;
  const int n = a.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  const size_t sbytes = xtc_stage_bytes(g);
  const unsigned abytes = (unsigned)((size_t)2 * g.nmb * 128 * g.kc * 4);
  const unsigned bhalf = (unsigned)(kXtcLines * g.kc * 4);  // bytes of one (hi or lo) data tile
  const unsigned tcols = xtc_tmem_cols(g);
  const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(kXtcLines >> 3) << 17) | ((128u >> 4) << 24);
  const unsigned lbo = 128, sbo = (unsigned)(g.kc >> 2) * 128;
  if (tid == 0) {
    mbar_init(&tl[0], 1);
    mbar_init(&tl[1], 1);
    mbar_init(&md[0], 1);
    mbar_init(&md[1], 1);
    mbar_init_fence();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;

  // per-thread sums (forward: |f| V, f^2 in FP32 and f V in FP64; inverse: delta^2 in FP32, gauge in FP32 pairs)
  float s_abs = 0.f, s_sq = 0.f;
  double s_fv = 0.0;
  ff s_mean(0.0f, 0.0f);
  const double fbar = (DIR == 0 && MODE == RHS_RESID && a.xa.defect_sum) ? *a.xa.defect_sum * a.xa.inv_volume : 0.0;
  const bool fstats = DIR == 0 && (a.xa.sq_out || a.xa.fv_out || a.xa.abs_out);

  unsigned use[2] = {0u, 0u};  // completed uses of each stage (its barrier phases)
  int gch = 0;                 // chunks issued by this CTA
  bool failed = false;
  const long ntiles = (a.nlines + kXtcLines - 1) / kXtcLines;
  for (long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const long line0 = tile * kXtcLines;
    if (tid < kXtcLines) {
      const long l = line0 + tid;
      lk[tid] = (int)(l / a.ny);
      lj[tid] = (int)(l - (long)lk[tid] * a.ny);
    }
    __syncthreads();
    int last = 0;
    for (int c = 0; c < g.nch; ++c, ++gch) {
      const int st = gch & 1;
      unsigned char* A = base + st * sbytes;
      float* B = reinterpret_cast<float*>(A + abytes);
      // the stage's previous products must be done before its buffers are refilled
      if (use[st] > 0 && !cta_wait(&md[st], (use[st] - 1) & 1)) {
        failed = true;
        break;
      }
      if (tid == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(&tl[st], abytes);
        bulk_copy_g2s(A, a.T + (size_t)c * (abytes / 4), abytes, &tl[st]);
      }
      // stage the data chunk: element e of the tile in core-matrix order (conflict-free stores)
      for (int e = tid; e < kXtcLines * g.kc; e += kXtcThreads) {
        const int cmi = e >> 5, within = e & 31;
        const int r = (cmi / (g.kc >> 2)) * 8 + (within >> 2);
        const int i = c * g.kc + (cmi % (g.kc >> 2)) * 4 + (within & 3);
        const long l = line0 + r;
        float x = 0.f;
        if (l < a.nlines && i < n && VOFP_IN(l * n + i, a.nlines * n, CHK_XTC)) {
          if (DIR == 0) {
            const int k = lk[r], j = lj[r];
            const double f = rhs_at<MODE>(a.xa, i, j, k, fbar);
            x = f32_lead_bits(f);
            if (a.xa.fsave) a.xa.fsave[l * n + i] = f;
            if (fstats) {
              s_abs = fmaf(fabsf(x), __ldg(a.xa.g.volf + k), s_abs);
              s_sq = fmaf(x, x, s_sq);
              if (a.xa.fv_out) s_fv = fma(f, __ldg(a.xa.g.vol + k), s_fv);
            }
          } else {
            x = __ldg(reinterpret_cast<const float*>(a.xi.S) + l * n + i);
          }
        }
        const float hi = tf32_rna(x);
        B[e] = hi;
        B[e + kXtcLines * g.kc] = tf32_rna(x - hi);
      }
      fence_proxy_async_smem();
      if (!cta_wait(&tl[st], use[st] & 1)) {
        failed = true;
        break;
      }
      tc_fence_after();
      if (tid == 0) {
        const unsigned a0 = smem_u32(A), b0 = smem_u32(B);
        for (int s = 0; s < (g.kc >> 3); ++s) {
          for (int mb = 0; mb < g.nmb; ++mb) {
            const unsigned d = tmem + (unsigned)(mb * kXtcLines);
            const unsigned first = (c == 0 && s == 0) ? 0u : 1u;
            const unsigned long long th = tc_desc(a0 + (unsigned)(mb * 128 * g.kc * 4) + s * 256, lbo, sbo);
            const unsigned long long tlo =
                tc_desc(a0 + (unsigned)((g.nmb + mb) * 128 * g.kc * 4) + s * 256, lbo, sbo);
            const unsigned long long xh = tc_desc(b0 + s * 256, lbo, sbo);
            const unsigned long long xl = tc_desc(b0 + bhalf + s * 256, lbo, sbo);
            tc_mma(d, th, xh, idesc, first);
            tc_mma(d, th, xl, idesc, 1u);
            tc_mma(d, tlo, xh, idesc, 1u);
          }
        }
        tc_commit(&md[st]);
      }
      ++use[st];
      last = st;
    }
    if (failed) break;
    // all products of the tile are done once the last stage's commit has arrived
    if (!cta_wait(&md[last], (use[last] - 1) & 1)) {
      failed = true;
      break;
    }
    tc_fence_after();
    // read back: warp w reads lane quarter (w & 3), half (w >> 2) of the tile's lines
    const int qd = warp & 3, half = warp >> 2;
    for (int mb = 0; mb < g.nmb; ++mb) {
      const int q = mb * 128 + qd * 32 + lane;
      for (int lb = 0; lb < kXtcLines / 2; lb += 8) {
        const int col = mb * kXtcLines + half * (kXtcLines / 2) + lb;
        float v[8];
        tc_ld8(tmem + ((unsigned)(qd * 32) << 16) + (unsigned)col, v);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int r = half * (kXtcLines / 2) + lb + u;
          const long l = line0 + r;
          if (l >= a.nlines || q >= n || !VOFP_IN(l * n + q, a.nlines * n, CHK_XTC)) continue;
          if (DIR == 0) {
            reinterpret_cast<float*>(a.xa.S)[l * n + q] = v[u];
          } else {
            const double w = f64_of_bits(v[u]);
            if (a.xi.p) {
              if (a.xi.accumulate)
                a.xi.p[l * n + q] += w;
              else
                a.xi.p[l * n + q] = w;
            }
            if (a.xi.d2_out) s_sq = fmaf(v[u], v[u], s_sq);
            if (a.xi.mean_out) s_mean += ff_of(v[u]) * a.xi.dzff[lk[r]];
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (failed) {
    // record it, let this CTA's copies and products in flight land (bounded), then free tensor memory
    if (tid == 0) {
      if (a.info) atomicOr(&a.info->timeout, 1u);
      for (int st = 0; st < 2; ++st) {
        mbar_wait_bounded(&tl[st], use[st] & 1);
        if (use[st] > 0) mbar_wait_bounded(&md[st], (use[st] - 1) & 1);
      }
    }
    tc_fence_before();
    __syncthreads();
  } else {
    // block sums into the convergence slots (as the FFT passes)
    if (DIR == 0) {
      if (a.xa.abs_out) {
        const double t = block_sum((double)s_abs, red);
        if (tid == 0 && t != 0) atomicAdd(a.xa.abs_out, t);
      }
      if (a.xa.sq_out) {
        const double t = block_sum((double)s_sq, red);
        if (tid == 0 && t != 0) atomicAdd(a.xa.sq_out, t);
      }
      if (a.xa.fv_out) {
        const double t = block_sum(s_fv, red);
        if (tid == 0 && t != 0) atomicAdd(a.xa.fv_out, t);
      }
    } else {
      if (a.xi.mean_out) {
        const double t = block_sum((double)s_mean, red);
        if (tid == 0 && t != 0) atomicAdd(a.xi.mean_out, t);
      }
      if (a.xi.d2_out) {
        const double t = block_sum((double)s_sq, red);
        if (tid == 0 && t != 0) atomicAdd(a.xi.d2_out, t);
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// ---- host side ------------------------------------------------------------------------------------------------
typedef void (*XtcKernel)(const XtcArgs);
template <int DIR, int MODE>
static void xtc_attr() {
  cudaFuncSetAttribute(k_xtc<DIR, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}
static void xtc_init_attributes() {
  if (!first_use_on_device(2)) return;
  xtc_attr<0, RHS_F>();
  xtc_attr<0, RHS_DIV>();
  xtc_attr<0, RHS_RESID>();
  xtc_attr<1, 0>();
}

// The tensor-core x passes apply to FP32 refinement plans with 8 <= nx <= 512 and at least nx lines (the
// tables are built in the plan's FP64 workspace), and only when the environment variable VOFP_X_TC is set to
// a non-zero value when the plan is created: measured on the GB300 they are slower than the FFT passes (the
// K-chunk pipeline is latency-bound: two CTA barriers per chunk, one CTA per SM), and FP32 accumulation of n
// products is several times less accurate than a log n stage FFT, which at 512^3 on the stretched grid leaves
// refinement results near the 1e-10 bar.  The FFT passes are the default.
size_t xtc_table_bytes(int nx, long nlines, int prec) {
  if (prec != VOFP_MIXED || nx < 8 || nx > kXtcMaxN || nlines < nx) return 0;
  const char* env = getenv("VOFP_X_TC");
  if (!env || env[0] == '\0' || env[0] == '0') return 0;
  return 2 * xtc_floats(xtc_geom(nx)) * sizeof(float);
}

int xtc_build(vofp_plan* pl, void* tables, cudaStream_t st) {
  const int n = pl->n[0];
  const XtcGeom g = xtc_geom(n);
  float* tf = reinterpret_cast<float*>(tables);
  float* ti = tf + xtc_floats(g);
  // identity lines in the scratch potential, their transforms in the FP64 right-hand-side buffer
  double* I = pl->P;
  double* O = pl->F;
  const size_t nn = (size_t)n * n;
  k_xtc_identity<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(I, n);
  int s = fp64_x_lines(pl, false, I, O, n, st);
  if (s) return s;
  k_xtc_pack<<<256, 256, 0, st>>>(O, n, g, tf);
  s = fp64_x_lines(pl, true, I, O, n, st);
  if (s) return s;
  k_xtc_pack<<<256, 256, 0, st>>>(O, n, g, ti);
  note_launches(3);
  pl->xtc_fwd = tf;
  pl->xtc_inv = ti;
  return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

static int xtc_grid(vofp_plan* pl, XtcKernel k, size_t smem, long tiles) {
  if (pl->xtc_grid <= 0) {
    int per_sm = 0, nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kXtcThreads, smem) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      return 0;
    }
    pl->xtc_grid = per_sm * nsm;
  }
  return (int)(tiles < pl->xtc_grid ? tiles : pl->xtc_grid);
}

bool xtc_xfwd(vofp_plan* pl, int mode, const XArgs& xa, cudaStream_t st) {
  if (!pl->xtc_fwd || (mode != RHS_F && mode != RHS_DIV && mode != RHS_RESID)) return false;
  xtc_init_attributes();
  XtcArgs a;
  memset(&a, 0, sizeof(a));
  a.n = pl->n[0];
  a.ny = pl->n[1];
  a.nlines = (long)pl->n[1] * pl->n[2];
  a.geo = xtc_geom(a.n);
  a.T = pl->xtc_fwd;
  a.xa = xa;
  a.info = pl->info;
  const size_t sm = xtc_smem_bytes(a.geo);
  const long tiles = (a.nlines + kXtcLines - 1) / kXtcLines;
  XtcKernel k = mode == RHS_F ? k_xtc<0, RHS_F> : (mode == RHS_DIV ? k_xtc<0, RHS_DIV> : k_xtc<0, RHS_RESID>);
  const int grid = xtc_grid(pl, k, sm, tiles);
  if (grid < 1) return false;
  const int kid = mode == RHS_F ? KID_XFWD : (mode == RHS_DIV ? KID_XFWD_DIV : KID_RESID);
  VOFP_LAUNCH(kid, st, (k<<<grid, kXtcThreads, sm, st>>>(a)));
  return true;
}

bool xtc_xinv(vofp_plan* pl, const XInvArgs& xi, cudaStream_t st) {
  if (!pl->xtc_inv) return false;
  xtc_init_attributes();
  XtcArgs a;
  memset(&a, 0, sizeof(a));
  a.n = pl->n[0];
  a.ny = pl->n[1];
  a.nlines = (long)pl->n[1] * pl->n[2];
  a.geo = xtc_geom(a.n);
  a.T = pl->xtc_inv;
  a.xi = xi;
  a.info = pl->info;
  const size_t sm = xtc_smem_bytes(a.geo);
  const long tiles = (a.nlines + kXtcLines - 1) / kXtcLines;
  const int grid = xtc_grid(pl, k_xtc<1, 0>, sm, tiles);
  if (grid < 1) return false;
  VOFP_LAUNCH(KID_XINV, st, (k_xtc<1, 0><<<grid, kXtcThreads, sm, st>>>(a)));
  return true;
}

}  // namespace vofp
