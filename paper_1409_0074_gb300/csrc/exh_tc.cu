// exh_tc.cu -- exhaustive greedy local design (Gramacy & Haaland, Sec 2.2) with
// the candidate scores of every step computed as a dense contraction on the
// tensor cores, one CTA (4 warps) per predictive location; local designs up to
// n = 64.  This is the exhaustive search of the LAGP_FP32_SCORE_TC form; the
// default LAGP_FP32_SCORE form keeps running sums instead and only adds the
// newest column of W per step (design_fp32.cu).
//
// Scoring (the factored form of Eq. alc, as in design_fp32.cu): with the
// correlation rows Kc (N' x j, Kc[r][i] = K(c_r, S_i)) and the inverse
// Cholesky factor L_j^{-1},
//     W = Kc L_j^{-T}   (row r: w_r = L_j^{-1} k_j(c_r)),
//     v_r = 1 + g - |w_r|^2,  num_r = w_r . z - K(c_r, x),  ALC_r = num_r^2 / v_r,
// z = L_j^{-1} k_j(x).  W is a tcgen05.mma kind::tf32 product of 128-candidate
// tiles (M = 128) with L_j^{-1} (N = j rounded up to 16, K = j rounded up to
// 8), 3xTF32 (hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM).  Thread t of
// the CTA owns candidate row t of a tile: it writes that row of the A operand,
// reads its row of W back from TMEM (tcgen05.ld 32x32b) and reduces v and
// num.  The block argmax (ties to the lower rank) picks the next point.
//
// FP64 state (the partitioned update in factored form, Sec 2.2): L_j^{-1} in
// global memory, grown by one row per step, and z, L^{-1} y; the predictive
// equations (Eq. predgp, preds2) at the end.  Each new row of L^{-1} is also
// written, split into TF32 hi + lo, into the B operand in shared memory.
//
// The correlation cache is kept in global memory already in the A operand's
// form: per 128-candidate tile, TF32 hi and lo blocks in the canonical K-major
// layout (XT_KMAX columns); each step writes one column (N' exponentials).
// A tile's operand then arrives by bulk copies (TMA), 16 row groups of jk/4
// core matrices each for hi and lo, and the copy of the next tile runs while
// the epilogue reads the current tile's scores from TMEM.
#include <cstdint>

#include "common.cuh"
#include "lagp_internal.h"

namespace lagp {

#define XT_THREADS 128
#define XT_KMAX 64     // largest local design on this path

struct XtParams {
  const double* X;
  const double* Y;
  int p, PP;
  const float* Xf;
  const double* xref;
  int64_t M;
  const int32_t* cand;
  int nc_max;
  const int32_t* nc_loc;
  int n0, n_max;
  const int32_t* n_loc;
  double theta, g;
  const double* theta_loc;   // per-location lengthscale [M] or null
  const double* center;
  double* mean;
  double* s2;
  int32_t* selected;
  double* tie_gap;
  int32_t* nevals;
  double* Linv;          // [slots][n_max][n_max]
  float* Kc;             // [slots][ceil(nc_max / 128)] tiles of 2 x 128 x XT_KMAX floats
  float* crow;           // [slots][nc_max][PP] the location's candidates' FP32 rows
  unsigned* status;
  unsigned* queue;       // work counter (zero at launch)
  const int32_t* order;  // item -> location, or null
  const unsigned* count; // items (device), or null (M)
  int32_t* promote;      // binary64 re-solve list, or null (promotion off)
  unsigned* promote_count;
};

#define XT_TILE_FLOATS (128 * XT_KMAX)   // one of hi / lo of a 128-candidate tile

// canonical no-swizzle K-major layout with XT_KMAX columns per row
__device__ __forceinline__ uint32_t xcanon(int row, int k) {
  return (uint32_t)((row >> 3) * ((XT_KMAX >> 2) * 128) + (k >> 2) * 128 + (row & 7) * 16 +
                    (k & 3) * 4);
}

__device__ __forceinline__ float xtf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

__device__ __forceinline__ uint64_t xdesc(uint32_t addr) {
  const uint32_t lbo = 128, sbo = (XT_KMAX / 4) * 128;
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void xmma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// 16 columns of this thread's TMEM lane
__device__ __forceinline__ void xld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// block sums of two values at once (one pass of shuffles and barriers)
// Sums over the block of FP64 terms held only by threads below `active`, to
// thread 0 (other threads keep partial values).  Only the warps holding terms
// shuffle and thread 0 adds the warp totals in warp order: bit-identical to a
// full block sum (the idle warps' totals are exact zeros) at a fraction of its
// FP64 instructions, which are scarce on this part.  Every thread must call.
__device__ __forceinline__ void xsum2_t0(double& a, double& b, int active, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int aw = min((active + 31) >> 5, XT_THREADS / 32);
  __syncthreads();   // earlier readers of red are done
  if (warp < aw) {
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { red[2 * warp] = a; red[2 * warp + 1] = b; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < aw; ++w) { ta += red[2 * w]; tb += red[2 * w + 1]; }
    a = ta;
    b = tb;
  }
}

__device__ __forceinline__ void xsum_t0(double& v, int active, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int aw = min((active + 31) >> 5, XT_THREADS / 32);
  __syncthreads();
  if (warp < aw) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < aw; ++w) t += red[w];
    v = t;
  }
}

struct XtSmem {
  static constexpr int B_BYTES = XT_KMAX * XT_KMAX * 4;   // L^{-1} rows, one of hi / lo
  static constexpr int A_BYTES = 128 * XT_KMAX * 4;       // candidate tile, one of hi / lo
  static constexpr int B_OFF = 0;
  static constexpr int A_OFF = 2 * B_BYTES;
  static constexpr int END = A_OFF + 2 * A_BYTES;         // 96 KB
};

__global__ void __launch_bounds__(XT_THREADS, 2) exh_tc_kernel(XtParams P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* Bhi = reinterpret_cast<float*>(smem + XtSmem::B_OFF);
  float* Blo = Bhi + XtSmem::B_BYTES / 4;
  float* Ahi = reinterpret_cast<float*>(smem + XtSmem::A_OFF);
  float* Alo = Ahi + XtSmem::A_BYTES / 4;
  // ld: row stride of the slot's L^{-1} (the part of a mixed launch that runs
  // here has n <= XT_KMAX); ldo: row stride of the per-step outputs
  const int p = P.p, PP = P.PP, ldo = P.n_max, nc_max = P.nc_max;
  const int ld = ldo < XT_KMAX ? ldo : XT_KMAX;
  // small state after the operands
  float* kap = reinterpret_cast<float*>(smem + XtSmem::END);          // [nc_max]
  float* zf = kap + ((nc_max + 3) & ~3);                             // [XT_KMAX]
  double* S64 = reinterpret_cast<double*>(zf + XT_KMAX);              // [XT_KMAX][p], 16B aligned
  double* kx = S64 + XT_KMAX * p;                                     // [XT_KMAX]
  double* z = kx + XT_KMAX;
  double* zy = z + XT_KMAX;
  double* kv = zy + XT_KMAX;
  double* lv = kv + XT_KMAX;
  double* ys = lv + XT_KMAX;                                          // [XT_KMAX] y of S
  double* red = ys + XT_KMAX;                                         // [8]
  float* fred = reinterpret_cast<float*>(red + 8);                    // [8]
  int* ired = reinterpret_cast<int*>(fred + 8);                       // [8]
  int* sel = ired + 8;                                                // [XT_KMAX]
  unsigned char* used = reinterpret_cast<unsigned char*>(sel + XT_KMAX);
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(used + nc_max) + 15) & ~(uintptr_t)15);   // MMA done
  uint64_t* bar_a = bar + 1;                                                  // A tile loaded
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bar + 2);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* s_item = tbase + 1;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar_a, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
        smem_u32(tbase)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tbase;
  // scratch of this CTA slot; the correlation tiles start zeroed, so that the
  // columns past j and the rows past N' that the MMAs read hold finite values
  double* Lg = P.Linv + (int64_t)blockIdx.x * ld * ld;
  const int ntc = (nc_max + 127) / 128;
  float* Kc = P.Kc + (int64_t)blockIdx.x * ntc * 2 * XT_TILE_FLOATS;
  float* crow = P.crow + (int64_t)blockIdx.x * nc_max * PP;
  for (int64_t i = tid; i < (int64_t)ntc * 2 * XT_TILE_FLOATS / 4; i += XT_THREADS)
    reinterpret_cast<float4*>(Kc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  uint32_t phase_a = 0;
  bool a_pending = false, m_pending = false;   // a bulk copy / MMA not yet waited for
  const float onepg = (float)(1.0 + P.g);
  const unsigned items = P.count ? *P.count : (unsigned)P.M;
  uint32_t phase = 0;
  bool timed_out = false;
  while (!timed_out) {
    if (tid == 0) *s_item = atomicAdd(P.queue, 1u);
    __syncthreads();
    const unsigned it = *s_item;
    __syncthreads();
    if (it >= items) break;
    const int64_t loc = P.order ? (int64_t)P.order[it] : (int64_t)it;
    const double theta = P.theta_loc ? P.theta_loc[loc] : P.theta;
    const float nit = (float)(-1.0 / theta);
    const double nit64 = -1.0 / theta;
    const int nc = P.nc_loc ? P.nc_loc[loc] : nc_max;
    const int n = P.n_loc ? P.n_loc[loc] : P.n_max;
    const int32_t* cl = P.cand + loc * nc_max;
    const double* xq = P.xref + loc * p;

    for (int i = tid; i < 2 * XtSmem::B_BYTES / 4; i += XT_THREADS) Bhi[i] = 0.f;
    // the candidates' FP32 rows, gathered once into the slot in rank order (the
    // correlation column of every step then reads them contiguously), and K(c_r, x)
    for (int r = tid; r < nc; r += XT_THREADS) {
      used[r] = 0;
      const float* c = P.Xf + (int64_t)cl[r] * PP;
      float d = 0.f;
      for (int k = 0; k < PP; k += 4) {
        const float4 v4 = *reinterpret_cast<const float4*>(c + k);
        *reinterpret_cast<float4*>(crow + (int64_t)r * PP + k) = v4;
      }
      for (int k = 0; k < p; ++k) {
        const float t = c[k] - (float)(xq[k] - P.center[k]);
        d = fmaf(t, t, d);
      }
      kap[r] = __expf(d * nit);
    }
    if (P.tie_gap) for (int i = tid; i < ldo; i += XT_THREADS) P.tie_gap[loc * ldo + i] = 0.0;
    if (P.nevals) for (int i = tid; i < ldo; i += XT_THREADS) P.nevals[loc * ldo + i] = 0;
    __syncthreads();

    int j = 0;
    bool ok = (n >= P.n0) && (n <= nc) && (n <= ld);

    // ---- append candidate rank rr: FP64 factor row, z, L^{-1}y, B row, Kc row ----
    auto add_point = [&](int rr) -> bool {
      const double* c = P.X + (int64_t)cl[rr] * p;
      if (tid < p) S64[j * p + tid] = c[tid];
      __syncthreads();
      // correlations of the new point with the design (and with x, on the idle thread j)
      for (int i = tid; i <= j; i += XT_THREADS) {
        if (i < j) {
          kv[i] = corr64_fast(S64 + i * p, S64 + j * p, p, nit64);
        } else {
          kx[j] = corr64_fast(S64 + j * p, xq, p, nit64);
          ys[j] = P.Y[cl[rr]];
          sel[j] = rr;
          used[rr] = 1;
        }
      }
      __syncthreads();
      double vv = 0.0;
      for (int i = tid; i < j; i += XT_THREADS) {
        const double* Li = Lg + (int64_t)i * ld;
        const double acc = dot64_ilp8(Li, kv, i + 1);
        lv[i] = acc;
        vv = fma(acc, acc, vv);
      }
      // thread 0 forms the pivot v = 1 + g - |l|^2 and 1 / sqrt(v)
      xsum_t0(vv, j, red);
      if (tid == 0) {
        const double v = (1.0 + P.g) - vv;
        red[0] = v;
        red[1] = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
      }
      __syncthreads();
      if (!(red[0] > 0.0)) return false;
      const double inv_d = red[1];
      for (int k = tid; k <= j; k += XT_THREADS) {
        double rk = inv_d;
        if (k < j) rk = -coldot64_ilp8(lv, Lg, ld, k, j) * inv_d;
        Lg[(int64_t)j * ld + k] = rk;
        const float h = xtf32((float)rk);
        const uint32_t off = xcanon(j, k) >> 2;
        Bhi[off] = h;
        Blo[off] = xtf32((float)(rk - (double)h));
      }
      __syncthreads();
      double zz = 0.0, zyy = 0.0;
      for (int k = tid; k <= j; k += XT_THREADS) {
        const double rk = Lg[(int64_t)j * ld + k];
        zz = fma(rk, kx[k], zz);
        zyy = fma(rk, ys[k], zyy);
      }
      xsum2_t0(zz, zyy, j + 1, red);
      if (tid == 0) {
        z[j] = zz;
        zy[j] = zyy;
        zf[j] = (float)zz;
      }
      // correlation cache column j: K(c_r, S_j) for every candidate, as A operand
      // (TF32 hi / lo) of its tile; then visible to the bulk copies
      const float* sj = crow + (int64_t)rr * PP;
      for (int q = tid; q < nc; q += XT_THREADS) {
        const float kv = __expf(sqdist_row32(crow + (int64_t)q * PP, sj, PP) * nit);
        const float h = xtf32(kv);
        float* tile = Kc + (int64_t)(q >> 7) * 2 * XT_TILE_FLOATS;
        const uint32_t off = xcanon(q & 127, j) >> 2;
        tile[off] = h;
        tile[XT_TILE_FLOATS + off] = xtf32(kv - h);
      }
      // this step's generic writes (the B row in shared memory, the cache column
      // in global memory) become visible to the tensor core and the bulk copies
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
      __syncthreads();
      ++j;
      return true;
    };

    for (int rr = 0; rr < P.n0 && ok; ++rr) ok = add_point(rr);

    for (int step = P.n0; step < n && ok; ++step) {
      const int jn = (j + 15) & ~15;       // N of the MMA
      const int jk = (j + 7) & ~7;         // K of the MMA
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(jn >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      float best = -1.f, second = -1.f;
      int bi = -1;
      // A tile t: 16 row groups x (jk / 4) core matrices of hi and of lo, one bulk
      // copy each, issued by the 32 lanes of warp 0 (lane l: row group l % 16,
      // hi for l < 16, lo above)
      const uint32_t rg_bytes = (uint32_t)jk * 32u;
      auto load_a = [&](int t) {
        a_pending = true;
        if (warp == 0) {
          if (lane == 0) mbar_expect_tx(bar_a, 32u * rg_bytes);
          __syncwarp();
          const int rg = lane & 15, part = lane >> 4;
          const float* src = Kc + (int64_t)t * 2 * XT_TILE_FLOATS + part * XT_TILE_FLOATS + rg * (XT_KMAX / 4) * 32;
          float* dst = (part ? Alo : Ahi) + rg * (XT_KMAX / 4) * 32;
          bulk_g2s(dst, src, rg_bytes, bar_a);
        }
      };
      const int ntile = (nc + 127) >> 7;
      load_a(0);
      for (int t = 0; t < ntile; ++t) {
        const int base = t << 7;
        const int r = base + tid;
        const bool live = r < nc;
        // tile t's operand in shared memory, then its MMAs
        bool got = mbar_wait(bar_a, phase_a);
        if (!__syncthreads_and(got)) {
          if (tid == 0) atomicOr(P.status, LAGP_DEV_TIMEOUT);
          ok = false;
          timed_out = true;
          break;
        }
        phase_a ^= 1u;
        a_pending = false;
        m_pending = true;
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo);
          const uint32_t bh = smem_u32(Bhi), bl = smem_u32(Blo);
          for (int ks = 0; ks < jk / 8; ++ks) {
            const uint32_t ko = ks * 256;
            xmma(taddr, xdesc(ah + ko), xdesc(bh + ko), idesc, ks > 0 ? 1u : 0u);
            xmma(taddr, xdesc(ah + ko), xdesc(bl + ko), idesc, 1u);
            xmma(taddr, xdesc(al + ko), xdesc(bh + ko), idesc, 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(bar))
                       : "memory");
        }
        bool done = mbar_wait(bar, phase);
        if (!__syncthreads_and(done)) {
          if (tid == 0) atomicOr(P.status, LAGP_DEV_TIMEOUT);
          ok = false;
          timed_out = true;
          break;
        }
        phase ^= 1u;
        m_pending = false;
        // the MMAs have read the A buffer: the next tile's copy overlaps the epilogue
        if (t + 1 < ntile) load_a(t + 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: row tid of W
        float vs = 0.f, ns = 0.f;
        const uint32_t row = taddr + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < jn; c0 += 16) {
          float w[16];
          xld16(row + c0, w);
  #pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int i = c0 + u;
            const float wi = i < j ? w[u] : 0.f;
            vs = fmaf(wi, wi, vs);
            ns = fmaf(wi, i < j ? zf[i] : 0.f, ns);
          }
        }
        if (live && !used[r]) {
          const float v = onepg - vs;
          const float num = ns - kap[r];
          const float alc = v > 0.f ? num * num / v : 0.f;
          if (alc > best) { second = best; best = alc; bi = r; }
          else if (alc > second) second = alc;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
      }
      if (!ok) break;
      // block argmax, ties to the lower rank; the second best for the gap
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const float os = __shfl_xor_sync(0xffffffffu, second, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) {
          second = fmaxf(best, os); best = ob; bi = oi;
        } else {
          second = fmaxf(second, ob);
        }
      }
      if (lane == 0) { fred[2 * warp] = best; fred[2 * warp + 1] = second; ired[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        float b = fred[0], s = fred[1];
        int ii = ired[0];
        for (int w = 1; w < XT_THREADS / 32; ++w) {
          const float ob = fred[2 * w], os = fred[2 * w + 1];
          const int oi = ired[w];
          if (ob > b || (ob == b && oi >= 0 && (ii < 0 || oi < ii))) { s = fmaxf(b, os); b = ob; ii = oi; }
          else s = fmaxf(s, ob);
        }
        ired[4] = ii;
        if (P.tie_gap) P.tie_gap[loc * ldo + (step - P.n0)] = (b > 0.f && s >= 0.f) ? (double)((b - s) / b) : 0.0;
      }
      __syncthreads();
      const int pick = ired[4];
      ok = (pick >= 0) && add_point(pick);
    }

    if (ok) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int i = tid; i < j; i += XT_THREADS) {
        a = fma(z[i], zy[i], a);
        b = fma(zy[i], zy[i], b);
        c = fma(z[i], z[i], c);
      }
      xsum2_t0(a, b, j, red);
      xsum_t0(c, j, red + 4);
      if (tid == 0) {
        P.mean[loc] = a;
        P.s2[loc] = b * ((1.0 + P.g) - c) / (double)j;
      }
    } else if (tid == 0) {
      P.mean[loc] = __longlong_as_double(0x7ff8000000000000ll);
      P.s2[loc] = __longlong_as_double(0x7ff8000000000000ll);
      atomicOr(P.status, LAGP_DEV_BAD_UPDATE);
    }
    if (P.selected)
      for (int i = tid; i < ldo; i += XT_THREADS) P.selected[loc * ldo + i] = (i < j) ? cl[sel[i]] : -1;
    if (P.promote && tid == 0) {
      // smallest binary64 pivot v of the design: the factor's diagonal holds
      // 1 / sqrt(v); a failed update promotes the location
      double vm = ok ? INFINITY : -1.0;
      for (int i = 0; i < j; ++i) {
        const double dg = Lg[(int64_t)i * ld + i];
        vm = fmin(vm, 1.0 / (dg * dg));
      }
      promote_location(P.promote, P.promote_count, loc, vm);
    }
  }
  // after a timeout: wait (bounded) for the copy or MMAs still in flight
  if (a_pending) mbar_wait(bar_a, phase_a);
  if (m_pending) mbar_wait(bar, phase);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(taddr));
  }
}

int exh_tc_max_n() { return XT_KMAX; }

size_t exh_tc_cache_floats(int nc_max) { return (size_t)((nc_max + 127) / 128) * 2 * XT_TILE_FLOATS; }

cudaError_t launch_exh_tc(const DesignArgs& a, cudaStream_t s) {
  XtParams P;
  P.X = a.X; P.Y = a.Y; P.p = a.p; P.PP = a.PP; P.Xf = a.ws->Xf; P.xref = a.xref; P.M = a.M;
  P.cand = a.cand; P.nc_max = a.nc_max; P.nc_loc = a.nc_loc; P.n0 = a.n0; P.n_max = a.n_max;
  P.n_loc = a.n_loc; P.theta = a.theta; P.theta_loc = a.theta_loc; P.g = a.g; P.center = a.ws->center; P.mean = a.mean;
  P.s2 = a.s2; P.selected = a.selected; P.tie_gap = a.tie_gap; P.nevals = a.nevals;
  P.Linv = a.ws->state64; P.Kc = a.ws->state32; P.status = a.ws->status;
  P.queue = a.ws->queue + 1; P.order = a.order; P.count = a.count;
  P.crow = a.ws->crow;
  P.promote = a.promote ? a.ws->promote : nullptr;
  P.promote_count = a.ws->status + 1;
  const size_t small = (size_t)((a.nc_max + 3) & ~3) * 4 + XT_KMAX * 4 + (size_t)XT_KMAX * a.p * 8 +
                       6 * XT_KMAX * 8 + 8 * 8 + 8 * 4 + 8 * 4 + XT_KMAX * 4 + a.nc_max + 96;
  const size_t sm = 1024 + XtSmem::END + small;
  cudaError_t err =
      cudaFuncSetAttribute(exh_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (err != cudaSuccess) return err;
  const int64_t grid = persistent_grid(exh_tc_kernel, XT_THREADS, sm, a.M, exh_slots(a.ws->chunk), 1,
                                       a.tune.exh_occ);
  if (grid < 0) return cudaErrorInvalidValue;
  if ((err = cudaMemsetAsync(P.queue, 0, sizeof(unsigned), s)) != cudaSuccess) return err;
  prof_begin("exh_tc", s);
  exh_tc_kernel<<<(unsigned)grid, XT_THREADS, sm, s>>>(P);
  prof_end(s);
  return cudaGetLastError();
}

}  // namespace lagp
