// ray32.cu -- ray search (Gramacy & Haaland, Sec 4) with FP32 scoring and an
// FP64 factor update, one warp per predictive location.
//
// Lane layout.  With R rays padded to RP (a power of two) and G = 32 / RP,
// lane = r * G + q works for ray r on every G-th row (q, q+G, ...) of each
// ALC evaluation.  All rays of a location advance together: a round evaluates
// ALC once for every ray still searching (its s = 0 point, its first golden-
// section point, or its next Brent trial point), then each ray updates its
// own Brent (1973) state.  A ray that has converged idles until the last ray
// of its location is done.  The warp never meets a CTA-wide barrier.
//
// Scoring (FP32, through the inverse Cholesky factor, as in design_fp32.cu):
//   kz_k = exp(-|S_k - z|^2 / theta),  w = L^{-1} kz,
//   ALC(z) = (w . (L^{-1} k(x)) - K(z, x))^2 / (1 + g - |w|^2).
// A ray is a straight segment z(s) = a + s d (Sec 4), so every correlation
// exponent along it is a quadratic in s:
//   -log2(e) |z(s) - S_k|^2 / theta = c_k + s (b_k + s gam),
//   c_k = nu |a - S_k|^2,  b_k = 2 nu d . (a - S_k),  gam = nu |d|^2,
// with nu = -log2(e) / theta.  c_k and b_k are formed once per greedy step;
// an evaluation then costs two FMAs and one base-2 exponential per design
// point instead of a p-coordinate distance.
// L^{-1} (FP32) sits in shared memory as lower-triangular rows padded with
// zeros to a multiple of 4, so every row is read as float4s.
// The factor itself grows in FP64 (the partitioned update in factored form,
// Sec 2.2) in global memory, packed lower-triangular.
//
// Scheduling.  The kernel is persistent: each warp takes the next location
// from a device work counter until the queue is empty, optionally through a
// permutation (largest local designs first, so that uneven n does not leave a
// long tail).  The FP64 scratch belongs to the warp slot, not the location, so
// it stays within a few hundred MB (L2-resident for moderate grids) however
// many locations a launch covers.
#include <cstdint>
#include <cstring>

#include "common.cuh"
#include "kdtree.cuh"
#include "lagp_internal.h"
#include "launch_plan.h"
#include "ray32_layout.h"

namespace lagp {

#define RAY_MAX_ROUNDS 1100         // bound on evaluation rounds per step

struct RayParams {
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
  const double* theta_loc; // per-location lengthscale [M] or null
  int R;
  const double* lo;
  const double* hi;
  const double* center;
  double* mean;
  double* s2;
  int32_t* selected;
  double* tie_gap;
  int32_t* nevals;
  double* g64;          // per warp slot: packed L^{-1} (n(n+1)/2) then z, L^{-1} y (n each)
  int64_t g64_stride;
  unsigned* status;
  unsigned* queue;      // work counter (zero at launch)
  const int32_t* order; // item -> location, or null (identity)
  const unsigned* count;// number of items (device), or null (M)
  int full;             // snap over all of X_N through the k-d tree
  KdView<float> kd;     // the tree in centred FP32 coordinates (full scope)
  int32_t* promote;     // binary64 re-solve list, or null (promotion off)
  unsigned* promote_count;
};

// 2^x by the hardware's base-2 exponential (PTX ex2.approx); the scoring
// correlations use exp(-d / theta) = 2^(-d log2(e) / theta), with log2(e) / theta
// formed once per location
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct Brent {
  float a, b, x, w, v, fx, fw, fv, d, e;
};

// Brent (1973) fmin on [0,1]: from the current state, either report
// convergence (false) or produce the next trial point u (true).  Same
// constants as the FP64 path: tol = 2^-13, sqrt(eps) = 2^-26.
__device__ __forceinline__ bool brent_next(Brent& s, float* u_out) {
  const float tol3 = 0x1p-13f / 3.f, sqrt_eps = 0x1p-26f;
  const float golden = 0.381966011250105151795f;
  const float m = 0.5f * (s.a + s.b);
  const float tol1 = sqrt_eps * fabsf(s.x) + tol3;
  const float tol2 = 2.f * tol1;
  if (fabsf(s.x - m) <= tol2 - 0.5f * (s.b - s.a)) return false;
  bool golden_step = true;
  if (fabsf(s.e) > tol1) {
    float r = (s.x - s.w) * (s.fx - s.fv);
    float q = (s.x - s.v) * (s.fx - s.fw);
    float pn = (s.x - s.v) * q - (s.x - s.w) * r;
    q = 2.f * (q - r);
    if (q > 0.f) pn = -pn; else q = -q;
    const float e_prev = s.e;
    s.e = s.d;
    if (fabsf(pn) < fabsf(0.5f * q * e_prev) && pn > q * (s.a - s.x) && pn < q * (s.b - s.x)) {
      s.d = pn / q;
      const float u_try = s.x + s.d;
      if (u_try - s.a < tol2 || s.b - u_try < tol2) s.d = (m - s.x >= 0.f) ? tol1 : -tol1;
      golden_step = false;
    }
  }
  if (golden_step) {
    s.e = (s.x < m) ? (s.b - s.x) : (s.a - s.x);
    s.d = golden * s.e;
  }
  float u;
  if (fabsf(s.d) >= tol1) u = s.x + s.d;
  else if (s.d >= 0.f) u = s.x + tol1;
  else u = s.x - tol1;
  *u_out = u;
  return true;
}

__device__ __forceinline__ void brent_take(Brent& s, float u, float fu) {
  if (fu <= s.fx) {
    if (u < s.x) s.b = s.x; else s.a = s.x;
    s.v = s.w; s.fv = s.fw;
    s.w = s.x; s.fw = s.fx;
    s.x = u; s.fx = fu;
  } else {
    if (u < s.x) s.a = u; else s.b = u;
    if (fu <= s.fw || s.w == s.x) {
      s.v = s.w; s.fv = s.fw;
      s.w = u; s.fw = fu;
    } else if (fu <= s.fv || s.v == s.x || s.v == s.w) {
      s.v = u; s.fv = fu;
    }
  }
}

__device__ __forceinline__ double warp_sum64(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

enum { PH_ALC0 = 0, PH_FIRST = 1, PH_ITER = 2, PH_DONE = 3 };

// One location, by one warp, in the warp's shared-memory region and FP64 slot.
template <int RP, int PP>
__device__ __forceinline__ void ray32_location(const RayParams& P, const int64_t loc, float* base,
                                               double* Lg) {
  constexpr int G = 32 / RP;
  const int lane = threadIdx.x & 31;
  const int p = P.p, ldn = P.n_max, R = P.R;
  const int nc = P.nc_loc ? P.nc_loc[loc] : P.nc_max;
  const int n = P.n_loc ? P.n_loc[loc] : P.n_max;
  const int32_t* cl = P.cand + loc * P.nc_max;
  const WarpLayout lay = warp_layout(ldn, PP, RP, P.nc_max);
  float* Lf = base + lay.lf;
  float* kzb = base + lay.kz;
  float* zf = base + lay.zf;
  float* Cb = base + lay.cb;          // c_k of ray r at Cb[r * KP + k]
  float* Bb = Cb + RP * kz_ld(ldn);   // b_k of ray r at Bb[r * KP + k]
  float* taub = base + lay.tau;
  float* xf = base + lay.x;
  float* lof = xf + PP;
  float* hif = lof + PP;
  float* xs = hif + PP;
  int* gsel = reinterpret_cast<int*>(base + lay.gsel);    // design indices
  int* stk = reinterpret_cast<int*>(base + lay.stk);
  float* bnd = base + lay.bnd;
  int* starts = reinterpret_cast<int*>(base + lay.starts);
  uint32_t* mask = reinterpret_cast<uint32_t*>(base + lay.mask);     // selected candidates
  uint32_t* smask = reinterpret_cast<uint32_t*>(base + lay.smask);   // this step's ray starts
  double* vmin = reinterpret_cast<double*>(base + lay.vm);
  const int KP = kz_ld(ldn);

  double* z64 = Lg + tri(ldn);
  double* zy64 = z64 + ldn;
  const double* xq = P.xref + loc * p;

  const double theta = P.theta_loc ? P.theta_loc[loc] : P.theta;
  // -log2(e) / theta: the correlations' exponentials as one base-2 exponential
  const float nit2 = (float)(-1.4426950408889634 / theta);
  const double nit64 = -1.0 / theta;
  const float onepg = (float)(1.0 + P.g);

  for (int i = lane; i < roff(ldn); i += 32) Lf[i] = 0.f;
  for (int i = lane; i < RP * KP; i += 32) kzb[i] = 0.f;
  for (int i = lane; i < (P.nc_max + 31) / 32; i += 32) { mask[i] = 0u; smask[i] = 0u; }
  if (lane < PP) {
    const bool in = lane < p;
    xf[lane] = in ? (float)(xq[lane] - P.center[lane]) : 0.f;
    lof[lane] = in ? (float)(P.lo[lane] - P.center[lane]) : 0.f;
    hif[lane] = in ? (float)(P.hi[lane] - P.center[lane]) : 0.f;
  }
  if (P.tie_gap) for (int i = lane; i < ldn; i += 32) P.tie_gap[loc * ldn + i] = 0.0;
  if (P.nevals) for (int i = lane; i < ldn; i += 32) P.nevals[loc * ldn + i] = 0;
  __syncwarp();

  int j = 0;
  bool ok = (n >= P.n0) && (n <= nc) && (n <= ldn);
  if (lane == 0) *vmin = INFINITY;

  // ---- append design point gi (candidate rank rr, or -1) (FP64 factor row) ----
  // k_j(x_new) and l = L_j^{-1} k_j(x_new) live in shared memory, in the
  // coefficient region, which no evaluation uses while a point is appended
  double* kvs = reinterpret_cast<double*>(Cb);
  double* ls = kvs + ldn;
  auto add_point = [&](int gi, int rr) -> bool {
    const double* c64 = P.X + (int64_t)gi * p;
    double kxj = 0.0;   // K(x_new, x), on lane j mod 32
    for (int i = lane; i <= j; i += 32) {
      if (i < j) kvs[i] = corr64_fast(P.X + (int64_t)gsel[i] * p, c64, p, nit64);
      else kxj = corr64_fast(c64, xq, p, nit64);
    }
    kxj = __shfl_sync(0xffffffffu, kxj, j & 31);
    __syncwarp();
    // l = L_j^{-1} k_j(x_new); v = 1 + g - |l|^2, d = sqrt(v), and by forward
    // substitution z_j = (K(x_new, x) - l . z) / d, (L^{-1} y)_j =
    // (y_new - l . L^{-1} y) / d, all from one pass.  A warp's FP64
    // instruction costs the same whatever its active lanes, so every lane
    // evaluates the scalar tail.
    double vv = 0.0, lz = 0.0, lzy = 0.0;
    for (int i = lane; i < j; i += 32) {
      const double acc = dot64_ilp(Lg + tri(i), kvs, i + 1);
      ls[i] = acc;
      vv = fma(acc, acc, vv);
      lz = fma(acc, z64[i], lz);
      lzy = fma(acc, zy64[i], lzy);
    }
    vv = warp_sum64(vv);
    lz = warp_sum64(lz);
    lzy = warp_sum64(lzy);
    __syncwarp();
    const double v = (1.0 + P.g) - vv;
    if (lane == 0) *vmin = v > 0.0 ? fmin(*vmin, v) : -1.0;
    if (!(v > 0.0)) return false;
    const double inv_d = rsqrt(v);
    double* Lj = Lg + tri(j);
    float* Lfj = Lf + roff(j);
    for (int k = lane; k < j; k += 32) {
      double a0 = 0.0, a1 = 0.0;
      int i = k;
      for (; i + 1 < j; i += 2) {
        a0 = fma(ls[i], Lg[tri(i) + k], a0);
        a1 = fma(ls[i + 1], Lg[tri(i + 1) + k], a1);
      }
      if (i < j) a0 = fma(ls[i], Lg[tri(i) + k], a0);
      const double rk = -(a0 + a1) * inv_d;
      Lj[k] = rk;
      Lfj[k] = (float)rk;
    }
    if (lane == 0) {
      Lj[j] = inv_d;
      Lfj[j] = (float)inv_d;
      gsel[j] = gi;
      if (rr >= 0) mask[rr >> 5] |= 1u << (rr & 31);
      const double zj = (kxj - lz) * inv_d;
      z64[j] = zj;
      zy64[j] = (P.Y[gi] - lzy) * inv_d;
      zf[j] = (float)zj;
    }
    __syncwarp();
    ++j;
    return true;
  };

  for (int rr = 0; rr < P.n0 && ok; ++rr) ok = add_point(cl[rr], rr);

  const int r = lane / G, q = lane % G;
  for (int step = P.n0; step < n && ok; ++step) {
    // ---- ray starts: unselected candidates of rank k0, k0+1, ... (mod |U|) ----
    // lane l owns mask words l, l + 32, ...; a warp scan of their unselected
    // counts locates the word holding each target rank
    {
      const int nU = nc - j;
      const int k0 = ray_offset(j, P.n0);
      const int nw = (nc + 31) >> 5;
      int seen = 0;
      for (int w0 = 0; w0 < nw; w0 += 32) {
        const int wd = w0 + lane;
        uint32_t un = 0u;
        if (wd < nw) {
          const int hi = min(32, nc - wd * 32);
          un = ~mask[wd] & (hi == 32 ? 0xffffffffu : ((1u << hi) - 1u));
        }
        const int c = __popc(un);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int first = seen + incl - c;
        for (int t = 0; t < R; ++t) {
          const int target = (k0 + t) % nU;
          if (target >= first && target < first + c) {
            uint32_t u = un;
            for (int q2 = target - first; q2 > 0; --q2) u &= u - 1u;   // drop lower bits
            const int rr = wd * 32 + __ffs(u) - 1;
            starts[t] = rr;
            smask[wd] |= 1u << (rr & 31);   // words are lane-owned: no race
          }
        }
        seen += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncwarp();
    // ---- segments (FP32): end = A + tau * 10 (A - x), cut at the design's box ----
    const bool ray_live = r < R;
    float len2 = 0.f, gam = 0.f, cx = 0.f, bx = 0.f;
    if (ray_live) {
      const float* a = P.Xf + (int64_t)cl[starts[r]] * PP;
      float tau = 1.f;
      for (int k = 0; k < p; ++k) {
        const float dk = 10.f * (a[k] - xf[k]);
        if (dk > 0.f) tau = fminf(tau, (hif[k] - a[k]) / dk);
        else if (dk < 0.f) tau = fminf(tau, (lof[k] - a[k]) / dk);
      }
      tau = fmaxf(tau, 0.f);
      if (q == 0) taub[r] = tau;
      float av[PP], dv[PP];
      float cxs = 0.f, bxs = 0.f;
#pragma unroll
      for (int k = 0; k < PP; ++k) {
        const float ak = a[k];
        const float ek = fmaf(tau, 10.f * (ak - xf[k]), ak);
        av[k] = ak;
        dv[k] = ek - ak;
        len2 = fmaf(dv[k], dv[k], len2);
        const float tx = ak - xf[k];
        cxs = fmaf(tx, tx, cxs);
        bxs = fmaf(dv[k], tx, bxs);
      }
      // the exponents of K(z(s), x) and of K(z(s), S_k), k < j, as
      // quadratics in s; quads past j get c = -inf (a zero correlation)
      gam = nit2 * len2;
      cx = nit2 * cxs;
      bx = 2.f * nit2 * bxs;
      float* cr = Cb + r * KP;
      float* br = Bb + r * KP;
      for (int k4 = q; 4 * k4 < j; k4 += G) {
        float cq[4], bq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = 4 * k4 + u;
          cq[u] = -__int_as_float(0x7f800000);
          bq[u] = 0.f;
          if (k < j) {
            const float* sk = P.Xf + (int64_t)gsel[k] * PP;
            float cs = 0.f, bs = 0.f;
#pragma unroll
            for (int c = 0; c < PP; c += 4) {
              const float4 s4 = *reinterpret_cast<const float4*>(sk + c);
              const float t0 = av[c] - s4.x, t1 = av[c + 1] - s4.y;
              const float t2 = av[c + 2] - s4.z, t3 = av[c + 3] - s4.w;
              cs = fmaf(t0, t0, cs); cs = fmaf(t1, t1, cs);
              cs = fmaf(t2, t2, cs); cs = fmaf(t3, t3, cs);
              bs = fmaf(dv[c], t0, bs); bs = fmaf(dv[c + 1], t1, bs);
              bs = fmaf(dv[c + 2], t2, bs); bs = fmaf(dv[c + 3], t3, bs);
            }
            cq[u] = nit2 * cs;
            bq[u] = 2.f * nit2 * bs;
          }
        }
        *reinterpret_cast<float4*>(cr + 4 * k4) = make_float4(cq[0], cq[1], cq[2], cq[3]);
        *reinterpret_cast<float4*>(br + 4 * k4) = make_float4(bq[0], bq[1], bq[2], bq[3]);
      }
    }
    __syncwarp();

    // ---- lockstep Brent over the rays ----
    int phase = ray_live ? PH_ALC0 : PH_DONE;
    float s_eval = 0.f, alc0 = 0.f, s_star = 0.f, alc_star = 0.f;
    int evals = 0;
    Brent st;
    st.a = 0.f; st.b = 1.f; st.x = st.w = st.v = 0.f; st.fx = st.fw = st.fv = 0.f;
    st.d = 0.f; st.e = 0.f;
    for (int round = 0; round < RAY_MAX_ROUNDS; ++round) {
      const bool active = phase != PH_DONE;
      if (!__any_sync(0xffffffffu, active)) break;
      float* kzr = kzb + r * KP;
      if (active) {
        // kz over quads of design points, two exponents per paired FMA
        const float* cr = Cb + r * KP;
        const float* br = Bb + r * KP;
        const float2 s2v = make_float2(s_eval, s_eval), g2 = make_float2(gam, gam);
        for (int k4 = q; 4 * k4 < j; k4 += G) {
          const float4 c4 = *reinterpret_cast<const float4*>(cr + 4 * k4);
          const float4 b4 = *reinterpret_cast<const float4*>(br + 4 * k4);
          const float2 t01 = __ffma2_rn(s2v, g2, make_float2(b4.x, b4.y));
          const float2 t23 = __ffma2_rn(s2v, g2, make_float2(b4.z, b4.w));
          const float2 e01 = __ffma2_rn(s2v, t01, make_float2(c4.x, c4.y));
          const float2 e23 = __ffma2_rn(s2v, t23, make_float2(c4.z, c4.w));
          *reinterpret_cast<float4*>(kzr + 4 * k4) =
              make_float4(ex2_approx(e01.x), ex2_approx(e01.y), ex2_approx(e23.x), ex2_approx(e23.y));
        }
      }
      __syncwarp();
      float vs = 0.f, ns = 0.f;
      if (active) {
        for (int i = q; i < j; i += G) {
          const float* Li = Lf + roff(i);
          const int len = (i + 4) & ~3;
          // two accumulators (elements 0, 2 and 1, 3 of each quad) in one
          // paired FMA per element pair
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll 2
          for (int k = 0; k < len; k += 4) {
            const float4 l4 = *reinterpret_cast<const float4*>(Li + k);
            const float4 k4 = *reinterpret_cast<const float4*>(kzr + k);
            acc = __ffma2_rn(make_float2(l4.x, l4.y), make_float2(k4.x, k4.y), acc);
            acc = __ffma2_rn(make_float2(l4.z, l4.w), make_float2(k4.z, k4.w), acc);
          }
          const float w = acc.x + acc.y;
          vs = fmaf(w, w, vs);
          ns = fmaf(w, zf[i], ns);
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        vs += __shfl_xor_sync(0xffffffffu, vs, o);
        ns += __shfl_xor_sync(0xffffffffu, ns, o);
      }
      float val = 0.f;
      if (active) {
        const float v = onepg - vs;
        const float num = ns - ex2_approx(fmaf(s_eval, fmaf(s_eval, gam, bx), cx));
        val = v > 0.f ? num * num / v : 0.f;
      }
      __syncwarp();
      if (active) {
        ++evals;
        bool more = false;
        float u = 0.f;
        if (phase == PH_ALC0) {
          alc0 = val;
          if (len2 > 0.f) { phase = PH_FIRST; s_eval = 0.381966011250105151795f; more = true; }
        } else if (phase == PH_FIRST) {
          st.x = st.w = st.v = s_eval;
          st.fx = st.fw = st.fv = -val;
          more = brent_next(st, &u);
          if (more) { s_eval = u; phase = PH_ITER; }
        } else {
          brent_take(st, s_eval, -val);
          more = brent_next(st, &u);
          if (more) s_eval = u;
        }
        if (more && evals > 1000) more = false;
        if (!more) {
          if (phase == PH_ALC0 || alc0 >= -st.fx) { s_star = 0.f; alc_star = alc0; }
          else { s_star = st.x; alc_star = -st.fx; }
          phase = PH_DONE;
        }
      }
    }
    // ---- best ray, its continuous point x* ----
    float best = -1.f, second = -1.f;
    int ib = 0, ev = 0;
    for (int rr = 0; rr < R; ++rr) {
      const float a_r = __shfl_sync(0xffffffffu, alc_star, rr * G);
      ev += __shfl_sync(0xffffffffu, evals, rr * G);
      if (a_r > best) { second = best; best = a_r; ib = rr; }
      else if (a_r > second) second = a_r;
    }
    const float sb = __shfl_sync(0xffffffffu, s_star, ib * G);
    if (lane < PP) {
      // the best ray's segment again, in the same operations as above
      const float ak = P.Xf[(int64_t)cl[starts[ib]] * PP + lane];
      const float ek = fmaf(taub[ib], 10.f * (ak - xf[lane]), ak);
      xs[lane] = fmaf(sb, ek - ak, ak);
    }
    __syncwarp();
    // ---- snap: nearest allowed unselected candidate (ties to the lower rank) ----
    // allowed: not one of this step's ray starts unless it coincides with x*;
    // if no candidate is allowed, the nearest unselected one (second pair)
    float2 nx[PP / 2];
#pragma unroll
    for (int k = 0; k < PP; k += 2) nx[k / 2] = make_float2(-xs[k], -xs[k + 1]);
    float bd0 = __int_as_float(0x7f800000), bd1 = bd0;
    int bi0 = 0x7fffffff, bi1 = 0x7fffffff;
    int pick_g = -1;                  // the full scope's pick (design index)
    if (P.full) {
      // nearest point of X_N outside the design; the step's starts are
      // forbidden unless they equal x*
      const KdView<float>& V = P.kd;
      auto excluded = [&](int32_t gi, int64_t pos, bool allow_starts) -> bool {
        for (int i = 0; i < j; ++i) if (gsel[i] == gi) return true;
        if (allow_starts) return false;
        for (int t = 0; t < R; ++t) {
          if (cl[starts[t]] != gi) continue;
          for (int k = 0; k < p; ++k) if (V.pts[pos * PP + k] != xs[k]) return true;
        }
        return false;
      };
      auto dist = [&](int64_t pos, int32_t) -> float {
        const float* c = V.pts + pos * PP;
        float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < PP; k += 4) {
          const float4 cv = *reinterpret_cast<const float4*>(c + k);
          const float2 t01 = __fadd2_rn(make_float2(cv.x, cv.y), nx[k / 2]);
          const float2 t23 = __fadd2_rn(make_float2(cv.z, cv.w), nx[k / 2 + 1]);
          d2 = __ffma2_rn(t01, t01, d2);
          d2 = __ffma2_rn(t23, t23, d2);
        }
        return d2.x + d2.y;
      };
      auto distx = [&](int64_t pos, int32_t) -> float {
        const float* c = V.pts + pos * PP;
        float d = 0.f;
        for (int k = 0; k < PP; ++k) { const float t = c[k] - xf[k]; d = fmaf(t, t, d); }
        return d;
      };
      const KdTop<float> b = kd_nearest<float>(V, xs, 1e-5f, stk, bnd, excluded, dist, distx);
      pick_g = b.i1;
    } else {
      // When the best ray kept s = 0, x* is its start, an allowed candidate at
      // distance 0; only a lower-ranked candidate at distance 0 (the same FP32
      // coordinates) could take it, so the scan stops at the start's rank.
      const int lim = (sb == 0.f) ? starts[ib] + 1 : nc;
      const int nw = (lim + 31) >> 5;
      const uint32_t bit = 1u << lane;
#pragma unroll 1
      for (int wd = 0; wd < nw; ++wd) {
        const int rr = wd * 32 + lane;
        if (rr < lim && !(mask[wd] & bit)) {
          const float* c = P.Xf + (int64_t)cl[rr] * PP;
          float2 d2 = make_float2(0.f, 0.f);
          bool same = true;                   // every coordinate equal to x*'s
#pragma unroll
          for (int k = 0; k < PP; k += 4) {
            const float4 cv = *reinterpret_cast<const float4*>(c + k);
            const float2 t01 = __fadd2_rn(make_float2(cv.x, cv.y), nx[k / 2]);
            const float2 t23 = __fadd2_rn(make_float2(cv.z, cv.w), nx[k / 2 + 1]);
            same &= (t01.x == 0.f) & (t01.y == 0.f) & (t23.x == 0.f) & (t23.y == 0.f);
            d2 = __ffma2_rn(t01, t01, d2);
            d2 = __ffma2_rn(t23, t23, d2);
          }
          const float d = d2.x + d2.y;
          if (d < bd1) { bd1 = d; bi1 = rr; }
          if ((same || !(smask[wd] & bit)) && d < bd0) { bd0 = d; bi0 = rr; }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od0 = __shfl_xor_sync(0xffffffffu, bd0, o);
      const int oi0 = __shfl_xor_sync(0xffffffffu, bi0, o);
      const float od1 = __shfl_xor_sync(0xffffffffu, bd1, o);
      const int oi1 = __shfl_xor_sync(0xffffffffu, bi1, o);
      if (od0 < bd0 || (od0 == bd0 && oi0 < bi0)) { bd0 = od0; bi0 = oi0; }
      if (od1 < bd1 || (od1 == bd1 && oi1 < bi1)) { bd1 = od1; bi1 = oi1; }
    }
    int pick = -1;
    if (!P.full) {
      pick = bi0 != 0x7fffffff ? bi0 : (bi1 != 0x7fffffff ? bi1 : -1);
      pick_g = pick >= 0 ? cl[pick] : -1;
    } else if (pick_g >= 0) {
      // its candidate rank, when it is one
      int rk = 0x7fffffff;
      for (int rr = lane; rr < nc; rr += 32) if (cl[rr] == pick_g) rk = min(rk, rr);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rk = min(rk, __shfl_xor_sync(0xffffffffu, rk, o));
      pick = rk != 0x7fffffff ? rk : -1;
    }
    __syncwarp();
    if (lane < R) smask[starts[lane] >> 5] = 0u;
    if (lane == 0) {
      if (P.tie_gap) P.tie_gap[loc * ldn + (step - P.n0)] =
          (best > 0.f && R > 1) ? (double)((best - second) / best) : 0.0;
      if (P.nevals) P.nevals[loc * ldn + (step - P.n0)] = ev;
    }
    ok = (pick_g >= 0) && add_point(pick_g, pick);
  }

  if (ok) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = lane; i < j; i += 32) {
      a = fma(z64[i], zy64[i], a);
      b = fma(zy64[i], zy64[i], b);
      c = fma(z64[i], z64[i], c);
    }
    a = warp_sum64(a);
    b = warp_sum64(b);
    c = warp_sum64(c);
    if (lane == 0) {
      P.mean[loc] = a;
      P.s2[loc] = b * ((1.0 + P.g) - c) / (double)j;
    }
  } else if (lane == 0) {
    P.mean[loc] = __longlong_as_double(0x7ff8000000000000ll);
    P.s2[loc] = __longlong_as_double(0x7ff8000000000000ll);
    atomicOr(P.status, LAGP_DEV_BAD_UPDATE);
  }
  if (P.selected)
    for (int i = lane; i < ldn; i += 32) P.selected[loc * ldn + i] = (i < j) ? gsel[i] : -1;
  if (lane == 0) promote_location(P.promote, P.promote_count, loc, *vmin);
}

// at least 20 resident warps per SM (at most 102 registers per thread)
template <int RP, int PP, int RW>
__global__ void __launch_bounds__(RW * 32, 20 / RW) ray32_kernel(RayParams P) {
  extern __shared__ __align__(16) float sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpLayout lay = warp_layout(P.n_max, PP, RP, P.nc_max);
  float* base = sm + (size_t)warp * (lay.bytes / 4);
  double* Lg = P.g64 + ((int64_t)blockIdx.x * RW + warp) * P.g64_stride;
  const unsigned items = P.count ? *P.count : (unsigned)P.M;
  for (;;) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(P.queue, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= items) break;
    ray32_location<RP, PP>(P, P.order ? (int64_t)P.order[it] : (int64_t)it, base, Lg);
    __syncwarp();
  }
}

// Warps per CTA that let the most locations reside on an SM at this shape:
// shared memory decides, under the launch bound's 20 warps per SM; ties go to
// 2, then 4, then 1, and 2 is the answer when no device can be queried.
int ray32_default_warps(int p, int n_max, int nc_max, int nrays) {
  int dev = 0, smem_sm = 0, reserved = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
          cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  int RP = 2;
  while (RP < nrays) RP <<= 1;
  const size_t wb = (size_t)warp_layout(n_max, (p + 3) / 4 * 4, RP, nc_max).bytes;
  return warps_per_cta_for_residency(wb, (size_t)smem_sm, (size_t)reserved, 20);
}

size_t ray32_g64_doubles(int n_max) { return (size_t)tri(n_max) + 2 * (size_t)n_max; }

// Warp slots for a chunk: at least one CTA of the widest choice (4 warps) and a
// multiple of 4, so that every warp of every launched CTA owns a slot.
int ray32_slots(int64_t chunk) {
  const int64_t s = chunk < RAY_SLOTS ? chunk : RAY_SLOTS;
  return (int)((s + 3) / 4 * 4);
}

template <int RP, int PP, int RW>
static cudaError_t ray32_go(const RayParams& P, size_t sm, int slots, cudaStream_t s) {
  auto k = ray32_kernel<RP, PP, RW>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (err != cudaSuccess) return err;
  const int64_t grid = persistent_grid(k, RW * 32, sm, P.M, slots, RW);
  if (grid < 0) return cudaErrorInvalidValue;
  if ((err = cudaMemsetAsync(P.queue, 0, sizeof(unsigned), s)) != cudaSuccess) return err;
  prof_begin("ray32", s);
  k<<<(unsigned)grid, RW * 32, sm, s>>>(P);
  prof_end(s);
  return cudaGetLastError();
}

cudaError_t launch_ray32(const DesignArgs& a, cudaStream_t s) {
  RayParams P;
  P.X = a.X; P.Y = a.Y; P.p = a.p; P.PP = a.PP; P.Xf = a.ws->Xf; P.xref = a.xref; P.M = a.M;
  P.cand = a.cand; P.nc_max = a.nc_max; P.nc_loc = a.nc_loc; P.n0 = a.n0; P.n_max = a.n_max;
  P.n_loc = a.n_loc; P.theta = a.theta; P.theta_loc = a.theta_loc; P.g = a.g; P.R = a.nrays; P.lo = a.ws->lo;
  P.hi = a.ws->hi; P.center = a.ws->center; P.mean = a.mean; P.s2 = a.s2;
  P.selected = a.selected; P.tie_gap = a.tie_gap; P.nevals = a.nevals; P.g64 = a.ws->state64;
  P.g64_stride = (int64_t)ray32_g64_doubles(a.n_max); P.status = a.ws->status;
  P.queue = a.ws->queue; P.order = a.order; P.count = a.count;
  P.full = a.full_scope;
  P.promote = a.promote ? a.ws->promote : nullptr;
  P.promote_count = a.ws->status + 1;
  if (P.full) {
    const KdTree& t = a.ws->kd;
    P.kd.box = t.box32; P.kd.stride = a.PP; P.kd.p = a.p; P.kd.D = t.D; P.kd.N = a.N;
    P.kd.perm = t.perm; P.kd.pts = t.pts32; P.kd.by_design = false;
  } else {
    std::memset(&P.kd, 0, sizeof(P.kd));
  }
  int RP = 2;
  while (RP < a.nrays) RP <<= 1;
  const WarpLayout lay = warp_layout(a.n_max, a.PP, RP, a.nc_max);
  const int RW = a.tune.ray_warps;
  const size_t sm = (size_t)lay.bytes * RW;
  const int slots = ray32_slots(a.ws->chunk);
  const int key = (RW * 100 + RP) * 100 + a.PP;
  switch (key) {
#define RAY_CASE(RWV, RPV, PPV) \
  case (RWV * 100 + RPV) * 100 + PPV: return ray32_go<RPV, PPV, RWV>(P, sm, slots, s);
#define RAY_CASES(RWV)                                                                   \
    RAY_CASE(RWV, 2, 4) RAY_CASE(RWV, 2, 8) RAY_CASE(RWV, 2, 12) RAY_CASE(RWV, 2, 16)     \
    RAY_CASE(RWV, 4, 4) RAY_CASE(RWV, 4, 8) RAY_CASE(RWV, 4, 12) RAY_CASE(RWV, 4, 16)     \
    RAY_CASE(RWV, 8, 4) RAY_CASE(RWV, 8, 8) RAY_CASE(RWV, 8, 12) RAY_CASE(RWV, 8, 16)     \
    RAY_CASE(RWV, 16, 4) RAY_CASE(RWV, 16, 8) RAY_CASE(RWV, 16, 12) RAY_CASE(RWV, 16, 16)
    RAY_CASES(1) RAY_CASES(2) RAY_CASES(4)
#undef RAY_CASES
#undef RAY_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace lagp
