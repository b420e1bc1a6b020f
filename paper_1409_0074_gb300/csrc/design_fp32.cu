// design_fp32.cu -- exhaustive greedy local design with FP32 candidate scoring
// and an FP64 factor update, one CTA per predictive location: the exhaustive
// search of the LAGP_FP32_SCORE form for every n, and of LAGP_FP32_SCORE_TC
// for the designs larger than its tensor-core scorer (exh_tc.cu) takes.  The
// ray search of these forms is in ray32.cu.
//
// Scoring form.  With K_j = L_j L_j^T (Cholesky) the ALC integrand of Eq. alc
// (sign reading as in the FP64 path) becomes
//     w = L_j^{-1} k_j(x'),  v = (1 + g) - |w|^2,
//     ALC(x') = (w . z - K(x', x))^2 / v,   z = L_j^{-1} k_j(x),
// the same quadratic forms as k^T K^{-1} k, evaluated through the inverse
// factor.  In FP32 this keeps the error of v near eps * sqrt(cond K) instead of
// eps * cond K: on the 8-d, N = 1e6 workload (cond K_50 ~ 1e6, v ~ 1e-4) an
// explicit-inverse FP32 score has errors as large as v itself, while the
// factored score stays near 5e-6.
//
// FP64 state (the partitioned update, Sec 2.2, in factored form): appending
// x_new with l = L_j^{-1} k_j(x_new), v = (1 + g) - |l|^2 (the Schur complement
// of the paper's update), d = sqrt(v) gives
//     L_{j+1}^{-1} = [[L_j^{-1}, 0], [-(L_j^{-T} l)^T / d, 1 / d]],
// so one new row per step, O(j^2).  z and L^{-1} y grow by one entry per step
// and the predictive equations (Eq. predgp, preds2) follow as
//     mu = z . (L^{-1} y),  psi = |L^{-1} y|^2,  sigma^2 = psi (1 + g - |z|^2) / n.
//
// Incremental scores.  Because the inverse factor only gains a row, every
// candidate's w (and z) only gains an entry per step: w_cj = row_j . K(S, c).
// Each CTA keeps |w_c|^2 and w_c . z as running sums per candidate, so a step
// costs O(N' j) instead of the O(N' j^2) of re-forming every w, and a full
// design O(N' n^2) instead of O(N' n^3); the sums see the same FP32 operations
// in the same order as a from-scratch evaluation would.
// Scoring coordinates are FP32 and centred on the design's bounding box.
#include <cstdint>

#include "common.cuh"
#include "lagp_internal.h"

namespace lagp {

#define D32_THREADS 256
#define D32_WARPS (D32_THREADS / 32)

struct D32Params {
  const double* X;
  const double* Y;
  int p, PP;
  const float* Xf;       // centred FP32 design [Npad][PP]
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
  double* Linv;          // [slots][n_max][n_max] FP64 inverse factor
  float* Kc;             // exhaustive: [slots][n_max][nc_max] FP32 correlation cache
  float* crow;           // [slots][nc_max][PP] the location's candidates' FP32 rows
  unsigned* status;
  unsigned* queue;       // work counter (zero at launch)
  const int32_t* order;  // item -> location, or null
  const unsigned* count; // items (device), or null (M)
  int32_t* promote;      // binary64 re-solve list, or null (promotion off)
  unsigned* promote_count;
};

struct L32 {
  float* Lf;       // [n_max] FP32 copy of the newest row of L^{-1}
  float* zf;       // [n_max]
  float* Sf;       // [n_max][PP] centred FP32 selected coordinates
  float* xf;       // [PP]
  float* vs;       // [nc_max] running |w_c|^2 of every candidate
  float* ns;       // [nc_max] running w_c . z
  float* kxc;      // [nc_max] K(c, x)
  float* red;      // [WARPS*4]
  double* S64;     // [n_max][p]
  double* xq;      // [p]
  double* kvec;    // [n_max]
  double* l;       // [n_max]
  double* z;       // [n_max]
  double* zy;      // [n_max]
  double* kx;      // [n_max]
  double* dred;    // [WARPS*4]
  int* sel;        // [n_max]
  int* ired;       // [WARPS*2]
  unsigned char* used;
  int j;
  float neg_inv_theta, onepg;
};

// lengthscale of the CTA's current location (kept out of the registers)
static __shared__ double d32_theta;

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sumd(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Sum over the block of FP64 terms held only by threads below `active`, to
// thread 0 (the other threads' a, b are left as their warp sums or unchanged).
// Only the warps holding terms shuffle, and thread 0 adds the warp totals in
// warp order, so the result is bit-identical to a full block sum (the idle
// warps' totals are exact zeros) at a fraction of its FP64 instructions,
// which are scarce on this part.  Every thread must call it.
__device__ __forceinline__ void sum_to_thread0(double& a, double& b, int active, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int aw = min((active + 31) >> 5, D32_WARPS);
  if (warp < aw) {
    a = warp_sumd(a);
    b = warp_sumd(b);
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
__device__ __forceinline__ void sum_to_thread0(double& a, int active, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int aw = min((active + 31) >> 5, D32_WARPS);
  if (warp < aw) {
    a = warp_sumd(a);
    if (lane == 0) red[warp] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0;
    for (int w = 0; w < aw; ++w) ta += red[w];
    a = ta;
  }
}

// best (value, index) over the block: larger value wins, ties to the lower index
struct VI { float v; int i; float v2; };
__device__ __forceinline__ VI vi_merge_max(VI a, VI b) {
  VI r;
  if (b.v > a.v || (b.v == a.v && b.i >= 0 && (a.i < 0 || b.i < a.i))) {
    r.v = b.v; r.i = b.i; r.v2 = fmaxf(a.v, b.v2);
  } else {
    r.v = a.v; r.i = a.i; r.v2 = fmaxf(a.v2, b.v);
  }
  return r;
}
__device__ VI block_best(VI t, float* fs, int* is) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    VI u;
    u.v = __shfl_xor_sync(0xffffffffu, t.v, o);
    u.i = __shfl_xor_sync(0xffffffffu, t.i, o);
    u.v2 = __shfl_xor_sync(0xffffffffu, t.v2, o);
    t = vi_merge_max(t, u);
  }
  if (lane == 0) { fs[2 * warp] = t.v; fs[2 * warp + 1] = t.v2; is[warp] = t.i; }
  __syncthreads();
  VI r; r.v = fs[0]; r.v2 = fs[1]; r.i = is[0];
  for (int w = 1; w < D32_WARPS; ++w) {
    VI u; u.v = fs[2 * w]; u.v2 = fs[2 * w + 1]; u.i = is[w];
    r = vi_merge_max(r, u);
  }
  __syncthreads();
  return r;
}

// candidate rank r's FP32 row, from the slot's gathered copy
__device__ __forceinline__ const float* cand_f(const D32Params& P, const float* crow, int r) {
  return crow + (int64_t)r * P.PP;
}

// Append candidate rank r: FP64 factor row, z, L^{-1}y, FP32 copies, the
// correlation-cache row K(S_j, c) and entry j of every unselected candidate's w.
// `best` receives this thread's part of the next search: the ALC of every
// unselected candidate the thread updates, from the running sums it has just
// written (the same arithmetic and candidate order as a separate pass).
__device__ bool add_point32(const D32Params& P, L32& L, const int32_t* cl, const float* crow,
                            int nc, int r, double* Lg, float* Kc_loc, VI* best) {
  const int tid = threadIdx.x, p = P.p, j = L.j, ld = P.n_max;
  const double* c = P.X + (int64_t)cl[r] * p;
  if (tid < p) L.S64[j * p + tid] = c[tid];
  if (tid < P.PP) L.Sf[j * P.PP + tid] = cand_f(P, crow, r)[tid];
  __syncthreads();
  const double nit64 = -1.0 / d32_theta;
  // correlations of the new point with the design, and with x (thread j)
  for (int i = tid; i <= j; i += blockDim.x) {
    if (i < j) L.kvec[i] = corr64_fast(L.S64 + i * p, L.S64 + j * p, p, nit64);
    else L.kx[j] = corr64_fast(L.S64 + j * p, L.xq, p, nit64);
  }
  __syncthreads();
  // l = L_j^{-1} k_j(x_new); thread 0 forms the pivot v = 1 + g - |l|^2, 1/sqrt(v)
  double vv = 0.0;
  for (int i = tid; i < j; i += blockDim.x) {
    const double acc = dot64_ilp(Lg + (int64_t)i * ld, L.kvec, i + 1);
    L.l[i] = acc;
    vv = fma(acc, acc, vv);
  }
  sum_to_thread0(vv, j, L.dred);
  double* piv = L.dred + 2 * D32_WARPS;
  if (tid == 0) {
    const double v = (1.0 + P.g) - vv;
    piv[0] = v;
    piv[1] = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
  }
  __syncthreads();
  if (!(piv[0] > 0.0)) return false;
  const double inv_d = piv[1];
  for (int k = tid; k < j; k += blockDim.x) {
    double a0 = 0.0, a1 = 0.0;
    int i = k;
    for (; i + 1 < j; i += 2) {
      a0 = fma(L.l[i], Lg[(int64_t)i * ld + k], a0);
      a1 = fma(L.l[i + 1], Lg[(int64_t)(i + 1) * ld + k], a1);
    }
    if (i < j) a0 = fma(L.l[i], Lg[(int64_t)i * ld + k], a0);
    const double rk = -(a0 + a1) * inv_d;
    Lg[(int64_t)j * ld + k] = rk;
    L.Lf[k] = (float)rk;
  }
  if (tid == 0) {
    Lg[(int64_t)j * ld + j] = inv_d;
    L.Lf[j] = (float)inv_d;
    L.sel[j] = r;
    L.used[r] = 1;
  }
  __syncthreads();
  // z_j = row_j . k(x), (L^{-1} y)_j = row_j . y_S
  double zz = 0.0, zyy = 0.0;
  for (int k = tid; k <= j; k += blockDim.x) {
    const double rk = Lg[(int64_t)j * ld + k];
    zz = fma(rk, L.kx[k], zz);
    zyy = fma(rk, P.Y[cl[L.sel[k]]], zyy);
  }
  sum_to_thread0(zz, zyy, j + 1, L.dred);
  if (tid == 0) {
    L.z[j] = zz;
    L.zy[j] = zyy;
    L.zf[j] = (float)zz;
  }
  __syncthreads();
  // Row j of L^{-1} is final once written, so w_c = L^{-1} k_j(c) only gains
  // the entry w_cj = row_j . K(S_{0..j}, c); |w_c|^2 and w_c . z are running
  // sums in the order i = 0, 1, ..., the same FP32 operations a from-scratch
  // evaluation at every step would perform.  Thread q owns candidates
  // q, q + blockDim, ..., and takes the newest entry from the register that
  // computed it.  Even terms go to a0 and odd terms to a1, in ascending order.
  const int64_t ldc = P.nc_max;
  float* row = Kc_loc + (int64_t)j * ldc;
  const float* sj = L.Sf + j * P.PP;
  const float* Lfj = L.Lf;
  const float zj = L.zf[j];
  VI b;
  b.v = -1.f; b.v2 = -1.f; b.i = -1;
  for (int q = tid; q < nc; q += blockDim.x) {
    const float kv = __expf(sqdist_row32(cand_f(P, crow, q), sj, P.PP) * L.neg_inv_theta);
    row[q] = kv;
    if (L.used[q]) continue;
    const float* kc = Kc_loc + q;
    float a0 = 0.f, a1 = 0.f;
    int k = 0;
#pragma unroll 4
    for (; k + 2 <= j; k += 2) {
      a0 = fmaf(Lfj[k], kc[k * ldc], a0);
      a1 = fmaf(Lfj[k + 1], kc[(k + 1) * ldc], a1);
    }
    if (k == j) {
      a0 = fmaf(Lfj[j], kv, a0);
    } else {
      a0 = fmaf(Lfj[k], kc[k * ldc], a0);
      a1 = fmaf(Lfj[j], kv, a1);
    }
    const float w = a0 + a1;
    const float nvs = fmaf(w, w, L.vs[q]), nns = fmaf(w, zj, L.ns[q]);
    L.vs[q] = nvs;
    L.ns[q] = nns;
    const float v = L.onepg - nvs;
    const float num = nns - L.kxc[q];
    const float alc = v > 0.f ? num * num / v : 0.f;
    if (alc > b.v) { b.v2 = b.v; b.v = alc; b.i = q; }
    else if (alc > b.v2) b.v2 = alc;
  }
  *best = b;
  __syncthreads();
  L.j = j + 1;
  return true;
}

// ----- exhaustive search, CUDA-core FP32 scoring ---------------------------------
// ALC_c = (w_c . z - K(c, x))^2 / ((1 + g) - |w_c|^2) from the running sums;
// the largest score wins, ties to the lower candidate rank.  Each thread's part
// comes from the update loop of the last appended point (add_point32).
__device__ int search_exh32(const L32& L, VI best, double* gap_out) {
  VI b = block_best(best, L.red, L.ired);
  *gap_out = (b.v > 0.f && b.v2 >= 0.f) ? (double)((b.v - b.v2) / b.v) : 0.0;
  return b.i;
}

// PROMOTE: with precision promotion (a separate instantiation, so that the
// default one carries none of its code)
template <bool PROMOTE>
__global__ void __launch_bounds__(D32_THREADS, 6) design32(D32Params P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_item;
  const int tid = threadIdx.x, p = P.p, PP = P.PP, ld = P.n_max;
  // scratch of this CTA slot
  double* Lg = P.Linv + (int64_t)blockIdx.x * ld * ld;
  float* Kc_loc = P.Kc + (int64_t)blockIdx.x * ld * P.nc_max;
  float* crow = P.crow + (int64_t)blockIdx.x * P.nc_max * PP;

  L32 L;
  double* dp = reinterpret_cast<double*>(smem);
  L.S64 = dp; dp += ld * p;
  L.xq = dp; dp += p;
  L.kvec = dp; dp += ld;
  L.l = dp; dp += ld;
  L.z = dp; dp += ld;
  L.zy = dp; dp += ld;
  L.kx = dp; dp += ld;
  L.dred = dp; dp += 4 * D32_WARPS;
  float* fp = reinterpret_cast<float*>(dp);
  L.Lf = fp; fp += ld;
  L.zf = fp; fp += ld;
  L.Sf = fp; fp += ld * PP;
  L.xf = fp; fp += PP;
  L.vs = fp; fp += P.nc_max;
  L.ns = fp; fp += P.nc_max;
  L.kxc = fp; fp += P.nc_max;
  L.red = fp; fp += 4 * D32_WARPS;
  int* ip = reinterpret_cast<int*>(fp);
  L.sel = ip; ip += ld;
  L.ired = ip; ip += 2 * D32_WARPS + 2;
  L.used = reinterpret_cast<unsigned char*>(ip);
  L.onepg = (float)(1.0 + P.g);
  L.neg_inv_theta = (float)(-1.0 / P.theta);
  if (threadIdx.x == 0) d32_theta = P.theta;
  const unsigned items = P.count ? *P.count : (unsigned)P.M;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(P.queue, 1u);
    __syncthreads();
    const unsigned it = s_item;
    __syncthreads();
    if (it >= items) break;
    const int64_t loc = P.order ? (int64_t)P.order[it] : (int64_t)it;
    const int nc = P.nc_loc ? P.nc_loc[loc] : P.nc_max;
    const int n = P.n_loc ? P.n_loc[loc] : P.n_max;
    const int32_t* cl = P.cand + loc * P.nc_max;
    L.j = 0;
    if (P.theta_loc) {
      const double th = P.theta_loc[loc];
      if (tid == 0) d32_theta = th;
      L.neg_inv_theta = (float)(-1.0 / th);
    }

    if (tid < p) L.xq[tid] = P.xref[loc * p + tid];
    if (tid < PP) L.xf[tid] = tid < p ? (float)(P.xref[loc * p + tid] - P.center[tid]) : 0.f;
    if (P.tie_gap) for (int i = tid; i < ld; i += blockDim.x) P.tie_gap[loc * ld + i] = 0.0;
    if (P.nevals) for (int i = tid; i < ld; i += blockDim.x) P.nevals[loc * ld + i] = 0;
    // the candidates' FP32 rows, gathered once into the slot in rank order
    for (int e = tid; e < nc * (PP >> 2); e += blockDim.x) {
      const int q = e / (PP >> 2), c4 = (e - q * (PP >> 2)) << 2;
      *reinterpret_cast<float4*>(crow + (int64_t)q * PP + c4) =
          *reinterpret_cast<const float4*>(P.Xf + (int64_t)cl[q] * PP + c4);
    }
    __syncthreads();
    for (int r = tid; r < nc; r += blockDim.x) {
      L.used[r] = 0;
      L.vs[r] = 0.f;
      L.ns[r] = 0.f;
      L.kxc[r] = __expf(sqdist_row32(cand_f(P, crow, r), L.xf, PP) * L.neg_inv_theta);
    }
    __syncthreads();

    bool ok = (n >= P.n0) && (n <= nc) && (n <= ld);
    VI part;
    for (int r = 0; r < P.n0 && ok; ++r) ok = add_point32(P, L, cl, crow, nc, r, Lg, Kc_loc, &part);
    for (int j = P.n0; j < n && ok; ++j) {
      double gap = 0.0;
      int ne = 0;
      int r = search_exh32(L, part, &gap);
      if (tid == 0) {
        if (P.tie_gap) P.tie_gap[loc * ld + (j - P.n0)] = gap;
        if (P.nevals) P.nevals[loc * ld + (j - P.n0)] = ne;
      }
      ok = (r >= 0) && add_point32(P, L, cl, crow, nc, r, Lg, Kc_loc, &part);
    }
    if (ok) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int i = tid; i < L.j; i += blockDim.x) {
        a = fma(L.z[i], L.zy[i], a);
        b = fma(L.zy[i], L.zy[i], b);
        c = fma(L.z[i], L.z[i], c);
      }
      sum_to_thread0(a, b, L.j, L.dred);
      sum_to_thread0(c, L.j, L.dred + 2 * D32_WARPS);
      if (tid == 0) {
        P.mean[loc] = a;
        P.s2[loc] = b * ((1.0 + P.g) - c) / (double)L.j;
      }
    } else if (tid == 0) {
      P.mean[loc] = __longlong_as_double(0x7ff8000000000000ll);
      P.s2[loc] = __longlong_as_double(0x7ff8000000000000ll);
      atomicOr(P.status, LAGP_DEV_BAD_UPDATE);
    }
    if (P.selected)
      for (int i = tid; i < ld; i += blockDim.x)
        P.selected[loc * ld + i] = (i < L.j) ? cl[L.sel[i]] : -1;
    if (PROMOTE && tid == 0) {
      // smallest binary64 pivot v of the design: the factor's diagonal holds
      // 1 / sqrt(v); a failed update promotes the location
      double vm = ok ? INFINITY : -1.0;
      for (int i = 0; i < L.j; ++i) {
        const double dg = Lg[(int64_t)i * ld + i];
        vm = fmin(vm, 1.0 / (dg * dg));
      }
      promote_location(P.promote, P.promote_count, loc, vm);
    }
  }
}

static size_t smem_design32(int n_max, int p, int PP, int nc_max) {
  size_t d = (size_t)n_max * p + p + 5 * n_max + 4 * D32_WARPS;
  size_t f = 2 * (size_t)n_max + (size_t)n_max * PP + PP + 3 * (size_t)nc_max + 4 * D32_WARPS;
  size_t i = (size_t)n_max + 2 * D32_WARPS + 2;
  return d * 8 + f * 4 + i * 4 + nc_max + 16;
}

cudaError_t launch_exh32(const DesignArgs& a, cudaStream_t s) {
  D32Params P;
  P.X = a.X; P.Y = a.Y; P.p = a.p; P.PP = a.PP; P.Xf = a.ws->Xf; P.xref = a.xref; P.M = a.M;
  P.cand = a.cand; P.nc_max = a.nc_max; P.nc_loc = a.nc_loc; P.n0 = a.n0; P.n_max = a.n_max;
  P.n_loc = a.n_loc; P.theta = a.theta; P.theta_loc = a.theta_loc; P.g = a.g;
  P.center = a.ws->center; P.mean = a.mean; P.s2 = a.s2;
  P.selected = a.selected; P.tie_gap = a.tie_gap; P.nevals = a.nevals; P.Linv = a.ws->state64;
  P.Kc = a.ws->state32; P.crow = a.ws->crow; P.status = a.ws->status;
  P.queue = a.ws->queue + 2; P.order = a.order; P.count = a.count;
  P.promote = a.promote ? a.ws->promote : nullptr;
  P.promote_count = a.ws->status + 1;
  size_t sm = smem_design32(a.n_max, a.p, a.PP, a.nc_max);
  auto k = P.promote ? design32<true> : design32<false>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (err != cudaSuccess) return err;
  const int64_t grid = persistent_grid(k, D32_THREADS, sm, a.M, exh_slots(a.ws->chunk), 1,
                                       a.tune.exh_occ);
  if (grid < 0) return cudaErrorInvalidValue;
  if ((err = cudaMemsetAsync(P.queue, 0, sizeof(unsigned), s)) != cudaSuccess) return err;
  prof_begin("design32_exhaustive", s);
  k<<<(unsigned)grid, D32_THREADS, sm, s>>>(P);
  prof_end(s);
  return cudaGetLastError();
}

}  // namespace lagp
