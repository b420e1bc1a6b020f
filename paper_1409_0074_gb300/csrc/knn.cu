// knn.cu -- brute-force tiled kNN candidate selection (Gramacy & Haaland,
// Sec 2.2: the local search is restricted to the N' nearest neighbours of x).
//
// Two stages:
//  1. knn_stream: each CTA owns 32 predictive locations (4 per warp) and
//     streams the whole design through shared memory in 256-point tiles moved
//     by bulk-copy (TMA) into a double buffer.  Distances are computed in FP32
//     from centred coordinates; a point enters its location's candidate
//     buffer when d32 <= tau + 2 err, where tau is the N'-th smallest buffered
//     d32 and err a proven bound on |d32 - d64|.  A warp radix-selects tau and
//     compacts the buffer whenever the next tile might overflow it.
//  2. knn_rank: one CTA per location computes the exact binary64 distances of
//     the surviving points in the oracle's operation order and bitonic-sorts
//     (d64, index) pairs; the first N' indices are the candidate list.
// Every true member of the N'-nearest set survives stage 1: at the end at
// least N' points have d32 <= tau, so the N'-th smallest d64 is at most
// tau + err, and any member has d32 <= d64 + err <= tau + 2 err.
//
// Pilot threshold (N >= 32 N').  Before the stream, knn_pilot estimates each
// location's N'-th distance from a stride sample of S = min(32768, N / 16)
// design points: with
// lambda = S N'/N sample points expected inside it, the m-th smallest sample
// distance, m = lambda + 4.5 sqrt(lambda) + 4, is above it except with
// probability ~1e-5.  The stream starts with tau = that value instead of
// infinity, so few points are buffered and the buffer rarely needs a
// compaction.  The estimate is checked, not trusted: at the end at least N'
// buffered points must lie at or below it (then the N'-th smallest d32 does
// too, and every point that could belong was admitted); a location that fails
// the check is streamed again with tau = infinity.
#include <cfloat>
#include <cstdint>

#include "common.cuh"
#include "knn_common.cuh"
#include "lagp_internal.h"

namespace lagp {

#define KNN_WARPS 8
#define KNN_QW 4   // locations per warp


// ---------------------------------------------------------------------------
// Preparation: bounding box (exact min/max), centred FP32 copy of the design,
// squared norms, largest squared norm.
// ---------------------------------------------------------------------------
__global__ void bbox_partial(const double* __restrict__ X, int64_t N, int p,
                             double* __restrict__ part /*[gridDim.x][2p]*/) {
  __shared__ double slo[256], shi[256];
  for (int k = 0; k < p; ++k) {
    double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
      double v = X[i * p + k];
      lo = fmin(lo, v);
      hi = fmax(hi, v);
    }
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
        shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      part[blockIdx.x * 2 * p + k] = slo[0];
      part[blockIdx.x * 2 * p + p + k] = shi[0];
    }
    __syncthreads();
  }
}

__global__ void bbox_final(const double* __restrict__ part, int nparts, int p,
                           double* __restrict__ lo, double* __restrict__ hi,
                           double* __restrict__ center) {
  int k = threadIdx.x;
  if (k >= p) return;
  double l = part[k], h = part[p + k];
  for (int b = 1; b < nparts; ++b) {
    l = fmin(l, part[b * 2 * p + k]);
    h = fmax(h, part[b * 2 * p + p + k]);
  }
  lo[k] = l;
  hi[k] = h;
  center[k] = 0.5 * (l + h);
}

// Xf[i][0..PP) = fl32(X[i] - center) (zero padded), nx[i] = |Xf[i]|^2 in FP32;
// rows N..Npad-1 are zero with nx = 1e30.  maxn2 receives max_{i<N} nx[i]
// (as ordered bits).
__global__ void design_to_f32(const double* __restrict__ X, int64_t N, int64_t Npad, int p, int PP,
                              const double* __restrict__ center, float* __restrict__ Xf,
                              float* __restrict__ nx, unsigned* __restrict__ maxn2_bits) {
  float local_max = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Npad;
       i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int k = 0; k < PP; ++k) {
      float v = 0.f;
      if (i < N && k < p) v = (float)(X[i * p + k] - center[k]);
      Xf[i * PP + k] = v;
      acc = fmaf(v, v, acc);
    }
    // padding rows get |x|^2 = 1e30, so that no distance to them passes
    nx[i] = i < N ? acc : 1e30f;
    if (i < N) local_max = fmaxf(local_max, acc);
  }
  for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxn2_bits, __float_as_uint(local_max));
}

template <int PP>
__device__ __forceinline__ void knn_d4(const float (&qf)[KNN_QW][PP], const float (&nq)[KNN_QW],
                                       const float (&xv)[PP], float nxp, float (&d)[KNN_QW]) {
#pragma unroll
  for (int a = 0; a < KNN_QW; ++a) {
    float dot = 0.f;
#pragma unroll
    for (int k = 0; k < PP; ++k) dot = fmaf(qf[a][k], xv[k], dot);
    d[a] = fmaf(-2.f, dot, nq[a] + nxp);
  }
}

// first bin (of 256 per location, lane l owning bins 8l..8l+7) at which the
// running count reaches k; *below receives the count before that bin
__device__ __forceinline__ int warp_bin_of_kth(const uint32_t* h, int k, int* below) {
  const int lane = threadIdx.x & 31;
  uint32_t c[8], tot = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) { c[b] = h[lane * 8 + b]; tot += c[b]; }
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const uint32_t excl = incl - tot;
  const int found = ((int)excl < k && (int)incl >= k);
  const uint32_t fm = __ballot_sync(0xffffffffu, found);
  int bin = 255, run_out = 0;
  if (found) {
    uint32_t run = excl;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      if ((int)(run + c[b]) >= k) { bin = lane * 8 + b; run_out = (int)run; break; }
      run += c[b];
    }
  }
  const int src = fm ? __ffs(fm) - 1 : 0;
  *below = __shfl_sync(0xffffffffu, run_out, src);
  return fm ? __shfl_sync(0xffffffffu, bin, src) : -1;
}

// Pilot thresholds: per location the upper edge of the 2^-8-wide bin (by the
// float bit pattern: exponent, then the top 8 mantissa bits) that holds the
// m-th smallest d32 of the S sample rows i * (N / S); +inf where the pilot
// does not apply (m > S, or more than cap - 2 tiles expected below it).
template <int PP>
__global__ void __launch_bounds__(KNN_WARPS * 32)
knn_pilot(const float* __restrict__ Xf, const float* __restrict__ nx, int64_t N, int64_t S, int p,
          const double* __restrict__ xref, int64_t M, const double* __restrict__ center,
          int nc_max, const int32_t* __restrict__ nc_loc, int cap, float* __restrict__ thr_out) {
  // the sample rows pass through shared memory a tile at a time, shared by
  // the CTA's warps (each sample row is read from L2 once per CTA and pass)
  constexpr int T = 2048 / PP;
  __shared__ uint32_t hist[KNN_WARPS][KNN_QW][256];
  __shared__ __align__(16) float sx[T * PP];
  __shared__ float sn[T];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q0 = (int64_t)blockIdx.x * (KNN_WARPS * KNN_QW) + warp * KNN_QW;
  float qf[KNN_QW][PP], nq[KNN_QW];
  int m[KNN_QW];
  const int64_t stride = N / S;
#pragma unroll
  for (int a = 0; a < KNN_QW; ++a) {
    const int64_t q = q0 + a;
    const bool live = q < M;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      float v = 0.f;
      if (live && k < p) v = (float)(xref[q * p + k] - center[k]);
      qf[a][k] = v;
      acc = fmaf(v, v, acc);
    }
    nq[a] = acc;
    const int nc = live ? (nc_loc ? nc_loc[q] : nc_max) : 0;
    const float lam = (float)S * (float)nc / (float)N;
    m[a] = (int)ceilf(lam + 4.5f * sqrtf(lam) + 4.f);
    // expected admitted points m N / S must leave two tiles of room
    if (!live || m[a] > S || (double)m[a] * (double)N / (double)S > (double)(cap - 2 * LAGP_KNN_TILE))
      m[a] = 0;
  }
  uint32_t b1[KNN_QW];
  int below[KNN_QW];
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = lane; i < KNN_QW * 256; i += 32) (&hist[warp][0][0])[i] = 0u;
    __syncwarp();
    for (int64_t t0 = 0; t0 < S; t0 += T) {
      const int cnt = (int)(S - t0 < T ? S - t0 : T);
      __syncthreads();   // the previous tile is consumed
      for (int e = threadIdx.x; e < cnt * (PP / 4); e += blockDim.x) {
        const int r = e / (PP / 4), c4 = (e - r * (PP / 4)) * 4;
        *reinterpret_cast<float4*>(sx + r * PP + c4) =
            __ldg(reinterpret_cast<const float4*>(Xf + (t0 + r) * stride * PP + c4));
      }
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) sn[e] = __ldg(nx + (t0 + e) * stride);
      __syncthreads();
      for (int i = lane; i < cnt; i += 32) {
        float xv[PP];
#pragma unroll
        for (int k = 0; k < PP; k += 4) {
          const float4 v4 = *reinterpret_cast<const float4*>(sx + i * PP + k);
          xv[k] = v4.x; xv[k + 1] = v4.y; xv[k + 2] = v4.z; xv[k + 3] = v4.w;
        }
        float d[KNN_QW];
        knn_d4<PP>(qf, nq, xv, sn[i], d);
#pragma unroll
        for (int a = 0; a < KNN_QW; ++a) {
          const uint32_t bits = __float_as_uint(fmaxf(d[a], 0.f));
          if (pass == 0) atomicAdd(&hist[warp][a][bits >> 23], 1u);
          else if ((bits >> 23) == b1[a]) atomicAdd(&hist[warp][a][(bits >> 15) & 255u], 1u);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < KNN_QW; ++a) {
      if (pass == 0) {
        const int b = warp_bin_of_kth(hist[warp][a], m[a] > 0 ? m[a] : 1, &below[a]);
        b1[a] = b < 0 ? 0u : (uint32_t)b;
      } else {
        int dummy = 0;
        const int b = warp_bin_of_kth(hist[warp][a], m[a] > 0 ? m[a] - below[a] : 1, &dummy);
        float thr = __uint_as_float((b1[a] << 23) | ((uint32_t)(b < 0 ? 255 : b) << 15) | 0x7fffu);
        if (m[a] == 0 || b < 0 || !(thr < __int_as_float(0x7f800000))) thr = __int_as_float(0x7f800000);
        if (lane == 0 && q0 + a < M) thr_out[q0 + a] = thr;
      }
    }
    __syncwarp();
  }
}

template <int PP>
__global__ void __launch_bounds__(KNN_WARPS * 32, 3)
knn_stream(const float* __restrict__ Xf, const float* __restrict__ nx, int64_t N, int64_t ntiles,
           int p, const double* __restrict__ xref, int64_t M, const double* __restrict__ center,
           const unsigned* __restrict__ maxn2_bits, int nc_max, const int32_t* __restrict__ nc_loc,
           int cap, KnnEntry* __restrict__ buf, int32_t* __restrict__ cnt_out,
           unsigned* __restrict__ status, const float* __restrict__ pilot, int redo) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* tile = reinterpret_cast<float*>(smem);                    // [2][TILE][PP]
  float* tnorm = tile + 2 * LAGP_KNN_TILE * PP;                     // [2][TILE]
  uint32_t* hist = reinterpret_cast<uint32_t*>(tnorm + 2 * LAGP_KNN_TILE);  // [WARPS][256]
  uint64_t* bar = reinterpret_cast<uint64_t*>(hist + KNN_WARPS * 256);      // [2]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q0 = (int64_t)blockIdx.x * (KNN_WARPS * KNN_QW) + warp * KNN_QW;

  float qf[KNN_QW][PP], nq[KNN_QW], err[KNN_QW], keep[KNN_QW];
  int cnt[KNN_QW], ncq[KNN_QW];
  bool live[KNN_QW];
  const float rmax = sqrtf(__uint_as_float(*maxn2_bits)) * 1.0001f;
  const float inf = __int_as_float(0x7f800000);
  bool any = false;
#pragma unroll
  for (int a = 0; a < KNN_QW; ++a) {
    int64_t q = q0 + a;
    live[a] = q < M;
    // redo pass: only the locations whose pilot threshold failed its check
    if (redo && live[a]) live[a] = cnt_out[q] < 0;
    any = any || live[a];
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      float v = 0.f;
      if (live[a] && k < p) v = (float)(xref[q * p + k] - center[k]);
      qf[a][k] = v;
      acc = fmaf(v, v, acc);
    }
    nq[a] = acc;
    float r = rmax + sqrtf(acc) * 1.0001f;
    err[a] = (float)(p + 12) * 0x1p-24f * 1.25f * r * r;
    const float thr = (live[a] && pilot) ? pilot[q] : inf;
    keep[a] = live[a] ? (thr < inf ? __fadd_ru(thr, 2.f * err[a]) : inf) : -1.f;
    cnt[a] = 0;
    ncq[a] = live[a] ? (nc_loc ? nc_loc[q] : nc_max) : 0;
  }
  if (!__syncthreads_or(any)) return;   // a redo pass with nothing to redo here

  const uint32_t tile_bytes = LAGP_KNN_TILE * PP * sizeof(float);
  const uint32_t norm_bytes = LAGP_KNN_TILE * sizeof(float);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 && s < ntiles; ++s) {
      mbar_expect_tx(&bar[s], tile_bytes + norm_bytes);
      bulk_g2s(tile + s * LAGP_KNN_TILE * PP, Xf + (int64_t)s * LAGP_KNN_TILE * PP, tile_bytes, &bar[s]);
      bulk_g2s(tnorm + s * LAGP_KNN_TILE, nx + (int64_t)s * LAGP_KNN_TILE, norm_bytes, &bar[s]);
    }
  }

  bool timed_out = false;
  for (int64_t t = 0; t < ntiles; ++t) {
    const int st = (int)(t & 1);
    if (!mbar_wait(&bar[st], (uint32_t)((t >> 1) & 1))) {
      timed_out = true;
    }
    if (__syncthreads_or(timed_out)) {
      if (threadIdx.x == 0) {
        atomicOr(status, LAGP_DEV_TIMEOUT);
        // drain the copies still in flight into this CTA's buffers (bounded)
        mbar_wait(&bar[st], (uint32_t)((t >> 1) & 1));
        if (t + 1 < ntiles) mbar_wait(&bar[st ^ 1], (uint32_t)(((t + 1) >> 1) & 1));
      }
      __syncthreads();
      break;
    }
    const float* T = tile + st * LAGP_KNN_TILE * PP;
    const float* TN = tnorm + st * LAGP_KNN_TILE;
    const int64_t base = t * LAGP_KNN_TILE;
#pragma unroll 1
    for (int s = 0; s < LAGP_KNN_TILE / 32; ++s) {
      const int pt = s * 32 + lane;
      const int64_t gi = base + pt;
      float xv[PP];
#pragma unroll
      for (int k = 0; k < PP; k += 4) {
        float4 v4 = *reinterpret_cast<const float4*>(T + pt * PP + k);
        xv[k] = v4.x; xv[k + 1] = v4.y; xv[k + 2] = v4.z; xv[k + 3] = v4.w;
      }
      const float nxp = TN[pt];
      float d[KNN_QW];
#pragma unroll
      for (int a = 0; a < KNN_QW; ++a) {
        float dot = 0.f;
#pragma unroll
        for (int k = 0; k < PP; ++k) dot = fmaf(qf[a][k], xv[k], dot);
        d[a] = fmaf(-2.f, dot, nq[a] + nxp);
      }
#pragma unroll
      for (int a = 0; a < KNN_QW; ++a) {
        const bool pass = d[a] <= keep[a];
        uint32_t m = __ballot_sync(0xffffffffu, pass);
        if (m) {
          int pos = cnt[a] + __popc(m & ((1u << lane) - 1u));
          if (pass && pos < cap) {
            KnnEntry e; e.d = fmaxf(d[a], 0.f); e.idx = (int32_t)gi;
            buf[(q0 + a) * (int64_t)cap + pos] = e;
          }
          cnt[a] += __popc(m);
        }
      }
    }
    // compact any buffer that the next tile could overflow
#pragma unroll
    for (int a = 0; a < KNN_QW; ++a) {
      if (live[a] && cnt[a] > cap - LAGP_KNN_TILE) {
        KnnEntry* e = buf + (q0 + a) * (int64_t)cap;
        int c = min(cnt[a], cap);
        if (cnt[a] > cap) atomicOr(status, LAGP_DEV_KNN_OVERFLOW);
        __syncwarp();
        uint32_t kb = warp_select_kth(e, c, ncq[a], hist + warp * 256);
        float kth = __uint_as_float(kb);
        keep[a] = fminf(keep[a], __fadd_ru(kth, 2.f * err[a]));
        cnt[a] = warp_compact(e, c, keep[a]);
        if (cnt[a] > cap - LAGP_KNN_TILE && lane == 0) atomicOr(status, LAGP_DEV_KNN_OVERFLOW);
      }
    }
    __syncthreads();  // every warp is done with stage st
    if (threadIdx.x == 0 && t + 2 < ntiles) {
      mbar_expect_tx(&bar[st], tile_bytes + norm_bytes);
      bulk_g2s(tile + st * LAGP_KNN_TILE * PP, Xf + (t + 2) * LAGP_KNN_TILE * PP, tile_bytes, &bar[st]);
      bulk_g2s(tnorm + st * LAGP_KNN_TILE, nx + (t + 2) * LAGP_KNN_TILE, norm_bytes, &bar[st]);
    }
  }
  // final: keep d32 <= (N'-th smallest) + 2 err
#pragma unroll
  for (int a = 0; a < KNN_QW; ++a) {
    if (!live[a]) continue;
    KnnEntry* e = buf + (q0 + a) * (int64_t)cap;
    int c = min(cnt[a], cap);
    __syncwarp();
    const float thr = pilot ? pilot[q0 + a] : inf;
    if (thr < inf) {
      // the pilot threshold holds if at least N' buffered points lie at or below it
      int below = 0;
      for (int i = lane; i < c; i += 32) below += (e[i].d <= thr) ? 1 : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
      if (below < ncq[a]) {
        if (lane == 0) cnt_out[q0 + a] = -1;   // stream this location again
        continue;
      }
    }
    if (c >= ncq[a] && ncq[a] > 0) {
      uint32_t kb = warp_select_kth(e, c, ncq[a], hist + warp * 256);
      c = warp_compact(e, c, __fadd_ru(__uint_as_float(kb), 2.f * err[a]));
    }
    if (lane == 0) cnt_out[q0 + a] = timed_out ? 0 : c;
  }
}

// ---------------------------------------------------------------------------
// Exact ranking: binary64 distances in the oracle's order, bitonic sort of
// (d64, index), first N' indices out.  Distances are non-negative, so their
// IEEE bit patterns order like the values: the sort compares 64-bit integers
// (FP64 compares would run on GB300's narrow FP64 pipe).  Up to 1024 pairs
// are sorted in registers, four per thread (element 4 t + u on thread t):
// strides 1 and 2 inside a thread, 4 to 64 between the lanes of a warp by
// shuffles, 128 to 512 through shared memory.  Larger sets take the same
// network entirely in shared memory.  The real pairs are distinct (distinct
// indices), so either way the order is the unique sorted one.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool kv_less(unsigned long long ka, int32_t ia, unsigned long long kb,
                                        int32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Sorts the 1024 pairs in kr/ir (four per thread) and leaves them in order in
// key/idx[0..1024), which must hold 1024 entries; blockDim.x == 256.
__device__ __forceinline__ void rank_sort1024(unsigned long long* kr, int32_t* ir,
                                              unsigned long long* key, int32_t* idx) {
  const int t = threadIdx.x;
  for (int k = 2; k <= 1024; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      if (jj >= 4) {
        const int pt = t ^ (jj >> 2);   // the partner thread, same u
        unsigned long long pk[4];
        int32_t pi[4];
        if (jj >= 128) {                 // another warp: through shared memory
          __syncthreads();
#pragma unroll
          for (int u = 0; u < 4; ++u) { key[4 * t + u] = kr[u]; idx[4 * t + u] = ir[u]; }
          __syncthreads();
#pragma unroll
          for (int u = 0; u < 4; ++u) { pk[u] = key[4 * pt + u]; pi[u] = idx[4 * pt + u]; }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            pk[u] = __shfl_xor_sync(0xffffffffu, kr[u], jj >> 2);
            pi[u] = __shfl_xor_sync(0xffffffffu, ir[u], jj >> 2);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * t + u;
          // the lower element of an ascending pair (or the upper of a
          // descending one) keeps the smaller
          const bool keep_min = ((i & jj) == 0) == ((i & k) == 0);
          const bool p_less = kv_less(pk[u], pi[u], kr[u], ir[u]);
          if (keep_min ? p_less : !p_less) { kr[u] = pk[u]; ir[u] = pi[u]; }
        }
      } else {
        // pairs (u, u + jj) inside the thread, with constant register indices
        auto ce = [&](unsigned long long& ka, int32_t& ia, unsigned long long& kb, int32_t& ib,
                      int u) {
          const bool up = ((4 * t + u) & k) == 0;
          if (kv_less(kb, ib, ka, ia) == up) {
            const unsigned long long tk = ka; ka = kb; kb = tk;
            const int32_t ti = ia; ia = ib; ib = ti;
          }
        };
        if (jj == 2) {
          ce(kr[0], ir[0], kr[2], ir[2], 0);
          ce(kr[1], ir[1], kr[3], ir[3], 1);
        } else {
          ce(kr[0], ir[0], kr[1], ir[1], 0);
          ce(kr[2], ir[2], kr[3], ir[3], 2);
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) { key[4 * t + u] = kr[u]; idx[4 * t + u] = ir[u]; }
  __syncthreads();
}
__global__ void __launch_bounds__(256)
knn_rank(const double* __restrict__ X, int p, const double* __restrict__ xref, int64_t M,
         int nc_max, const int32_t* __restrict__ nc_loc, int cap,
         const KnnEntry* __restrict__ buf, const int32_t* __restrict__ cnt,
         int32_t* __restrict__ cand /*[M][nc_max]*/, unsigned* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_rank[];
  const int64_t q = blockIdx.x;
  if (q >= M) return;
  const int c = cnt[q];
  const int nc = nc_loc ? nc_loc[q] : nc_max;
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem_rank);
  int32_t* idx = reinterpret_cast<int32_t*>(key + cap);
  __shared__ double xq[LAGP_MAX_P];
  if (threadIdx.x < p) xq[threadIdx.x] = xref[q * p + threadIdx.x];
  int sz = 1;
  while (sz < c) sz <<= 1;
  __syncthreads();
  const KnnEntry* e = buf + q * (int64_t)cap;
  // the register form needs 1024 slots of shared memory for its exchanges
  if (sz <= 1024 && cap >= 1024 && blockDim.x == 256) {
    unsigned long long kr[4];
    int32_t ir[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = 4 * threadIdx.x + u;
      if (i < c) {
        const int32_t gi = e[i].idx;
        kr[u] = (unsigned long long)__double_as_longlong(sqdist64(X + (int64_t)gi * p, xq, p));
        ir[u] = gi;
      } else {
        kr[u] = ~0ull;
        ir[u] = 0x7fffffff;
      }
    }
    rank_sort1024(kr, ir, key, idx);
  } else {
  for (int i = threadIdx.x; i < sz; i += blockDim.x) {
    if (i < c) {
      int32_t gi = e[i].idx;
      key[i] = (unsigned long long)__double_as_longlong(sqdist64(X + (int64_t)gi * p, xq, p));
      idx[i] = gi;
    } else {
      key[i] = ~0ull;
      idx[i] = 0x7fffffff;
    }
  }
  __syncthreads();
  for (int k = 2; k <= sz; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int t = threadIdx.x; t < (sz >> 1); t += blockDim.x) {
        // t-th compare-exchange pair of this stage
        const int i = ((t & ~(jj - 1)) << 1) | (t & (jj - 1));
        const int l = i | jj;
        const bool up = (i & k) == 0;
        const unsigned long long ki = key[i], kl = key[l];
        const int32_t ii = idx[i], il = idx[l];
        const bool gt = (ki > kl) || (ki == kl && ii > il);
        if (gt == up) {
          key[i] = kl; key[l] = ki;
          idx[i] = il; idx[l] = ii;
        }
      }
      __syncthreads();
    }
  }
  }
  if (c < nc && threadIdx.x == 0) atomicOr(status, LAGP_DEV_KNN_OVERFLOW);
  // ranks this location lacks (a flagged overflow or timeout) repeat a valid
  // index, so that the design kernels never read outside the design
  const int32_t fill = c > 0 ? idx[0] : 0;
  for (int r = threadIdx.x; r < nc_max; r += blockDim.x)
    cand[q * nc_max + r] = (r < nc) ? (r < c ? idx[r] : fill) : -1;
}

// ---------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------
size_t knn_smem_stream(int PP) {
  return (size_t)2 * LAGP_KNN_TILE * PP * 4 + 2 * LAGP_KNN_TILE * 4 + KNN_WARPS * 256 * 4 + 16;
}

// Buffer entries per location: room for N' survivors, a whole tile of new
// inserts before the next compaction, and N'/2 (at least 64) entries of slack
// for distances within the error margin of the N'-th.  A power of two, as the
// bitonic sort of knn_rank wants.
int knn_cap(int nc_max) {
  // with the pilot threshold about 2.2 N' points are admitted
  const int need = (5 * nc_max) / 2 + LAGP_KNN_TILE;
  int cap = 512;
  while (cap < need) cap <<= 1;
  return cap;
}

cudaError_t launch_prepare(const double* X, int64_t N, int p, int PP, int64_t Npad,
                           const Workspace& ws, cudaStream_t s) {
  const int parts = 64;
  prof_begin("bbox_partial", s);
  bbox_partial<<<parts, 256, 0, s>>>(X, N, p, ws.bbox_part);
  prof_end(s);
  prof_begin("bbox_final", s);
  bbox_final<<<1, 32, 0, s>>>(ws.bbox_part, parts, p, ws.lo, ws.hi, ws.center);
  prof_end(s);
  cudaMemsetAsync(ws.maxn2, 0, sizeof(unsigned), s);
  prof_begin("design_to_f32", s);
  design_to_f32<<<1216, 256, 0, s>>>(X, N, Npad, p, PP, ws.center, ws.Xf, ws.nx, ws.maxn2);
  prof_end(s);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if ((err = launch_design_to_tc(N, p, PP, Npad, ws, s)) != cudaSuccess) return err;
  // the k-d tree of the unlimited ray scope, when the workspace has one
  return ws.kd.perm ? launch_kd_build(X, ws.Xf, N, p, PP, ws.kd, s) : cudaSuccess;
}

cudaError_t launch_knn(const double* X, int64_t N, int p, int PP, int64_t Npad,
                       const double* xref, int64_t M, int nc_max, const int32_t* nc_loc,
                       int32_t* cand, const Workspace& ws, cudaStream_t s) {
  const int cap = knn_cap(nc_max);
  const int64_t ntiles = Npad / LAGP_KNN_TILE;
  const int qpb = KNN_WARPS * KNN_QW;
  dim3 grid((unsigned)((M + qpb - 1) / qpb));
  size_t sm = knn_smem_stream(PP);
  // pilot thresholds where the design is large against N'
  const bool pilot = N >= (int64_t)32 * nc_max;
  const int64_t S = N / 16 < 32768 ? N / 16 : 32768;
  KnnEntry* kbuf = reinterpret_cast<KnnEntry*>(ws.knn_buf);
  cudaError_t err;
  switch (PP) {
#define KNN_CASE(V)                                                                          \
  case V:                                                                                    \
    err = cudaFuncSetAttribute(knn_stream<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                               (int)sm);                                                     \
    if (err != cudaSuccess) return err;                                                      \
    if (pilot) {                                                                             \
      prof_begin("knn_pilot", s);                                                            \
      knn_pilot<V><<<grid, KNN_WARPS * 32, 0, s>>>(ws.Xf, ws.nx, N, S, p, xref, M, ws.center, \
                                                   nc_max, nc_loc, cap, ws.knn_thr);         \
      prof_end(s);                                                                           \
    }                                                                                        \
    if (pilot) {                                                                             \
      err = launch_knn_tc(Npad, p, xref, M, nc_max, nc_loc, cap, ws, s);                     \
      if (err != cudaSuccess) return err;                                                    \
    } else {                                                                                 \
      prof_begin("knn_stream", s);                                                           \
      knn_stream<V><<<grid, KNN_WARPS * 32, sm, s>>>(ws.Xf, ws.nx, N, ntiles, p, xref, M,    \
                                                     ws.center, ws.maxn2, nc_max, nc_loc,    \
                                                     cap, kbuf, ws.knn_cnt, ws.status,       \
                                                     nullptr, 0);                            \
      prof_end(s);                                                                           \
    }                                                                                        \
    if (pilot) {                                                                             \
      prof_begin("knn_stream_redo", s);                                                      \
      knn_stream<V><<<grid, KNN_WARPS * 32, sm, s>>>(ws.Xf, ws.nx, N, ntiles, p, xref, M,    \
                                                     ws.center, ws.maxn2, nc_max, nc_loc,    \
                                                     cap, kbuf, ws.knn_cnt, ws.status,       \
                                                     nullptr, 1);                            \
      prof_end(s);                                                                           \
    }                                                                                        \
    break;
    KNN_CASE(4)
    KNN_CASE(8)
    KNN_CASE(12)
    KNN_CASE(16)
#undef KNN_CASE
    default:
      return cudaErrorInvalidValue;
  }
  size_t smr = (size_t)cap * (8 + 4);
  err = cudaFuncSetAttribute(knn_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
  if (err != cudaSuccess) return err;
  prof_begin("knn_rank", s);
  knn_rank<<<(unsigned)M, 256, smr, s>>>(X, p, xref, M, nc_max, nc_loc, cap,
                                         reinterpret_cast<const KnnEntry*>(ws.knn_buf),
                                         ws.knn_cnt, cand, ws.status);
  prof_end(s);
  return cudaGetLastError();
}

}  // namespace lagp
