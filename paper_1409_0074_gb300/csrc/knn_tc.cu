// knn_tc.cu -- kNN candidate filter with the distances on the tensor cores
// (Gramacy & Haaland, Sec 2.2: the local search is restricted to the N'
// nearest neighbours of x), used where the pilot thresholds apply (N >= 32 N').
//
// Squared distances as one contraction.  With centred FP32 coordinates a
// (location) and b (design point),
//     |a - b|^2 = sum_i (-2 a_i) b_i + |a|^2 * 1 + 1 * |b|^2,
// so a location row A = [-2a, |a|^2, 1, 0..] times a design row
// B = [b, 1, |b|^2, 0..] (K = p + 2 rounded up to a multiple of 8) is the
// distance.  Both operands are split into TF32 hi + lo and the product is
// hi*hi + hi*lo + lo*hi with FP32 accumulation in TMEM (3xTF32).
//
// CTA = 128 locations (MMA M = 128, one TMEM lane each); the design streams in
// 128-point tiles (MMA N = 128), prepared once per design in the tensor
// cores' canonical K-major layout so that a tile is one bulk copy.
//   warp 16     producer: bulk copies into a 6-stage shared-memory ring
//   warp 17     MMA issuer: 3 K/8 tcgen05.mma per tile into one of four TMEM
//               accumulators of 128 columns
//   warps 0-15  epilogue, four groups of four warps; group g takes the tiles
//               t = g mod 4 from accumulator g.  A thread owns one location
//               (its TMEM lane), reads the tile's 128 distances with
//               tcgen05.ld and compares them with its own threshold; a point
//               that passes is appended to the location's buffer.  Groups of
//               four distances with no pass in any lane of the warp (the
//               common case) are skipped after one minimum and one vote.
// The threshold is the pilot's estimate of the N'-th distance plus 2 err and
// stays fixed, so the buffer needs no compaction during the stream.  Each
// epilogue group appends to its own quarter of the location's buffer with a
// counter in a register (no atomics in the stream).  At the end a location is
// valid when at least N' of its entries lie at or below the pilot value and no
// quarter overflowed; otherwise it is marked for the streaming kernel's exact
// pass (threshold infinity).  knn_finalize joins the quarters and keeps the
// entries within the N'-th smallest + 2 err for the exact ranking.
// A batch with fewer location tiles than SMs splits the design into segments,
// one CTA each (grid y); the segments of a location append to its buffer
// through a global counter (passes are rare), and knn_tc_join decides its
// validity once all of them are done.  The buffered set is the same.  A larger
// batch runs whole waves of one CTA per SM unsplit and splits only the tiles
// of its last, partial wave, so that they spread over the SMs that would
// otherwise idle.
//
// err bounds |d_tc - d64| for the 3xTF32 contraction: operand splitting
// (3 * 2^-22 |A_k B_k| per term), FP32 accumulation over 3K products
// (2^-23 of the running sum each) and FP32 input rounding, all bounded by
// multiples of (|a| + |b|)^2; (K + 16) 2^-21 (|a| + |b|)^2, with a 25% margin.
// Every wait is bounded; a timeout sets LAGP_DEV_TIMEOUT and all roles stop.
#include <cstdint>

#include "common.cuh"
#include "knn_common.cuh"
#include "lagp_internal.h"
#include "launch_plan.h"

namespace lagp {

#define KT_M 128          // locations per CTA (MMA M)
#define KT_N 128          // design points per tile (MMA N)
#define KT_GROUPS 4       // epilogue groups = TMEM accumulators
#define KT_EPI_WARPS (4 * KT_GROUPS)
#define KT_THREADS (KT_EPI_WARPS * 32 + 64)
#define KT_STAGES 6
#define KT_EPI_BAR 1      // named barrier of the epilogue warps

__host__ __device__ __forceinline__ int kt_ka(int p) { return (p + 2 + 7) & ~7; }

// byte offset of (row, k) in the canonical no-swizzle K-major layout: 8-row x
// 16-byte core matrices; the KA/4 k-chunks of a row group are adjacent (128
// bytes apart), row groups KA/4 * 128 bytes apart.
__host__ __device__ __forceinline__ uint32_t kt_canon(int row, int k, int KA) {
  return (uint32_t)((row >> 3) * ((KA >> 2) * 128) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float kt_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

__device__ __forceinline__ float kt_err(int KA, float r) {
  return (float)(KA + 16) * 0x1p-21f * 1.25f * r * r;
}

// Design tiles [tile][hi | lo][KT_N rows x KA] in canonical order from the
// centred FP32 copy: row i = [Xf_i, 1, |Xf_i|^2, 0..]; rows past N are
// [0.., 0, 1e30, 0..] (distance 1e30: they never pass).
__global__ void design_to_tc(const float* __restrict__ Xf, const float* __restrict__ nx, int64_t N,
                             int64_t Npad, int p, int PP, int KA, float* __restrict__ out) {
  const int64_t total = Npad * KA;
  const int64_t tile_floats = (int64_t)KT_N * KA;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / KA;
    const int k = (int)(e - i * KA);
    float v = 0.f;
    if (i < N) {
      if (k < p) v = Xf[i * PP + k];
      else if (k == p) v = 1.f;
      else if (k == p + 1) v = nx[i];
    } else if (k == p + 1) {
      v = 1e30f;
    }
    const float hi = kt_tf32(v);
    const float lo = kt_tf32(v - hi);
    const int64_t t = i / KT_N;
    const uint32_t off = kt_canon((int)(i - t * KT_N), k, KA) >> 2;
    out[t * 2 * tile_floats + off] = hi;
    out[t * 2 * tile_floats + tile_floats + off] = lo;
  }
}

__device__ __forceinline__ uint64_t kt_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((128u >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void kt_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void kt_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void kt_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void kt_epi_barrier() {
  asm volatile("bar.sync %0, %1;" ::"n"(KT_EPI_BAR), "n"(KT_EPI_WARPS * 32) : "memory");
}

// 64 columns of this thread's TMEM lane: two 32-column loads, one wait
__device__ __forceinline__ void kt_ld32x2(uint32_t addr, uint32_t (&v)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(addr));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]),
        "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]),
        "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]),
        "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
        "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]),
        "=r"(v[62]), "=r"(v[63])
      : "r"(addr + 32));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int KA>
struct KtSmem {
  static constexpr int A_BYTES = KT_M * KA * 4;        // location operand, one of hi / lo
  static constexpr int TILE_BYTES = KT_N * KA * 4;     // design tile, one of hi / lo
  static constexpr int STAGE_BYTES = 2 * TILE_BYTES;
  static constexpr int A_OFF = 0;
  static constexpr int S_OFF = 2 * A_BYTES;
  static constexpr int KEEP_OFF = S_OFF + KT_STAGES * STAGE_BYTES;
  static constexpr int THR_OFF = KEEP_OFF + KT_M * 4;
  static constexpr int CNT_OFF = THR_OFF + KT_M * 4;            // [KT_GROUPS][KT_M]
  static constexpr int BELOW_OFF = CNT_OFF + KT_GROUPS * KT_M * 4;
  static constexpr int BAR_OFF = BELOW_OFF + KT_M * 4;
  static constexpr int MISC_OFF = BAR_OFF + (2 * KT_STAGES + 2 * KT_GROUPS) * 8;
  // + alignment slack; at least 120 KB so that one CTA (which takes all 512
  // TMEM columns) is resident per SM
  static constexpr int BYTES = (MISC_OFF + 16 + 1024) > 120 * 1024 ? (MISC_OFF + 16 + 1024)
                                                                   : 120 * 1024;
};

template <int KA, bool SPLIT>
__global__ void __launch_bounds__(KT_THREADS, 1)
knn_tc(const float* __restrict__ Btiles, int64_t ntiles, int p, const double* __restrict__ xref,
       int64_t M, const double* __restrict__ center, const unsigned* __restrict__ maxn2_bits,
       int nc_max, const int32_t* __restrict__ nc_loc, int cap, const float* __restrict__ pilot,
       KnnEntry* __restrict__ buf, int32_t* __restrict__ cnt_out, int32_t* __restrict__ seg_out,
       unsigned* __restrict__ status, int64_t tile0) {
  using L = KtSmem<KA>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* Ahi = reinterpret_cast<float*>(smem + L::A_OFF);
  float* Alo = reinterpret_cast<float*>(smem + L::A_OFF + L::A_BYTES);
  float* keep_sm = reinterpret_cast<float*>(smem + L::KEEP_OFF);
  float* thr_sm = reinterpret_cast<float*>(smem + L::THR_OFF);
  int* cnt_sm = reinterpret_cast<int*>(smem + L::CNT_OFF);
  int* below_sm = reinterpret_cast<int*>(smem + L::BELOW_OFF);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + KT_STAGES;
  uint64_t* tfull = empty + KT_STAGES;
  uint64_t* tempty = tfull + KT_GROUPS;
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(smem + L::MISC_OFF);
  int* abort_flag = reinterpret_cast<int*>(smem + L::MISC_OFF + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t q0 = (tile0 + (int64_t)blockIdx.x) * KT_M;
  // design segment of this CTA: tiles [t_lo, t_lo + nt) (the whole design
  // unless the launch splits it over gridDim.y CTAs per location tile)
  const int64_t t_lo = SPLIT ? (int64_t)blockIdx.y * ntiles / gridDim.y : 0;
  const int64_t nt = SPLIT ? (int64_t)(blockIdx.y + 1) * ntiles / gridDim.y - t_lo : ntiles;
  const float rdes = sqrtf(__uint_as_float(*maxn2_bits)) * 1.0001f;
  const float inf = __int_as_float(0x7f800000);

  // ---- per-location state and operand A = [-2a, |a|^2, 1, 0..] ----
  for (int c = tid; c < KT_M; c += blockDim.x) {
    const int64_t q = q0 + c;
    float qn = 0.f;
    if (q < M)
      for (int k = 0; k < p; ++k) {
        const float a = (float)(xref[q * p + k] - center[k]);
        qn = fmaf(a, a, qn);
      }
    const float r = rdes + sqrtf(qn) * 1.0001f;
    const float thr = q < M ? pilot[q] : inf;
    // no pilot value: nothing is buffered and the exact pass takes the location
    thr_sm[c] = thr;
    keep_sm[c] = thr < inf ? __fadd_ru(thr, 2.f * kt_err(KA, r)) : -1.f;
    below_sm[c] = 0;
  }
  for (int e = tid; e < KT_M * KA; e += blockDim.x) {
    const int c = e / KA, k = e - c * KA;
    const int64_t q = q0 + c;
    float v = 0.f;
    if (q < M) {
      if (k < p) {
        v = -2.f * (float)(xref[q * p + k] - center[k]);
      } else if (k == p) {
        float acc = 0.f;
        for (int i = 0; i < p; ++i) {
          const float a = (float)(xref[q * p + i] - center[i]);
          acc = fmaf(a, a, acc);
        }
        v = acc;
      } else if (k == p + 1) {
        v = 1.f;
      }
    }
    const float hi = kt_tf32(v);
    const uint32_t off = kt_canon(c, k, KA) >> 2;
    Ahi[off] = hi;
    Alo[off] = kt_tf32(v - hi);
  }
  if (tid == 0) {
    for (int s = 0; s < KT_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < KT_GROUPS; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 128); }
    *abort_flag = 0;
    fence_mbar_init();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tmem_base;
  volatile int* abort_v = abort_flag;

  if (warp == KT_EPI_WARPS) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t t = 0; t < nt; ++t) {
        const int s = (int)(t % KT_STAGES);
        if (t >= KT_STAGES) {
          if (*abort_v || !mbar_wait(&empty[s], (uint32_t)(((t / KT_STAGES) - 1) & 1))) {
            *abort_v = 1;
            break;
          }
        }
        mbar_expect_tx(&full[s], L::STAGE_BYTES);
        bulk_g2s(smem + L::S_OFF + s * L::STAGE_BYTES,
                 Btiles + (t_lo + t) * (int64_t)(L::STAGE_BYTES / 4), L::STAGE_BYTES, &full[s]);
        issued = t + 1;
      }
      if (*abort_v) {   // copies in flight land before the CTA can exit
        for (int64_t t = issued > KT_STAGES ? issued - KT_STAGES : 0; t < issued; ++t)
          mbar_wait(&full[t % KT_STAGES], (uint32_t)((t / KT_STAGES) & 1));
      }
    }
  } else if (warp == KT_EPI_WARPS + 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KT_N >> 3) << 17) |
                             ((uint32_t)(KT_M >> 4) << 24);
      const uint32_t sbo = (KA / 4) * 128;
      const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo);
      int64_t committed = 0;
      for (int64_t t = 0; t < nt; ++t) {
        const int s = (int)(t % KT_STAGES), b = (int)(t % KT_GROUPS);
        bool ok = !*abort_v && mbar_wait(&full[s], (uint32_t)((t / KT_STAGES) & 1));
        if (ok && t >= KT_GROUPS)
          ok = !*abort_v && mbar_wait(&tempty[b], (uint32_t)(((t / KT_GROUPS) - 1) & 1));
        if (!ok) { *abort_v = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t b_hi = smem_u32(smem + L::S_OFF + s * L::STAGE_BYTES);
        const uint32_t b_lo = b_hi + L::TILE_BYTES;
        const uint32_t d = taddr + (uint32_t)(b * KT_N);
#pragma unroll
        for (int ks = 0; ks < KA / 8; ++ks) {
          const uint32_t ko = ks * 256;
          kt_mma(d, kt_desc(a_hi + ko, sbo), kt_desc(b_hi + ko, sbo), idesc, ks > 0 ? 1u : 0u);
          kt_mma(d, kt_desc(a_hi + ko, sbo), kt_desc(b_lo + ko, sbo), idesc, 1u);
          kt_mma(d, kt_desc(a_lo + ko, sbo), kt_desc(b_hi + ko, sbo), idesc, 1u);
        }
        kt_commit(&empty[s]);
        kt_commit(&tfull[b]);
        committed = t + 1;
      }
      if (*abort_v && committed > 0) {   // the last MMAs finish before TMEM is freed
        const int64_t t = committed - 1;
        mbar_wait(&tfull[t % KT_GROUPS], (uint32_t)((t / KT_GROUPS) & 1));
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int g = warp >> 2, quarter = warp & 3;
    const int c = quarter * 32 + lane;                     // this thread's location
    const int64_t q = q0 + c;
    const uint32_t lane_base = taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * KT_N);
    const float keep = keep_sm[c], thr = thr_sm[c];
    const int seg = cap / KT_GROUPS;                       // this group's quarter of the buffer
    KnnEntry* qb = buf + q * (int64_t)cap + g * seg;
    int mycnt = 0, mybelow = 0;
    for (int64_t t = g; t < nt; t += KT_GROUPS) {
      const bool ok = !*abort_v && mbar_wait(&tfull[g], (uint32_t)((t / KT_GROUPS) & 1));
      if (!__all_sync(0xffffffffu, ok)) *abort_v = 1;
      if (*abort_v) {
        // still release the accumulator so that no role waits on it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        kt_arrive(&tempty[g]);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int32_t pbase = (int32_t)((t_lo + t) * KT_N);
#pragma unroll 1
      for (int c0 = 0; c0 < KT_N; c0 += 64) {
        // two 32-column loads, one wait
        uint32_t v[64];
        kt_ld32x2(lane_base + c0, v);
        if (c0 == KT_N - 64) {
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          kt_arrive(&tempty[g]);
        }
#pragma unroll
        for (int u4 = 0; u4 < 64; u4 += 4) {
          // at a pass rate of ~0.2%, most 4-value groups hold no pass in any
          // lane of the warp: the group's minimum, one vote, and the group is
          // skipped without a compare and branch per value
          const float m4 = fminf(fminf(__uint_as_float(v[u4]), __uint_as_float(v[u4 + 1])),
                                 fminf(__uint_as_float(v[u4 + 2]), __uint_as_float(v[u4 + 3])));
          if (!__any_sync(0xffffffffu, m4 <= keep)) continue;
#pragma unroll
          for (int u = u4; u < u4 + 4; ++u) {
            const float d = __uint_as_float(v[u]);
            if (d <= keep) {
              if (SPLIT) {
                // segments of one location share its buffer through a counter
                KnnEntry e;
                e.d = fmaxf(d, 0.f);
                e.idx = pbase + c0 + u;
                const int slot = atomicAdd(&seg_out[q * KT_GROUPS], 1);
                if (slot < cap) buf[q * (int64_t)cap + slot] = e;
              } else if (mycnt < seg) {
                KnnEntry e;
                e.d = fmaxf(d, 0.f);
                e.idx = pbase + c0 + u;
                qb[mycnt] = e;
              }
              ++mycnt;
              mybelow += (d <= thr) ? 1 : 0;
            }
          }
        }
      }
    }
    cnt_sm[g * KT_M + c] = mycnt;
    atomicAdd(&below_sm[c], mybelow);
    kt_epi_barrier();
    if (SPLIT) {
      // the location's totals come together in knn_tc_join once every
      // segment is done
      if (g == 0 && q < M && below_sm[c] > 0) atomicAdd(&seg_out[q * KT_GROUPS + 1], below_sm[c]);
    } else if (g == 0 && q < M) {
      const int nc = nc_loc ? nc_loc[q] : nc_max;
      int n = 0;
      bool over = false;
      for (int gg = 0; gg < KT_GROUPS; ++gg) {
        const int k = cnt_sm[gg * KT_M + c];
        over = over || k > seg;
        seg_out[q * KT_GROUPS + gg] = k;
        n += k;
      }
      // valid: no overflow and at least N' entries at or below the pilot value
      cnt_out[q] = (*abort_v) ? 0 : ((!over && below_sm[c] >= nc && thr < inf) ? n : -1);
    }
  }
  if (tid == 0 && *abort_v) atomicOr(status, LAGP_DEV_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr));
  }
}

// After a split launch: a location is valid when its buffer did not overflow
// and at least N' of its entries lie at or below the pilot value; its entries
// are then the first count of the buffer (one quarter, as finalize reads it).
__global__ void knn_tc_join(int64_t q_begin, int64_t M, int nc_max,
                            const int32_t* __restrict__ nc_loc, int cap,
                            const float* __restrict__ pilot, int32_t* __restrict__ cnt,
                            int32_t* __restrict__ seg, const unsigned* __restrict__ status) {
  const int64_t q = q_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= M) return;
  const int total = seg[q * KT_GROUPS], below = seg[q * KT_GROUPS + 1];
  const int nc = nc_loc ? nc_loc[q] : nc_max;
  const bool thr_ok = pilot[q] < __int_as_float(0x7f800000);
  // after a timed-out stream (status already set) nothing of it is kept
  cnt[q] = (*status & LAGP_DEV_TIMEOUT) ? 0
                                        : ((total <= cap && below >= nc && thr_ok) ? total : -1);
  seg[q * KT_GROUPS] = total <= cap ? total : cap;
  seg[q * KT_GROUPS + 1] = 0;
  seg[q * KT_GROUPS + 2] = 0;
  seg[q * KT_GROUPS + 3] = 0;
}

// Keep, per valid location, the buffered entries within the N'-th smallest
// distance + 2 err (one warp per location); invalid locations (-1) are left to
// the exact pass.
__global__ void __launch_bounds__(256)
knn_finalize(const double* __restrict__ xref, int64_t M, int p, int KA,
             const double* __restrict__ center, const unsigned* __restrict__ maxn2_bits,
             int nc_max, const int32_t* __restrict__ nc_loc, int cap, KnnEntry* __restrict__ buf,
             int32_t* __restrict__ cnt, const int32_t* __restrict__ seg_cnt) {
  __shared__ uint32_t hist[8][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * 8 + warp;
  if (q >= M) return;
  const int c = cnt[q];
  const int nc = nc_loc ? nc_loc[q] : nc_max;
  if (c < 0 || c < nc || nc <= 0) return;
  float qn = 0.f;
  for (int k = 0; k < p; ++k) {
    const float a = (float)(xref[q * p + k] - center[k]);
    qn = fmaf(a, a, qn);
  }
  const float r = sqrtf(__uint_as_float(*maxn2_bits)) * 1.0001f + sqrtf(qn) * 1.0001f;
  KnnEntry* e = buf + q * (int64_t)cap;
  // join the quarters: quarter g (count k_g) moves down to the end of the
  // entries before it; reading a chunk before writing it keeps the forward
  // copy safe (the destination never passes the source)
  const int seg = cap / KT_GROUPS;
  int at = seg_cnt[q * KT_GROUPS];
  for (int g = 1; g < KT_GROUPS; ++g) {
    const int k = seg_cnt[q * KT_GROUPS + g];
    for (int b0 = 0; b0 < k; b0 += 32) {
      KnnEntry v;
      const bool in = b0 + lane < k;
      if (in) v = e[g * seg + b0 + lane];
      __syncwarp();
      if (in) e[at + b0 + lane] = v;
      __syncwarp();
    }
    at += k;
  }
  const uint32_t kb = warp_select_kth(e, c, nc, hist[warp]);
  const int nn = warp_compact(e, c, __fadd_ru(__uint_as_float(kb), 2.f * kt_err(KA, r)));
  if (lane == 0) cnt[q] = nn;
}

size_t knn_tc_tile_floats(int64_t Npad, int p) { return (size_t)Npad * kt_ka(p) * 2; }

cudaError_t launch_design_to_tc(int64_t N, int p, int PP, int64_t Npad, const Workspace& ws,
                                cudaStream_t s) {
  prof_begin("design_to_tc", s);
  design_to_tc<<<1216, 256, 0, s>>>(ws.Xf, ws.nx, N, Npad, p, PP, kt_ka(p), ws.Btc);
  prof_end(s);
  return cudaGetLastError();
}

cudaError_t launch_knn_tc(int64_t Npad, int p, const double* xref, int64_t M, int nc_max,
                          const int32_t* nc_loc, int cap, const Workspace& ws, cudaStream_t s) {
  const int KA = kt_ka(p);
  const int64_t ntiles = Npad / KT_N;
  const int64_t tiles = (M + KT_M - 1) / KT_M;
  KnnEntry* kbuf = reinterpret_cast<KnnEntry*>(ws.knn_buf);
  cudaError_t err;
  int sms = 0, dev = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return err;
  // whole waves unsplit, the rest split over the SMs (launch_plan.h)
  int64_t body = tiles, nseg = 1;
  knn_tc_plan(tiles, sms, ntiles, &body, &nseg);
  const int64_t rest = tiles - body, q_split = body * KT_M;
  if (rest > 0 && (err = cudaMemsetAsync(ws.knn_seg + KT_GROUPS * q_split, 0,
                                         sizeof(int32_t) * KT_GROUPS * (M - q_split), s)) !=
                      cudaSuccess)
    return err;
  switch (KA) {
#define KT_CASE(V)                                                                              \
  case V: {                                                                                     \
    const size_t sm = KtSmem<V>::BYTES;                                                         \
    for (int part = 0; part < 2; ++part) {                                                      \
      const int64_t n_part = part == 0 ? body : rest;                                           \
      if (n_part == 0) continue;                                                                \
      auto kern = part == 0 ? knn_tc<V, false> : knn_tc<V, true>;                               \
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);   \
      if (err != cudaSuccess) return err;                                                       \
      const dim3 g3((unsigned)n_part, part == 0 ? 1u : (unsigned)nseg);                         \
      prof_begin("knn_tc", s);                                                                  \
      kern<<<g3, KT_THREADS, sm, s>>>(ws.Btc, ntiles, p, xref, M, ws.center, ws.maxn2, nc_max,  \
                                      nc_loc, cap, ws.knn_thr, kbuf, ws.knn_cnt, ws.knn_seg,    \
                                      ws.status, part == 0 ? 0 : body);                         \
      prof_end(s);                                                                              \
    }                                                                                           \
    break;                                                                                      \
  }
    KT_CASE(8)
    KT_CASE(16)
    KT_CASE(24)
#undef KT_CASE
    default:
      return cudaErrorInvalidValue;
  }
  if (rest > 0) {
    prof_begin("knn_tc_join", s);
    knn_tc_join<<<(unsigned)((M - q_split + 255) / 256), 256, 0, s>>>(
        q_split, M, nc_max, nc_loc, cap, ws.knn_thr, ws.knn_cnt, ws.knn_seg, ws.status);
    prof_end(s);
  }
  prof_begin("knn_finalize", s);
  knn_finalize<<<(unsigned)((M + 7) / 8), 256, 0, s>>>(xref, M, p, KA, ws.center, ws.maxn2,
                                                       nc_max, nc_loc, cap, kbuf, ws.knn_cnt,
                                                       ws.knn_seg);
  prof_end(s);
  return cudaGetLastError();
}

}  // namespace lagp
