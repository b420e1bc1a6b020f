// common.cuh -- device helpers shared by the CUDA kernels of the laGP library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define LAGP_MAX_P 16        // input dimension limit
#define LAGP_MAX_N 128       // local design size limit
#define LAGP_MAX_RAYS 16     // rays per greedy step limit
#define LAGP_KNN_TILE 256    // design points per streamed kNN tile

// Device status bits (written with atomicOr into the workspace status word).
#define LAGP_DEV_TIMEOUT 1u        // a bounded wait ran out
#define LAGP_DEV_KNN_OVERFLOW 2u   // more tied kNN candidates than the buffer holds
#define LAGP_DEV_BAD_UPDATE 4u     // a Schur complement v <= 0 (location gets NaN)

// Bound of every mbarrier wait, in SM clock cycles (about 2 s at 2 GHz).
#define LAGP_WAIT_CYCLES 4000000000ll

// Smallest binary64 pivot below which an FP32-scoring location is solved
// again in binary64 under precision promotion (the reasoning is with
// LAGP_PROMOTE in lagp.h).
#define LAGP_PROMOTE_PIVOT_DEV 3e-5

namespace lagp {

// Precision promotion: one thread per location appends `loc` to the list
// of binary64 re-solves when the smallest pivot v of its local design is below
// the threshold (or not a number).  count[0] indexes the list of this launch,
// count[1] totals the call.  list == null: promotion is off.
__device__ __forceinline__ void promote_location(int32_t* list, unsigned* count, int64_t loc,
                                                 double vmin) {
  if (list && !(vmin >= LAGP_PROMOTE_PIVOT_DEV)) {
    list[atomicAdd(count, 1u)] = (int32_t)loc;
    atomicAdd(count + 1, 1u);
  }
}

// exp(x) in binary64 by Cody & Waite (1980) argument reduction x = k ln2 + r,
// |r| <= ln2/2, the degree-13 Taylor polynomial of e^r by Horner's rule, and an
// exact scaling by 2^k.  Results below the normal range (x < -708) are 0.
// Every operation is an explicitly rounded multiply or add, so the value does
// not depend on compiler contraction.  The FP64 parity path uses it so that
// correlations are reproducible bit for bit on any IEEE-754 machine.
__device__ __forceinline__ double exp_cw(double x) {
  if (x != x) return x;
  if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
  if (x < -708.0) return 0.0;
  const double inv_ln2 = 0x1.71547652b82fep+0;
  const double ln2_hi = 0x1.62e42fee00000p-1;
  const double ln2_lo = 0x1.a39ef35793c76p-33;
  double kd = rint(__dmul_rn(x, inv_ln2));
  double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kd, ln2_hi)), __dmul_rn(kd, ln2_lo));
  double s = 1.0 / 6227020800.0;
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 479001600.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 39916800.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 3628800.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 362880.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 40320.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 5040.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 720.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 120.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 24.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0 / 6.0);
  s = __dadd_rn(__dmul_rn(s, r), 0.5);
  s = __dadd_rn(__dmul_rn(s, r), 1.0);
  s = __dadd_rn(__dmul_rn(s, r), 1.0);
  return ldexp(s, (int)kd);
}

// Squared distance in binary64, ascending coordinate order, no contraction.
__device__ __forceinline__ double sqdist64(const double* a, const double* b, int p) {
  double acc = 0.0;
  for (int k = 0; k < p; ++k) {
    double t = __dsub_rn(a[k], b[k]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

// Squared distance in binary32 between a row of the FP32 design copy (global,
// 16-byte aligned, PP a multiple of 4: read as float4) and any PP floats, in
// ascending coordinate order with one FMA per coordinate.
__device__ __forceinline__ float sqdist_row32(const float* __restrict__ row, const float* b, int PP) {
  float d = 0.f;
  for (int k = 0; k < PP; k += 4) {
    const float4 c = *reinterpret_cast<const float4*>(row + k);
    float t = c.x - b[k]; d = fmaf(t, t, d);
    t = c.y - b[k + 1]; d = fmaf(t, t, d);
    t = c.z - b[k + 2]; d = fmaf(t, t, d);
    t = c.w - b[k + 3]; d = fmaf(t, t, d);
  }
  return d;
}

// Isotropic Gaussian correlation exp(-||a-b||^2 / theta) in binary64.
__device__ __forceinline__ double corr64(const double* a, const double* b, int p, double theta) {
  return exp_cw(-(__ddiv_rn(sqdist64(a, b, p), theta)));
}

// exp(x) in binary64 for x <= 0 by the same method as exp_cw (Cody-Waite
// reduction, degree-13 Taylor polynomial on |r| <= ln2/2, scaling by 2^k),
// evaluated with fused multiply-adds: a few ulp, and about half the FP64
// instructions of exp_cw.  Results below the normal range are 0.
__device__ __forceinline__ double exp_neg_fma(double x) {
  if (x < -708.0) return 0.0;
  const double inv_ln2 = 0x1.71547652b82fep+0;
  const double ln2_hi = 0x1.62e42fee00000p-1;
  const double ln2_lo = 0x1.a39ef35793c76p-33;
  const double kd = rint(x * inv_ln2);
  double r = fma(-kd, ln2_hi, x);
  r = fma(-kd, ln2_lo, r);
  double s = 1.0 / 6227020800.0;
  s = fma(s, r, 1.0 / 479001600.0);
  s = fma(s, r, 1.0 / 39916800.0);
  s = fma(s, r, 1.0 / 3628800.0);
  s = fma(s, r, 1.0 / 362880.0);
  s = fma(s, r, 1.0 / 40320.0);
  s = fma(s, r, 1.0 / 5040.0);
  s = fma(s, r, 1.0 / 720.0);
  s = fma(s, r, 1.0 / 120.0);
  s = fma(s, r, 1.0 / 24.0);
  s = fma(s, r, 1.0 / 6.0);
  s = fma(s, r, 0.5);
  s = fma(s, r, 1.0);
  s = fma(s, r, 1.0);
  // 2^k with k in [-1022, 0]: add k to the exponent field of s (s in [0.7, 1.5])
  return __longlong_as_double(__double_as_longlong(s) + (long long)(int)kd * (1ll << 52));
}

// Correlation in binary64 for the FP32-scoring form's factor update: the same
// quantity as corr64, with FMA contraction and a multiply by -1/theta instead
// of the division (no bit-exactness with the oracle is needed there, only
// binary64 accuracy).
__device__ __forceinline__ double corr64_fast(const double* a, const double* b, int p,
                                              double neg_inv_theta) {
  double d0 = 0.0, d1 = 0.0;
  int k = 0;
  for (; k + 1 < p; k += 2) {
    const double t0 = a[k] - b[k], t1 = a[k + 1] - b[k + 1];
    d0 = fma(t0, t0, d0);
    d1 = fma(t1, t1, d1);
  }
  if (k < p) { const double t = a[k] - b[k]; d0 = fma(t, t, d0); }
  return exp_neg_fma((d0 + d1) * neg_inv_theta);
}

// sum_{k=0..len-1} u[k] * v[k] in binary64 with eight independent accumulators,
// so that eight loads of u (global memory) are in flight at a time and no
// single FMA chain sets the pace (GB300's FP64 and L2 latencies).
__device__ __forceinline__ double dot64_ilp8(const double* u, const double* v, int len) {
  double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int k = 0;
  for (; k + 7 < len; k += 8) {
#pragma unroll
    for (int t = 0; t < 8; ++t) a[t] = fma(u[k + t], v[k + t], a[t]);
  }
  for (; k < len; ++k) a[0] = fma(u[k], v[k], a[0]);
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// sum_{i=k..j-1} u[i] * M[i * ld + k] (a column of a row-major matrix) in
// binary64, eight accumulators as above
__device__ __forceinline__ double coldot64_ilp8(const double* u, const double* M, int64_t ld, int k,
                                                int j) {
  double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int i = k;
  for (; i + 7 < j; i += 8) {
#pragma unroll
    for (int t = 0; t < 8; ++t) a[t] = fma(u[i + t], M[(int64_t)(i + t) * ld + k], a[t]);
  }
  for (; i < j; ++i) a[0] = fma(u[i], M[(int64_t)i * ld + k], a[0]);
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// sum_{k=0..len-1} u[k] * v[k] in binary64 with four independent accumulators
// (GB300's FP64 latency makes a single FMA chain the critical path).
__device__ __forceinline__ double dot64_ilp(const double* u, const double* v, int len) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = 0;
  for (; k + 3 < len; k += 4) {
    a0 = fma(u[k], v[k], a0);
    a1 = fma(u[k + 1], v[k + 1], a1);
    a2 = fma(u[k + 2], v[k + 2], a2);
    a3 = fma(u[k + 3], v[k + 3], a3);
  }
  for (; k < len; ++k) a0 = fma(u[k], v[k], a0);
  return (a0 + a1) + (a2 + a3);
}

__device__ __forceinline__ double relgap64(double a, double b) {
  double m = fmax(fabs(a), fabs(b));
  if (m == 0.0) return 0.0;
  return __ddiv_rn(fabs(__dsub_rn(a, b)), m);
}

__device__ __forceinline__ int ray_offset(int j, int n0) {
  int t = j - n0 + 1;
  if (t < 1) return 0;
  int q = 1;
  while ((q + 1) * (q + 1) <= t) ++q;
  return t % q;
}

// ----- mbarrier / bulk-copy (TMA) helpers -----------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared, completion signalled on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Waits for phase `parity` of the barrier; gives up after LAGP_WAIT_CYCLES
// and returns false (the caller records LAGP_DEV_TIMEOUT and stops).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  while (clock64() - t0 < LAGP_WAIT_CYCLES) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace lagp
