// ray32_layout.h -- shared-memory layout of one warp (one location) of the
// FP32-scoring ray kernel, and the index arithmetic of its row storage.  Free
// of CUDA so that the host tests compile it; KD_STACK (the k-d tree walk's
// stack depth) comes from kdtree.cuh, or from the compiler's command line.
#pragma once

#ifndef KD_STACK
#error "KD_STACK must be defined before ray32_layout.h"
#endif

#if defined(__CUDACC__)
#define LAGP_HD __device__ __host__ __forceinline__
#define LAGP_HDI __host__ __device__ inline
#else
#define LAGP_HD inline
#define LAGP_HDI inline
#endif

namespace lagp {

// start of row i in the zero-padded FP32 row storage (rows of length
// (i+1) rounded up to a multiple of 4)
LAGP_HD int roff(int i) {
  const int a = i >> 2, b = i & 3;
  return 4 * (i + 2 * a * (a - 1) + a * b);
}
LAGP_HD int tri(int i) { return i * (i + 1) / 2; }
// row length of the kz buffer: a multiple of 4 whose quarter is odd, so that
// the rays' float4 reads fall on different banks
LAGP_HD int kz_ld(int n) {
  int k = (n + 3) & ~3;
  if (((k >> 2) & 1) == 0) k += 4;
  return k;
}

struct WarpLayout {
  int lf, kz, cb, zf, tau, x, gsel, stk, bnd, starts, mask, smask, vm, bytes;
};

LAGP_HDI WarpLayout warp_layout(int n, int PP, int RP, int nc) {
  WarpLayout w;
  int off = 0;   // in 4-byte words, float region first (16-byte aligned pieces)
  auto take = [&](int words) { int o = off; off += (words + 3) & ~3; return o; };
  w.lf = take(roff(n));
  w.kz = take(RP * kz_ld(n));
  // per-ray exponent coefficients c_k then b_k (rows of kz_ld(n)); the k-d
  // tree walk of the full-scope snap (nodes, then their box distances) and
  // the factor update's two binary64 work vectors (n each) run after the
  // step's evaluations and reuse this space
  const int cbw = 2 * RP * kz_ld(n);
  w.cb = take(cbw > 2 * KD_STACK ? cbw : 2 * KD_STACK);
  w.stk = w.cb;
  w.bnd = w.cb + KD_STACK;
  w.zf = take((n + 3) & ~3);
  w.tau = take(RP);            // each ray's segment: end = a + tau * 10 (a - x)
  w.x = take(4 * PP);          // xf, lof, hif, xs
  w.gsel = take(n);            // design indices of the selected points
  w.starts = take(RP);
  w.mask = take((nc + 31) / 32);
  w.smask = take((nc + 31) / 32);
  w.vm = take(2);              // smallest binary64 pivot of the location (lane 0)
  w.bytes = off * 4;
  return w;
}

}  // namespace lagp
