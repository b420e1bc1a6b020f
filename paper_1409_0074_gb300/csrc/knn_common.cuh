// knn_common.cuh -- candidate-buffer entries and the warp routines that
// select the k-th smallest buffered distance and compact a buffer, shared by
// the streaming (knn.cu) and tensor-core (knn_tc.cu) kNN filters.
#pragma once
#include <cstdint>

namespace lagp {

struct __align__(8) KnnEntry {
  float d;
  int32_t idx;
};

// ---------------------------------------------------------------------------
// Warp radix select: the k-th smallest (1-based) of cnt non-negative float
// keys in e[0..cnt), returned as its bit pattern.  hist: 256 words of this
// warp's shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_select_kth(const KnnEntry* e, int cnt, int k, uint32_t* hist) {
  const int lane = threadIdx.x & 31;
  uint32_t prefix = 0, pmask = 0;
  int kk = k;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = lane; b < 256; b += 32) hist[b] = 0;
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
      uint32_t key = __float_as_uint(e[i].d);
      if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncwarp();
    // lane owns bins 8*lane .. 8*lane+7
    uint32_t c[8], tot = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) { c[b] = hist[lane * 8 + b]; tot += c[b]; }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t excl = incl - tot;
    // the lane whose range holds the kk-th key finds the digit
    int found = ((int)excl < kk && (int)incl >= kk);
    uint32_t fmask = __ballot_sync(0xffffffffu, found);
    int src = __ffs(fmask) - 1;
    uint32_t digit = 0;
    int kk_new = kk;
    if (lane == src) {
      uint32_t run = excl;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        if ((int)(run + c[b]) >= kk) { digit = lane * 8 + b; kk_new = kk - (int)run; break; }
        run += c[b];
      }
    }
    digit = __shfl_sync(0xffffffffu, digit, src < 0 ? 0 : src);
    kk = __shfl_sync(0xffffffffu, kk_new, src < 0 ? 0 : src);
    prefix |= digit << shift;
    pmask |= 255u << shift;
    __syncwarp();
  }
  return prefix;
}

// Keep entries with d <= keep (stable, in place); returns the new count.
__device__ __forceinline__ int warp_compact(KnnEntry* e, int cnt, float keep) {
  const int lane = threadIdx.x & 31;
  int out = 0;
  for (int base = 0; base < cnt; base += 32) {
    int i = base + lane;
    KnnEntry v;
    bool ok = false;
    if (i < cnt) { v = e[i]; ok = v.d <= keep; }
    __syncwarp();
    uint32_t m = __ballot_sync(0xffffffffu, ok);
    if (ok) e[out + __popc(m & ((1u << lane) - 1u))] = v;
    out += __popc(m);
    __syncwarp();
  }
  return out;
}

// squared FP32 distance of a design row to the 4 locations of a warp, in the
// stream's form |q|^2 + |x|^2 - 2 q.x
}  // namespace lagp
