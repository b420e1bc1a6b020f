// kdtree.cuh -- spatial index over the design X_N for the unlimited ray scope:
// the snap of a ray step (Sec 4) searches all of X_N outside the current local
// design, which the paper allows (Sec 5 places no N' limit on ray searches).
//
// Tree.  An implicit k-d tree over tree positions 0..N-1: heap node 1 is the
// root with positions [0, N); node v of range [a, b) has children 2v over
// [a, m) and 2v+1 over [m, b), m = (a + b) / 2.  At level L the split runs
// along coordinate L mod p: the build orders every node's range by that
// coordinate (kdtree.cu), so the children are the lower and upper halves.
// Leaves are the nodes at depth D, the smallest depth whose ranges hold at
// most KD_LEAF points.  Every node keeps the exact bounding box of its points,
// in the centred FP32 coordinates (FP32 scoring form) and in binary64 (parity
// form).
//
// Query.  One warp finds, exactly, the nearest point to x* outside the design
// (and, for the step's decision gap, the second smallest distance): depth
// first, nearer child first, a node skipped when its box is farther than the
// second-best distance so far (with a relative margin above the rounding of
// both distances).  A leaf gives one point per lane.  Ties go to the point
// nearer to x, then to the lower design index.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace lagp {

#define KD_LEAF 32
#define KD_STACK 40

__host__ __device__ inline int kd_depth(int64_t N) {
  int D = 0;
  while (((N + ((int64_t)1 << D) - 1) >> D) > KD_LEAF) ++D;
  return D;
}
__host__ __device__ inline int64_t kd_nodes(int D) { return (int64_t)2 << D; }

// Positions [a, b) of heap node v (at level `level`).
__device__ __forceinline__ void kd_range(int64_t N, int64_t v, int level, int64_t* a,
                                         int64_t* b) {
  int64_t lo = 0, hi = N;
  for (int l = level - 1; l >= 0; --l) {
    const int64_t m = (lo + hi) >> 1;
    if ((v >> l) & 1) lo = m; else hi = m;
  }
  *a = lo;
  *b = hi;
}

template <typename T>
struct KdTop {
  T d1, dx1, d2;
  int32_t i1;    // design index of the best, or -1
};

// Lexicographic (d, dx, index) order of the best; d2 keeps the second
// smallest distance (equal to d1 when two points tie).
template <typename T>
__device__ __forceinline__ KdTop<T> kd_merge(KdTop<T> a, KdTop<T> b) {
  const bool b_first = b.i1 >= 0 &&
      (a.i1 < 0 || b.d1 < a.d1 ||
       (b.d1 == a.d1 && (b.dx1 < a.dx1 || (b.dx1 == a.dx1 && b.i1 < a.i1))));
  KdTop<T> r;
  if (b_first) { r = b; r.d2 = a.d1 < b.d2 ? a.d1 : b.d2; }
  else { r = a; r.d2 = b.d1 < a.d2 ? b.d1 : a.d2; }
  return r;
}

template <typename T>
__device__ __forceinline__ KdTop<T> kd_warp_merge(KdTop<T> t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    KdTop<T> u;
    u.d1 = __shfl_xor_sync(0xffffffffu, t.d1, o);
    u.dx1 = __shfl_xor_sync(0xffffffffu, t.dx1, o);
    u.d2 = __shfl_xor_sync(0xffffffffu, t.d2, o);
    u.i1 = __shfl_xor_sync(0xffffffffu, t.i1, o);
    t = kd_merge(t, u);
  }
  return t;
}

// A view of the tree for one arithmetic.  box: [kd_nodes(D)][2][stride] (lo
// row, then hi row); point(pos, k): coordinate k of the point at tree
// position pos; perm: tree position -> design index.
template <typename T>
struct KdView {
  const T* box;
  int stride, p, D;
  int64_t N;
  const int32_t* perm;
  const T* pts;        // FP32: tree-ordered rows [N][stride]; binary64: the design [N][p]
  bool by_design;      // pts indexed by design index (binary64) or by position (FP32)
  __device__ __forceinline__ T point(int64_t pos, int32_t gi, int k) const {
    return by_design ? pts[(int64_t)gi * p + k] : pts[pos * stride + k];
  }
};

// Squared distances from xs to the boxes of nodes c0 = 2v and c0 + 1, one
// half-warp per child and one lane per coordinate (p <= 16), summed by
// shuffles; every lane receives both.
template <typename T>
__device__ __forceinline__ void kd_child_lbs(const KdView<T>& V, int64_t v, T xk, T* l0, T* l1) {
  const int lane = threadIdx.x & 31, k = lane & 15;
  const int64_t c = 2 * v + (lane >> 4);
  T t = 0;
  if (k < V.p) {
    const T* lo = V.box + c * 2 * V.stride;
    const T a = lo[k] - xk, b = xk - lo[V.stride + k];
    t = a > 0 ? a : (b > 0 ? b : (T)0);
    t = t * t;
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  *l0 = __shfl_sync(0xffffffffu, t, 0);
  *l1 = __shfl_sync(0xffffffffu, t, 16);
}

// Nearest point to xs outside the design (and its second-best distance).
// Warp-collective; every lane returns the same result.  excluded(gi, pos,
// allow_starts) says whether design point gi (at tree position pos) may not be
// picked; with no allowed point at all the search repeats with the ray starts
// allowed.  dist(pos, gi) and distx(pos, gi) give a point's squared distances
// to x* and to x in the form's own arithmetic.  stk / bnd: KD_STACK entries
// per warp (a pending node and its box distance).
template <typename T, typename Excl, typename Dist, typename DistX>
__device__ KdTop<T> kd_nearest(const KdView<T>& V, const T* xs, T margin, int* stk, T* bnd,
                               Excl excluded, Dist dist, DistX distx) {
  const int lane = threadIdx.x & 31;
  const T inf = (T)INFINITY;
  const T xk = (lane & 15) < V.p ? xs[lane & 15] : (T)0;
  KdTop<T> best;
  for (int pass = 0; pass < 2; ++pass) {
    best.d1 = inf; best.dx1 = inf; best.d2 = inf; best.i1 = -1;
    if (lane == 0) { stk[0] = 1; bnd[0] = 0; }
    int sp = 1;
    __syncwarp();
    while (sp > 0) {
      --sp;
      const int64_t v = stk[sp];
      const T lbv = bnd[sp];
      __syncwarp();
      if (lbv > best.d2 * ((T)1 + margin)) continue;
      const int level = 31 - __clz((int)v);
      if (level == V.D) {
        int64_t a, b;
        kd_range(V.N, v, level, &a, &b);
        const int64_t pos = a + lane;
        KdTop<T> t;
        t.d1 = inf; t.dx1 = inf; t.d2 = inf; t.i1 = -1;
        bool near = false;
        T d = inf;
        int32_t gi = -1;
        if (pos < b) {
          gi = V.perm[pos];
          d = dist(pos, gi);
          near = d <= best.d2;
        }
        // most leaves hold no point nearer than the second best: no merge
        if (!__any_sync(0xffffffffu, near)) continue;
        if (near && !excluded(gi, pos, pass == 1)) {
          t.d1 = d;
          t.dx1 = distx(pos, gi);
          t.i1 = gi;
        }
        best = kd_merge(best, kd_warp_merge(t));
      } else {
        T l0, l1;
        kd_child_lbs(V, v, xk, &l0, &l1);
        const bool right_first = l1 < l0;
        if (lane == 0) {
          stk[sp] = (int)(2 * v + (right_first ? 0 : 1));
          bnd[sp] = right_first ? l0 : l1;
          stk[sp + 1] = (int)(2 * v + (right_first ? 1 : 0));
          bnd[sp + 1] = right_first ? l1 : l0;
        }
        sp += 2;
        __syncwarp();
      }
    }
    if (best.i1 >= 0) break;
  }
  return best;
}

// Workspace pieces of the tree (design part of the workspace).
struct KdTree {
  int D;
  int32_t* perm;     // [N] tree position -> design index
  float* pts32;      // [N][PP] centred FP32 rows in tree order
  float* box32;      // [nodes][2][PP]
  double* box64;     // [nodes][2][p]
  uint64_t* keys;    // [2][N] sort scratch
  int32_t* vals;     // [N] sort scratch
  uint32_t* hist;    // [256][blocks] sort scratch
};

size_t kd_bytes(int64_t N, int p, int PP);
void kd_carve(int64_t N, int p, int PP, char* base, KdTree* t);
cudaError_t launch_kd_build(const double* X, const float* Xf, int64_t N, int p, int PP,
                            const KdTree& t, cudaStream_t s);

}  // namespace lagp
