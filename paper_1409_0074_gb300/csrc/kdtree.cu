// kdtree.cu -- build of the implicit k-d tree of kdtree.cuh over the design.
//
// Level L (0 .. D-1) orders the positions of every level-L node by the
// node's split coordinate L mod p: one stable least-significant-digit radix
// sort of the keys (node << 32 | coordinate bits), 8 bits a pass, over all
// positions.  Sorting by node as the high digits keeps every node's points in
// its own range, so after the last level each node's children are the lower
// and upper halves of its range.  Ties in a coordinate keep the previous
// order, so the tree is deterministic.  Then the tree-ordered FP32 rows are
// gathered and the node boxes are formed from the leaves upwards.
#include <cstdint>

#include "kdtree.cuh"
#include "lagp_internal.h"

namespace lagp {

#define RS_TILE 4096

static int rs_blocks(int64_t N) { return (int)((N + RS_TILE - 1) / RS_TILE); }

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t kd_bytes(int64_t N, int p, int PP) {
  const int64_t nodes = kd_nodes(kd_depth(N));
  return al256(sizeof(int32_t) * N) + al256(sizeof(float) * N * PP) +
         al256(sizeof(float) * nodes * 2 * PP) + al256(sizeof(double) * nodes * 2 * p) +
         al256(sizeof(uint64_t) * 2 * N) + al256(sizeof(int32_t) * N) +
         al256(sizeof(uint32_t) * 256 * (size_t)rs_blocks(N));
}

void kd_carve(int64_t N, int p, int PP, char* base, KdTree* t) {
  const int D = kd_depth(N);
  const int64_t nodes = kd_nodes(D);
  size_t off = 0;
  auto take = [&](size_t b) { char* q = base ? base + off : nullptr; off += al256(b); return q; };
  t->D = D;
  t->perm = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * N));
  t->pts32 = reinterpret_cast<float*>(take(sizeof(float) * N * PP));
  t->box32 = reinterpret_cast<float*>(take(sizeof(float) * nodes * 2 * PP));
  t->box64 = reinterpret_cast<double*>(take(sizeof(double) * nodes * 2 * p));
  t->keys = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * 2 * N));
  t->vals = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * N));
  t->hist = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 256 * (size_t)rs_blocks(N)));
}

// keys of level `level`: the position's node (relative index within the level)
// in the high word, the order-preserving bits of coordinate `dim` below
__global__ void kd_keys(const int32_t* __restrict__ perm, const float* __restrict__ Xf, int64_t N,
                        int PP, int level, int dim, int first, uint64_t* __restrict__ keys,
                        int32_t* __restrict__ vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t gi = first ? (int32_t)i : perm[i];
    int64_t lo = 0, hi = N;
    uint32_t node = 0;
    for (int l = 0; l < level; ++l) {
      const int64_t m = (lo + hi) >> 1;
      if (i < m) { hi = m; node = node << 1; }
      else { lo = m; node = (node << 1) | 1u; }
    }
    uint32_t u = __float_as_uint(Xf[(int64_t)gi * PP + dim]);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    keys[i] = ((uint64_t)node << 32) | u;
    vals[i] = gi;
  }
}

// digit counts of each tile, stored digit-major: hist[digit][block]
__global__ void rs_hist(const uint64_t* __restrict__ keys, int64_t N, int shift,
                        uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
  const int64_t t1 = t0 + RS_TILE < N ? t0 + RS_TILE : N;
  for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x)
    atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive prefix sum of hist[0 .. total) in place (one block of 1024 threads)
__global__ void rs_scan(uint32_t* __restrict__ hist, int64_t total) {
  __shared__ uint32_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (total + 1023) / 1024;
  const int64_t a = t * per, b = a + per < total ? a + per : total;
  uint32_t s = 0;
  for (int64_t i = a; i < b; ++i) s += hist[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {     // inclusive scan of the partial sums
    const uint32_t v = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = t > 0 ? part[t - 1] : 0u;
  for (int64_t i = a; i < b; ++i) {
    const uint32_t c = hist[i];
    hist[i] = run;
    run += c;
  }
}

// stable scatter of one tile by one warp, 32 keys at a time in order
__global__ void rs_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                           uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t N,
                           int shift, const uint32_t* __restrict__ hist) {
  __shared__ uint32_t base[256];
  const int lane = threadIdx.x;
  for (int d = lane; d < 256; d += 32) base[d] = hist[(int64_t)d * gridDim.x + blockIdx.x];
  __syncwarp();
  const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
  const int64_t t1 = t0 + RS_TILE < N ? t0 + RS_TILE : N;
  for (int64_t c0 = t0; c0 < t1; c0 += 32) {
    const int64_t i = c0 + lane;
    const bool valid = i < t1;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const uint64_t k = kin[i];
      const uint32_t dig = (uint32_t)(k >> shift) & 255u;
      const unsigned peers = __match_any_sync(act, dig);
      const unsigned below = peers & ((1u << lane) - 1u);
      const uint32_t pos = base[dig] + (uint32_t)__popc(below);
      kout[pos] = k;
      vout[pos] = vin[i];
      __syncwarp(act);
      if (below == 0u) base[dig] += (uint32_t)__popc(peers);   // the group's first lane
    }
    __syncwarp();
  }
}

__global__ void kd_copy(const int32_t* __restrict__ src, int32_t* __restrict__ dst, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void kd_gather(const int32_t* __restrict__ perm, const float* __restrict__ Xf,
                          int64_t N, int PP, float* __restrict__ pts) {
  const int64_t total = N * PP;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = e / PP;
    const int k = (int)(e - pos * PP);
    pts[e] = Xf[(int64_t)perm[pos] * PP + k];
  }
}

// leaf boxes: one warp per leaf, lane k takes coordinate k
__global__ void kd_leaf_box(const int32_t* __restrict__ perm, const float* __restrict__ pts,
                            const double* __restrict__ X, int64_t N, int p, int PP, int D,
                            float* __restrict__ box32, double* __restrict__ box64) {
  const int lane = threadIdx.x & 31;
  const int64_t leaf = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nleaf = (int64_t)1 << D;
  if (leaf >= nleaf) return;
  const int64_t v = nleaf + leaf;
  int64_t a, b;
  kd_range(N, v, D, &a, &b);
  if (lane < PP) {
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t pos = a; pos < b; ++pos) {
      const float c = pts[pos * PP + lane];
      lo = fminf(lo, c);
      hi = fmaxf(hi, c);
    }
    box32[v * 2 * PP + lane] = lo;
    box32[v * 2 * PP + PP + lane] = hi;
  }
  if (lane < p) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t pos = a; pos < b; ++pos) {
      const double c = X[(int64_t)perm[pos] * p + lane];
      lo = fmin(lo, c);
      hi = fmax(hi, c);
    }
    box64[v * 2 * p + lane] = lo;
    box64[v * 2 * p + p + lane] = hi;
  }
}

// boxes of level `level` as the union of their children's
__global__ void kd_up(int level, int p, int PP, float* __restrict__ box32,
                      double* __restrict__ box64) {
  const int64_t n = (int64_t)1 << level;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * PP) return;
  const int64_t v = n + e / PP;
  const int k = (int)(e % PP);
  const float* c0 = box32 + 2 * v * 2 * PP;
  const float* c1 = c0 + 2 * PP;
  box32[v * 2 * PP + k] = fminf(c0[k], c1[k]);
  box32[v * 2 * PP + PP + k] = fmaxf(c0[PP + k], c1[PP + k]);
  if (k < p) {
    const double* d0 = box64 + 2 * v * 2 * p;
    const double* d1 = d0 + 2 * p;
    box64[v * 2 * p + k] = fmin(d0[k], d1[k]);
    box64[v * 2 * p + p + k] = fmax(d0[p + k], d1[p + k]);
  }
}

cudaError_t launch_kd_build(const double* X, const float* Xf, int64_t N, int p, int PP,
                            const KdTree& t, cudaStream_t s) {
  const int D = t.D;
  if (D + 2 > KD_STACK) return cudaErrorInvalidValue;
  const int nblk = rs_blocks(N);
  const unsigned g = (unsigned)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
  prof_begin("kd_build", s);
  uint64_t* kb[2] = {t.keys, t.keys + N};
  for (int level = 0; level < D; ++level) {
    // keys into buffer 0 (values: the current order, identity at level 0)
    kd_keys<<<g, 256, 0, s>>>(t.perm, Xf, N, PP, level, level % p, level == 0, kb[0], t.vals);
    int cur = 0;                 // keys in kb[cur]; values in t.vals for cur = 0 at start
    int32_t* vcur = t.vals;
    int32_t* valt = t.perm;
    const int passes = 4 + (level + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
      const int shift = 8 * ps;
      rs_hist<<<nblk, 256, 0, s>>>(kb[cur], N, shift, t.hist);
      rs_scan<<<1, 1024, 0, s>>>(t.hist, (int64_t)256 * nblk);
      rs_scatter<<<nblk, 32, 0, s>>>(kb[cur], vcur, kb[cur ^ 1], valt, N, shift, t.hist);
      cur ^= 1;
      int32_t* tmp = vcur;
      vcur = valt;
      valt = tmp;
    }
    if (vcur != t.perm) kd_copy<<<g, 256, 0, s>>>(vcur, t.perm, N);
  }
  if (D == 0) kd_keys<<<g, 256, 0, s>>>(t.perm, Xf, N, PP, 0, 0, 1, kb[0], t.perm);
  kd_gather<<<g, 256, 0, s>>>(t.perm, Xf, N, PP, t.pts32);
  const int64_t nleaf = (int64_t)1 << D;
  kd_leaf_box<<<(unsigned)((nleaf * 32 + 255) / 256), 256, 0, s>>>(t.perm, t.pts32, X, N, p, PP,
                                                                   D, t.box32, t.box64);
  for (int level = D - 1; level >= 0; --level) {
    const int64_t work = ((int64_t)1 << level) * PP;
    kd_up<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(level, p, PP, t.box32, t.box64);
  }
  prof_end(s);
  return cudaGetLastError();
}

}  // namespace lagp
