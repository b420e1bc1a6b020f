// schedule.cu -- work order and launch choices of the persistent FP32-scoring
// kernels.
//
// Work order.  The cost of a location grows like n^3 (ray search: every
// evaluation is an O(j^2) triangular product, steps j = n0..n-1) and, for the
// exhaustive search, also in proportion to N'.  With uneven n and N' per
// location the persistent kernels take work largest-first (a counting sort on a
// logarithmic cost bucket, 8 buckets per doubling), so that the last locations
// to start are small ones and the launch ends without a long tail.  The order
// only schedules: every location's result is computed the same way whatever its
// position.
#include <cmath>
#include <mutex>

#include "../../include/lagp.h"
#include "common.cuh"
#include "lagp_internal.h"

namespace lagp {

int exh_slots(int64_t chunk) { return (int)(chunk < EXH_SLOTS ? chunk : EXH_SLOTS); }

int ctas_per_sm(const void* kernel, int threads, size_t smem) {
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, kernel) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess)
    return 0;
  const size_t per_cta = smem + fa.sharedSizeBytes + (size_t)reserved;
  int n = blk_sm;
  const int by_smem = (int)((size_t)smem_sm / per_cta);
  if (by_smem < n) n = by_smem;
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((fa.numRegs + 7) / 8) * 8 * 32;   // allocation per warp
  if (regs_warp > 0 && regs_sm / (regs_warp * warps) < n) n = regs_sm / (regs_warp * warps);
  if (thr_sm / (warps * 32) < n) n = thr_sm / (warps * 32);
  return n > 0 ? n : 0;
}

Tune default_tune() {
  Tune t;
  t.ray_warps = 2;
  t.lpt = 1;
  t.exh_occ = 1;
  return t;
}

// part (bit 8) and descending cost bucket (bits 0-7) of each location
__global__ void order_key_kernel(const int32_t* __restrict__ n_loc,
                                 const int32_t* __restrict__ nc_loc, int64_t M, int n_max,
                                 int nc_max, int search, int split_n, int lpt, unsigned* hist,
                                 uint16_t* key) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int n = n_loc ? n_loc[i] : n_max;
  const int nc = nc_loc ? nc_loc[i] : nc_max;
  const float nf = (float)(n > 1 ? n : 1), ncf = (float)(nc > 1 ? nc : 1);
  // ray: evaluations (~20 per ray step) of O(j^2) plus an O(N') snap per step;
  // exhaustive: N' candidates of O(j^2) per step
  const float cost = (search != LAGP_EXHAUSTIVE) ? nf * nf * nf * 7.f + nf * ncf
                                                 : nf * nf * nf * ncf;
  int b = lpt ? (int)floorf(8.f * log2f(cost)) : 0;
  b = b < 0 ? 0 : (b > 255 ? 255 : b);
  const int part = (split_n > 0 && n > split_n) ? 1 : 0;
  const unsigned k = (unsigned)(part << 8) | (unsigned)(255 - b);
  key[i] = (uint16_t)k;
  atomicAdd(&hist[k], 1u);
}

// exclusive scan of each part's 256 buckets (two threads, one per part)
__global__ void order_scan_kernel(unsigned* hist, unsigned* count) {
  const int part = threadIdx.x;
  if (part > 1) return;
  unsigned run = 0;
  for (int b = 0; b < 256; ++b) {
    const unsigned c = hist[part * 256 + b];
    hist[part * 256 + b] = run;
    run += c;
  }
  count[part] = run;
}

__global__ void order_scatter_kernel(const uint16_t* __restrict__ key, int64_t M, int64_t stride,
                                     unsigned* offs, int32_t* order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const unsigned k = key[i];
  const unsigned pos = atomicAdd(&offs[k], 1u);
  order[(int64_t)(k >> 8) * stride + pos] = (int32_t)i;
}

cudaError_t launch_order(const DesignArgs& a, int search, int split_n, int lpt, cudaStream_t s) {
  const Workspace& w = *a.ws;
  cudaError_t err = cudaMemsetAsync(w.order_hist, 0, 512 * sizeof(unsigned), s);
  if (err != cudaSuccess) return err;
  const unsigned blocks = (unsigned)((a.M + 255) / 256);
  prof_begin("order", s);
  order_key_kernel<<<blocks, 256, 0, s>>>(a.n_loc, a.nc_loc, a.M, a.n_max, a.nc_max, search,
                                          split_n, lpt, w.order_hist, w.order_key);
  order_scan_kernel<<<1, 32, 0, s>>>(w.order_hist, w.order_count);
  order_scatter_kernel<<<blocks, 256, 0, s>>>(w.order_key, a.M, w.chunk, w.order_hist, w.order);
  prof_end(s);
  return cudaGetLastError();
}

// ----- launch choices: process-wide cache keyed by the shape --------------------
namespace {
struct TuneEntry {
  int p, n_max, nc_max, nrays, search, uneven;
  Tune t;
};
std::mutex g_tune_mu;
TuneEntry g_tune[64];
int g_tune_n = 0;
}  // namespace

Tune lookup_tune(int p, int n_max, int nc_max, int nrays, int search, int uneven) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int i = 0; i < g_tune_n; ++i) {
    const TuneEntry& e = g_tune[i];
    if (e.p == p && e.n_max == n_max && e.nc_max == nc_max && e.nrays == nrays &&
        e.search == search && e.uneven == uneven)
      return e.t;
  }
  Tune t = default_tune();
  if (search != LAGP_EXHAUSTIVE) t.ray_warps = ray32_default_warps(p, n_max, nc_max, nrays);
  return t;
}

void store_tune(int p, int n_max, int nc_max, int nrays, int search, int uneven, const Tune& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int i = 0; i < g_tune_n; ++i) {
    TuneEntry& e = g_tune[i];
    if (e.p == p && e.n_max == n_max && e.nc_max == nc_max && e.nrays == nrays &&
        e.search == search && e.uneven == uneven) {
      e.t = t;
      return;
    }
  }
  const int slot = g_tune_n < 64 ? g_tune_n++ : 63;   // the table keeps the last 64 shapes
  g_tune[slot] = TuneEntry{p, n_max, nc_max, nrays, search, uneven, t};
}

// code = ray_warps | lpt << 4 | (exh_occ - 1) << 5
int encode_tune(const Tune& t) { return t.ray_warps | (t.lpt << 4) | ((t.exh_occ - 1) << 5); }

bool decode_tune(int code, Tune* t) {
  const int rw = code & 15;
  if (rw != 1 && rw != 2 && rw != 4) return false;
  if (code & ~63) return false;
  t->ray_warps = rw;
  t->lpt = (code >> 4) & 1;
  t->exh_occ = ((code >> 5) & 1) + 1;
  return true;
}

}  // namespace lagp
