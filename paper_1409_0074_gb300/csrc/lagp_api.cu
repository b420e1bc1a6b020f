// lagp_api.cu -- C ABI entry points: argument checks, workspace layout, and the
// sequence of launches (prepare -> per chunk: kNN, greedy design + predict).
#include <cstring>

#include "../../include/lagp.h"
#include "common.cuh"
#include "lagp_internal.h"

namespace lagp {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Locations per chunk: bounded by a per-search cap and by keeping the kNN
// candidate buffers within 16 GiB.
static int64_t chunk_for(int64_t M, int search, int precision, int nc_max, int64_t N) {
  int64_t cap = 131072;
  if (search == LAGP_EXHAUSTIVE && precision == LAGP_FP64) cap = 16384;
  const int64_t per_loc = (int64_t)8 * knn_cap(nc_max);
  const int64_t by_mem = ((int64_t)16 << 30) / per_loc;
  if (by_mem < cap) cap = by_mem > 128 ? by_mem : 128;
  return M < cap ? (M > 0 ? M : 1) : cap;
}

namespace {
struct Carver {
  char* b;
  size_t off;
  void* take(size_t bytes) {
    void* ptr = b ? b + off : nullptr;
    off += align256(bytes);
    return ptr;
  }
};
}  // namespace

// Per-request part: the status word first (laGP_status reads it there), then
// the kNN buffers, candidates, per-slot scratch and the work order.
size_t layout_request(const Shape& sh, void* base, Workspace* ws) {
  Workspace scratch;
  Workspace* w = ws ? ws : &scratch;   // sizes only when ws is null
  Carver c{static_cast<char*>(base), 0};
  w->status = static_cast<unsigned*>(c.take(4 * sizeof(unsigned)));
  const int64_t ch = sh.chunk;
  w->knn_buf = c.take((size_t)8 * ch * knn_cap(sh.nc_max));
  w->knn_cnt = static_cast<int32_t*>(c.take(sizeof(int32_t) * ch));
  w->knn_thr = static_cast<float*>(c.take(sizeof(float) * ch));
  w->knn_seg = static_cast<int32_t*>(c.take(sizeof(int32_t) * 4 * ch));
  w->cand = static_cast<int32_t*>(c.take(sizeof(int32_t) * ch * sh.nc_max));
  size_t s64 = 0, s32 = 0;
  if (sh.precision == LAGP_FP64) {
    if (sh.search == LAGP_EXHAUSTIVE) s64 = sizeof(double) * ch * sh.n_max * sh.nc_max;
  } else if (sh.search != LAGP_EXHAUSTIVE) {
    s64 = sizeof(double) * ray32_slots(ch) * ray32_g64_doubles(sh.n_max);
  } else {
    const size_t slots = exh_slots(ch);
    s64 = sizeof(double) * slots * sh.n_max * sh.n_max;
    // correlation cache per slot: [n_max][nc_max] (CUDA-core scorer), or for
    // the tensor-core form also its operand tiles, the larger
    size_t per = (size_t)sh.n_max * sh.nc_max;
    if (sh.precision == LAGP_FP32_SCORE_TC && exh_tc_cache_floats(sh.nc_max) > per)
      per = exh_tc_cache_floats(sh.nc_max);
    s32 = sizeof(float) * slots * per;
  }
  w->state64 = static_cast<double*>(c.take(s64));
  w->state32 = static_cast<float*>(c.take(s32));
  const bool fp32_exh = sh.precision != LAGP_FP64 && sh.search == LAGP_EXHAUSTIVE;
  w->crow = static_cast<float*>(
      c.take(fp32_exh ? sizeof(float) * exh_slots(ch) * sh.nc_max * sh.PP : 0));
  w->queue = static_cast<unsigned*>(c.take(4 * sizeof(unsigned)));
  w->order = static_cast<int32_t*>(c.take(sizeof(int32_t) * 2 * ch));
  w->order_hist = static_cast<unsigned*>(c.take(512 * sizeof(unsigned)));
  w->order_count = static_cast<unsigned*>(c.take(2 * sizeof(unsigned)));
  w->order_key = static_cast<uint16_t*>(c.take(sizeof(uint16_t) * ch));
  // precision promotion: the re-solve list and, for exhaustive search, the
  // binary64 correlation cache of its CTAs
  w->promote = static_cast<int32_t*>(c.take(sh.promote ? sizeof(int32_t) * ch : 0));
  const int64_t pslots = ch < PROMOTE_SLOTS ? ch : PROMOTE_SLOTS;
  w->promote64 = static_cast<double*>(c.take(sh.promote && sh.search == LAGP_EXHAUSTIVE
      ? sizeof(double) * pslots * sh.n_max * sh.nc_max : 0));
  w->chunk = ch;
  return c.off;
}

// Design part: bounding box, centred FP32 copy and its row norms.
size_t layout_design(const Shape& sh, void* base, Workspace* ws) {
  Workspace scratch;
  Workspace* w = ws ? ws : &scratch;   // sizes only when ws is null
  Carver c{static_cast<char*>(base), 0};
  w->maxn2 = static_cast<unsigned*>(c.take(4 * sizeof(unsigned)));
  w->bbox_part = static_cast<double*>(c.take(sizeof(double) * 64 * 2 * sh.p));
  w->lo = static_cast<double*>(c.take(sizeof(double) * sh.p));
  w->hi = static_cast<double*>(c.take(sizeof(double) * sh.p));
  w->center = static_cast<double*>(c.take(sizeof(double) * sh.p));
  w->Xf = static_cast<float*>(c.take(sizeof(float) * sh.Npad * sh.PP));
  w->nx = static_cast<float*>(c.take(sizeof(float) * sh.Npad));
  w->Btc = static_cast<float*>(c.take(sizeof(float) * knn_tc_tile_floats(sh.Npad, sh.p)));
  if (sh.search == LAGP_RAY_FULL) {
    kd_carve(sh.N, sh.p, sh.PP, static_cast<char*>(c.take(kd_bytes(sh.N, sh.p, sh.PP))), &w->kd);
  } else {
    std::memset(&w->kd, 0, sizeof(w->kd));
  }
  return c.off;
}

size_t layout_workspace(const Shape& sh, void* base, Workspace* ws) {
  Workspace w;
  std::memset(&w, 0, sizeof(w));
  const size_t r = layout_request(sh, base, &w);
  const size_t d = layout_design(sh, base ? static_cast<char*>(base) + r : nullptr, &w);
  if (ws) *ws = w;
  return r + d;
}

bool make_shape(int64_t N, int p, int64_t M, int n0, int n, int N_close, int nrays, int search,
                int precision, Shape* sh, bool knn_only) {
  if (p < 1 || p > LAGP_MAX_P || N < 1 || M < 0) return false;
  if (n0 < 1 || n0 > n || n > LAGP_MAX_N || n > N_close || N_close > N || N_close > 4096)
    return false;
  if (search != LAGP_EXHAUSTIVE && search != LAGP_RAY && search != LAGP_RAY_FULL) return false;
  const int form = precision & ~LAGP_PROMOTE;
  if (form != LAGP_FP32_SCORE && form != LAGP_FP32_SCORE_TC &&
      (form != LAGP_FP64 || precision != LAGP_FP64))
    return false;
  if (N > (int64_t)0x7fffff00) return false;   // int32 design indices
  int R = nrays <= 0 ? p : nrays;
  if (!knn_only && search != LAGP_EXHAUSTIVE && (R > LAGP_MAX_RAYS || R > N_close - n))
    return false;
  sh->N = N;
  sh->p = p;
  sh->PP = (p + 3) / 4 * 4;
  sh->Npad = (N + LAGP_KNN_TILE - 1) / LAGP_KNN_TILE * LAGP_KNN_TILE;
  sh->M = M;
  sh->n0 = n0;
  sh->n_max = n;
  sh->nc_max = N_close;
  sh->nrays = (search != LAGP_EXHAUSTIVE) ? R : 1;
  sh->search = search;
  sh->precision = form;
  sh->promote = (precision & LAGP_PROMOTE) != 0;
  sh->chunk = chunk_for(M, search, form, N_close, N);
  return true;
}

}  // namespace lagp

using namespace lagp;

extern "C" size_t laGP_workspace_bytes(int64_t N, int p, int64_t M, int n, int N_close,
                                       int nrays, int search, int precision) {
  Shape sh;
  if (!make_shape(N, p, M, 1, n, N_close, nrays, search, precision, &sh)) return 0;
  return layout_workspace(sh, nullptr, nullptr);
}

namespace lagp {

// FP32-scoring greedy design + prediction of one chunk.
static cudaError_t run_design32(const DesignArgs& a0, int search, int precision, bool uneven,
                                cudaStream_t s) {
  const Workspace& ws = *a0.ws;
  DesignArgs a = a0;
  a.order = nullptr;
  a.count = nullptr;
  cudaError_t e;
  if (search != LAGP_EXHAUSTIVE) {
    if (uneven && a.tune.lpt) {
      if ((e = launch_order(a, search, 0, 1, s)) != cudaSuccess) return e;
      a.order = ws.order;
      a.count = ws.order_count;
    }
    return launch_ray32(a, s);
  }
  // exhaustive, FP32_SCORE: the incremental CUDA-core scorer for every size
  if (precision == LAGP_FP32_SCORE) {
    if (uneven && a.tune.lpt) {
      if ((e = launch_order(a, search, 0, 1, s)) != cudaSuccess) return e;
      a.order = ws.order;
      a.count = ws.order_count;
    }
    return launch_exh32(a, s);
  }
  // exhaustive, FP32_SCORE_TC: tensor-core scorer for local designs up to its
  // size limit, CUDA-core scorer above it (decided per location)
  const int lim = exh_tc_max_n();
  if (!uneven) return a.n_max <= lim ? launch_exh_tc(a, s) : launch_exh32(a, s);
  const int split = a.n_max > lim ? lim : 0;
  if ((e = launch_order(a, search, split, a.tune.lpt, s)) != cudaSuccess) return e;
  a.order = ws.order;
  a.count = ws.order_count;
  if (split == 0) return launch_exh_tc(a, s);
  if ((e = launch_exh_tc(a, s)) != cudaSuccess) return e;
  DesignArgs b = a;
  b.order = ws.order + ws.chunk;
  b.count = ws.order_count + 1;
  return launch_exh32(b, s);
}

// Greedy design + prediction of one chunk whose candidates are in ws.cand.
// With LAGP_PROMOTE the FP32 forms list the locations whose smallest binary64
// pivot fell below LAGP_PROMOTE_PIVOT, and the binary64 kernels then solve
// those again (the count stays on the device: no host synchronisation).
static cudaError_t run_design(const DesignArgs& a0, int search, int precision, bool uneven,
                              cudaStream_t s) {
  if (precision == LAGP_FP64) return launch_design_fp64(a0, search, s);
  const Workspace& ws = *a0.ws;
  cudaError_t e;
  if (a0.promote && (e = cudaMemsetAsync(ws.status + 1, 0, sizeof(unsigned), s)) != cudaSuccess)
    return e;
  if ((e = run_design32(a0, search, precision, uneven, s)) != cudaSuccess || !a0.promote) return e;
  DesignArgs b = a0;
  b.order = nullptr;
  b.count = nullptr;
  return launch_design_fp64(b, search, s, ws.promote, ws.status + 1, ws.promote64, PROMOTE_SLOTS);
}

static DesignArgs chunk_args(const Shape& sh, const Call& c, const Workspace& ws, int64_t c0,
                             int64_t Mc, const Tune& t) {
  DesignArgs a;
  const int n = sh.n_max;
  a.X = c.design; a.Y = c.y; a.N = sh.N; a.p = sh.p; a.PP = sh.PP; a.xref = c.xref + c0 * sh.p;
  a.M = Mc; a.cand = ws.cand; a.nc_max = sh.nc_max;
  a.nc_loc = c.nclose_loc ? c.nclose_loc + c0 : nullptr; a.n0 = sh.n0; a.n_max = n;
  a.n_loc = c.n_loc ? c.n_loc + c0 : nullptr; a.theta = c.theta; a.g = c.g; a.nrays = sh.nrays;
  a.theta_loc = c.theta_loc ? c.theta_loc + c0 : nullptr;
  a.full_scope = sh.search == LAGP_RAY_FULL ? 1 : 0;
  a.mean = c.mean + c0; a.s2 = c.s2 + c0;
  a.selected = c.selected ? c.selected + c0 * n : nullptr;
  a.tie_gap = c.tie_gap ? c.tie_gap + c0 * n : nullptr;
  a.nevals = c.nevals ? c.nevals + c0 * n : nullptr;
  a.ws = &ws; a.order = nullptr; a.count = nullptr; a.tune = t;
  a.promote = sh.promote;
  return a;
}

// The whole path on the stream: prepare, then per chunk kNN and design.
int enqueue(const Shape& sh, const Call& c, const Workspace& ws, const Tune& t, cudaStream_t s,
            bool prepared) {
  if (cudaMemsetAsync(ws.status, 0, 3 * sizeof(unsigned), s) != cudaSuccess) return LAGP_ERR_CUDA;
  if (!prepared && launch_prepare(c.design, sh.N, sh.p, sh.PP, sh.Npad, ws, s) != cudaSuccess)
    return LAGP_ERR_CUDA;
  const bool uneven = c.n_loc || c.nclose_loc;
  for (int64_t c0 = 0; c0 < sh.M; c0 += sh.chunk) {
    const int64_t Mc = (sh.M - c0 < sh.chunk) ? sh.M - c0 : sh.chunk;
    const int32_t* ncl = c.nclose_loc ? c.nclose_loc + c0 : nullptr;
    if (launch_knn(c.design, sh.N, sh.p, sh.PP, sh.Npad, c.xref + c0 * sh.p, Mc, sh.nc_max, ncl,
                   ws.cand, ws, s) != cudaSuccess)
      return LAGP_ERR_CUDA;
    const DesignArgs a = chunk_args(sh, c, ws, c0, Mc, t);
    if (run_design(a, sh.search, sh.precision, uneven, s) != cudaSuccess) return LAGP_ERR_CUDA;
  }
  return LAGP_OK;
}

static int check_call(int64_t N, int p, const double* xref, int64_t M, int n0, int n,
                      int N_close, double theta, double g, int search, int nrays, int precision,
                      const double* design, const double* y, double* mean, double* s2,
                      void* workspace, size_t workspace_bytes, Shape* sh, Workspace* ws) {
  if (!make_shape(N, p, M, n0, n, N_close, nrays, search, precision, sh)) return LAGP_ERR_INVALID;
  if (!(theta > 0.0) || !(g >= 0.0) || theta != theta) return LAGP_ERR_INVALID;
  if (M == 0) return 1;
  if (!design || !y || !xref || !mean || !s2 || !workspace) return LAGP_ERR_INVALID;
  const size_t need = layout_workspace(*sh, workspace, ws);
  if (workspace_bytes < need) return LAGP_ERR_WORKSPACE;
  return LAGP_OK;
}

Tune tune_for(const Shape& sh, bool uneven) {
  return lookup_tune(sh.p, sh.n_max, sh.nc_max, sh.nrays, sh.search, uneven ? 1 : 0);
}

}  // namespace lagp

extern "C" int laGP_build_and_predict(const double* design, const double* y, int64_t N, int p,
                                      const double* xref, int64_t M, int n0, int n, int N_close,
                                      double theta, double g, int search, int nrays,
                                      int precision, const int32_t* n_loc,
                                      const int32_t* nclose_loc, double* mean, double* s2,
                                      int32_t* selected, double* tie_gap, int32_t* nevals,
                                      void* workspace, size_t workspace_bytes, void* stream) {
  Shape sh;
  Workspace ws;
  const int rc = check_call(N, p, xref, M, n0, n, N_close, theta, g, search, nrays, precision,
                            design, y, mean, s2, workspace, workspace_bytes, &sh, &ws);
  if (rc != LAGP_OK) return rc > 0 ? LAGP_OK : rc;
  const Call c{design, y, xref, theta, g, n_loc, nclose_loc, mean, s2, selected, tie_gap, nevals};
  return enqueue(sh, c, ws, tune_for(sh, n_loc || nclose_loc), static_cast<cudaStream_t>(stream),
                 false);
}

extern "C" int laGP_autotune(const double* design, const double* y, int64_t N, int p,
                             const double* xref, int64_t M, int n0, int n, int N_close,
                             double theta, double g, int search, int nrays, int precision,
                             const int32_t* n_loc, const int32_t* nclose_loc, double* mean,
                             double* s2, void* workspace, size_t workspace_bytes, void* stream,
                             int* choice) {
  Shape sh;
  Workspace ws;
  const int rc = check_call(N, p, xref, M, n0, n, N_close, theta, g, search, nrays, precision,
                            design, y, mean, s2, workspace, workspace_bytes, &sh, &ws);
  if (rc != LAGP_OK) return rc > 0 ? LAGP_ERR_INVALID : rc;
  if (!choice) return LAGP_ERR_INVALID;
  const bool uneven = n_loc || nclose_loc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (sh.precision == LAGP_FP64) {   // the FP64 kernels have no launch choices
    *choice = encode_tune(default_tune());
    return LAGP_OK;
  }
  // candidates: every choice that matters for this shape
  Tune cand[12];
  int nc = 0;
  const int lpts = uneven ? 2 : 1;
  for (int l = lpts - 1; l >= 0; --l) {
    if (search != LAGP_EXHAUSTIVE) {
      for (int rw : {2, 1, 4}) cand[nc++] = Tune{rw, l, 1};
    } else {
      for (int occ : {1, 2}) cand[nc++] = Tune{2, l, occ};
    }
  }
  // kNN of the first chunk once; then each candidate's design launch, timed
  const Call c{design, y, xref, theta, g, n_loc, nclose_loc, mean, s2, nullptr, nullptr, nullptr};
  const int64_t Mc = sh.M < sh.chunk ? sh.M : sh.chunk;
  if (cudaMemsetAsync(ws.status, 0, 3 * sizeof(unsigned), s) != cudaSuccess) return LAGP_ERR_CUDA;
  if (launch_prepare(design, sh.N, sh.p, sh.PP, sh.Npad, ws, s) != cudaSuccess) return LAGP_ERR_CUDA;
  if (launch_knn(design, sh.N, sh.p, sh.PP, sh.Npad, xref, Mc, sh.nc_max, nclose_loc, ws.cand, ws,
                 s) != cudaSuccess)
    return LAGP_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LAGP_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return LAGP_ERR_CUDA; }
  int best = 0;
  float best_ms = 0.f;
  int out = LAGP_OK;
  for (int i = 0; i < nc && out == LAGP_OK; ++i) {
    const DesignArgs a = chunk_args(sh, c, ws, 0, Mc, cand[i]);
    float ms = 0.f;
    if (run_design(a, search, sh.precision, uneven, s) != cudaSuccess ||    // warm-up
        cudaEventRecord(e0, s) != cudaSuccess ||
        run_design(a, search, sh.precision, uneven, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      out = LAGP_ERR_CUDA;
      break;
    }
    if (i == 0 || ms < best_ms) { best = i; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out != LAGP_OK) return out;
  unsigned st = 0;
  if (cudaMemcpy(&st, ws.status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LAGP_ERR_CUDA;
  if (st) return LAGP_ERR_DEVICE;
  store_tune(sh.p, sh.n_max, sh.nc_max, sh.nrays, search, uneven ? 1 : 0, cand[best]);
  *choice = encode_tune(cand[best]);
  return LAGP_OK;
}

extern "C" int laGP_tune_get(int p, int n, int N_close, int nrays, int search, int uneven,
                             int* choice) {
  if (!choice || p < 1 || p > LAGP_MAX_P) return LAGP_ERR_INVALID;
  const int R = (search != LAGP_EXHAUSTIVE) ? (nrays <= 0 ? p : nrays) : 1;
  *choice = encode_tune(lookup_tune(p, n, N_close, R, search, uneven ? 1 : 0));
  return LAGP_OK;
}

extern "C" int laGP_tune_set(int p, int n, int N_close, int nrays, int search, int uneven,
                             int choice) {
  Tune t;
  if (!decode_tune(choice, &t) || p < 1 || p > LAGP_MAX_P) return LAGP_ERR_INVALID;
  if (search != LAGP_EXHAUSTIVE && search != LAGP_RAY && search != LAGP_RAY_FULL)
    return LAGP_ERR_INVALID;
  const int R = (search != LAGP_EXHAUSTIVE) ? (nrays <= 0 ? p : nrays) : 1;
  store_tune(p, n, N_close, R, search, uneven ? 1 : 0, t);
  return LAGP_OK;
}

extern "C" size_t laGP_knn_workspace_bytes(int64_t N, int p, int64_t M, int N_close) {
  Shape sh;
  if (!make_shape(N, p, M, 1, 1, N_close, 1, LAGP_RAY, LAGP_FP64, &sh, true)) return 0;
  return layout_workspace(sh, nullptr, nullptr);
}

extern "C" int laGP_knn(const double* design, int64_t N, int p, const double* xref, int64_t M,
                        int N_close, int32_t* cand, void* workspace, size_t workspace_bytes,
                        void* stream) {
  Shape sh;
  if (!make_shape(N, p, M, 1, 1, N_close, 1, LAGP_RAY, LAGP_FP64, &sh, true))
    return LAGP_ERR_INVALID;
  if (M == 0) return LAGP_OK;
  if (!design || !xref || !cand || !workspace) return LAGP_ERR_INVALID;
  Workspace ws;
  const size_t need = layout_workspace(sh, workspace, &ws);
  if (workspace_bytes < need) return LAGP_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(ws.status, 0, 3 * sizeof(unsigned), s) != cudaSuccess) return LAGP_ERR_CUDA;
  if (launch_prepare(design, N, p, sh.PP, sh.Npad, ws, s) != cudaSuccess) return LAGP_ERR_CUDA;
  for (int64_t c0 = 0; c0 < M; c0 += sh.chunk) {
    const int64_t Mc = (M - c0 < sh.chunk) ? M - c0 : sh.chunk;
    if (launch_knn(design, N, p, sh.PP, sh.Npad, xref + c0 * p, Mc, N_close, nullptr,
                   cand + c0 * N_close, ws, s) != cudaSuccess)
      return LAGP_ERR_CUDA;
  }
  return LAGP_OK;
}

extern "C" int laGP_status(void* workspace, void* stream, unsigned* status) {
  if (!workspace || !status) return LAGP_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned host = 0;
  unsigned* dev = static_cast<unsigned*>(workspace);   // the status word leads the workspace
  if (cudaMemcpyAsync(&host, dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return LAGP_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LAGP_ERR_CUDA;
  if (cudaMemsetAsync(dev, 0, sizeof(unsigned), s) != cudaSuccess) return LAGP_ERR_CUDA;
  *status = host;
  return host ? LAGP_ERR_DEVICE : LAGP_OK;
}

extern "C" int laGP_promoted(void* workspace, void* stream, int64_t* count) {
  if (!workspace || !count) return LAGP_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned host = 0;
  // status word 2 totals the promoted locations of the call
  const unsigned* dev = static_cast<const unsigned*>(workspace) + 2;
  if (cudaMemcpyAsync(&host, dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LAGP_ERR_CUDA;
  *count = host;
  return LAGP_OK;
}

// Host form: [design | y | xref | n_loc | nclose_loc | mean | s2 | selected | tie_gap |
// nevals | device workspace]
namespace {
struct HostLayout {
  size_t design, y, xref, nloc, ncloc, mean, s2, sel, gap, nev, ws, total;
};
HostLayout host_layout(int64_t N, int p, int64_t M, int n, size_t ws_bytes) {
  HostLayout h;
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off += (b + 255) & ~(size_t)255; return o; };
  h.design = take(sizeof(double) * N * p);
  h.y = take(sizeof(double) * N);
  h.xref = take(sizeof(double) * M * p);
  h.nloc = take(sizeof(int32_t) * M);
  h.ncloc = take(sizeof(int32_t) * M);
  h.mean = take(sizeof(double) * M);
  h.s2 = take(sizeof(double) * M);
  h.sel = take(sizeof(int32_t) * M * n);
  h.gap = take(sizeof(double) * M * n);
  h.nev = take(sizeof(int32_t) * M * n);
  h.ws = take(ws_bytes);
  h.total = off;
  return h;
}
}  // namespace

extern "C" size_t laGP_host_workspace_bytes(int64_t N, int p, int64_t M, int n, int N_close,
                                            int nrays, int search, int precision) {
  size_t w = laGP_workspace_bytes(N, p, M, n, N_close, nrays, search, precision);
  if (w == 0) return 0;
  return host_layout(N, p, M, n, w).total;
}

extern "C" int laGP_build_and_predict_host(const double* design, const double* y, int64_t N,
                                           int p, const double* xref, int64_t M, int n0, int n,
                                           int N_close, double theta, double g, int search,
                                           int nrays, int precision, const int32_t* n_loc,
                                           const int32_t* nclose_loc, double* mean, double* s2,
                                           int32_t* selected, double* tie_gap, int32_t* nevals,
                                           void* workspace, size_t workspace_bytes,
                                           void* stream) {
  const size_t wsb = laGP_workspace_bytes(N, p, M, n, N_close, nrays, search, precision);
  if (wsb == 0) return LAGP_ERR_INVALID;
  if (M == 0) return LAGP_OK;
  if (!design || !y || !xref || !mean || !s2 || !workspace) return LAGP_ERR_INVALID;
  HostLayout h = host_layout(N, p, M, n, wsb);
  if (workspace_bytes < h.total) return LAGP_ERR_WORKSPACE;
  char* b = static_cast<char*>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto h2d = [&](size_t off, const void* src, size_t bytes) {
    return cudaMemcpyAsync(b + off, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
  };
  auto d2h = [&](void* dst, size_t off, size_t bytes) {
    return cudaMemcpyAsync(dst, b + off, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  };
  if (!h2d(h.design, design, sizeof(double) * N * p) || !h2d(h.y, y, sizeof(double) * N) ||
      !h2d(h.xref, xref, sizeof(double) * M * p))
    return LAGP_ERR_CUDA;
  if (n_loc && !h2d(h.nloc, n_loc, sizeof(int32_t) * M)) return LAGP_ERR_CUDA;
  if (nclose_loc && !h2d(h.ncloc, nclose_loc, sizeof(int32_t) * M)) return LAGP_ERR_CUDA;
  int rc = laGP_build_and_predict(
      reinterpret_cast<const double*>(b + h.design), reinterpret_cast<const double*>(b + h.y), N,
      p, reinterpret_cast<const double*>(b + h.xref), M, n0, n, N_close, theta, g, search, nrays,
      precision, n_loc ? reinterpret_cast<const int32_t*>(b + h.nloc) : nullptr,
      nclose_loc ? reinterpret_cast<const int32_t*>(b + h.ncloc) : nullptr,
      reinterpret_cast<double*>(b + h.mean), reinterpret_cast<double*>(b + h.s2),
      selected ? reinterpret_cast<int32_t*>(b + h.sel) : nullptr,
      tie_gap ? reinterpret_cast<double*>(b + h.gap) : nullptr,
      nevals ? reinterpret_cast<int32_t*>(b + h.nev) : nullptr, b + h.ws, wsb, stream);
  if (rc != LAGP_OK) return rc;
  if (!d2h(mean, h.mean, sizeof(double) * M) || !d2h(s2, h.s2, sizeof(double) * M))
    return LAGP_ERR_CUDA;
  if (selected && !d2h(selected, h.sel, sizeof(int32_t) * M * n)) return LAGP_ERR_CUDA;
  if (tie_gap && !d2h(tie_gap, h.gap, sizeof(double) * M * n)) return LAGP_ERR_CUDA;
  if (nevals && !d2h(nevals, h.nev, sizeof(int32_t) * M * n)) return LAGP_ERR_CUDA;
  unsigned st = 0;
  return laGP_status(b + h.ws, stream, &st);
}

// ----- local designs coupled with local inference for theta ---------------------------

extern "C" size_t laGP_mle_workspace_bytes(int64_t N, int p, int64_t M, int n, int N_close,
                                           int nrays, int search, int precision) {
  Shape sh;
  if (!mle_shape_ok(p, n) || !make_shape(N, p, M, 1, n, N_close, nrays, search, precision, &sh))
    return 0;
  return layout_workspace(sh, nullptr, nullptr) + align256(sizeof(int32_t) * sh.chunk * n);
}

extern "C" int laGP_build_and_predict_mle(const double* design, const double* y, int64_t N,
                                          int p, const double* xref, int64_t M, int n0, int n,
                                          int N_close, double theta0, double g, double tmin,
                                          double tmax, int stages, int search, int nrays,
                                          int precision, double* theta_out, double* mean,
                                          double* s2, int32_t* selected, void* workspace,
                                          size_t workspace_bytes, void* stream) {
  if ((stages != 1 && stages != 2) || !mle_shape_ok(p, n)) return LAGP_ERR_INVALID;
  if (!(tmin > 0.0) || !(tmax > tmin) || !(tmax < 1e300)) return LAGP_ERR_INVALID;
  Shape sh;
  Workspace ws;
  const int rc = check_call(N, p, xref, M, n0, n, N_close, theta0, g, search, nrays, precision,
                            design, y, mean, s2, workspace, workspace_bytes, &sh, &ws);
  if (rc != LAGP_OK) return rc > 0 ? LAGP_OK : rc;
  if (!theta_out) return LAGP_ERR_INVALID;
  const size_t base = layout_workspace(sh, nullptr, nullptr);
  if (workspace_bytes < base + align256(sizeof(int32_t) * sh.chunk * n)) return LAGP_ERR_WORKSPACE;
  int32_t* selbuf = reinterpret_cast<int32_t*>(static_cast<char*>(workspace) + base);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(ws.status, 0, 3 * sizeof(unsigned), s) != cudaSuccess) return LAGP_ERR_CUDA;
  if (launch_prepare(design, sh.N, sh.p, sh.PP, sh.Npad, ws, s) != cudaSuccess)
    return LAGP_ERR_CUDA;
  const Tune t = tune_for(sh, false);
  for (int64_t c0 = 0; c0 < sh.M; c0 += sh.chunk) {
    const int64_t Mc = (sh.M - c0 < sh.chunk) ? sh.M - c0 : sh.chunk;
    if (launch_knn(design, sh.N, sh.p, sh.PP, sh.Npad, xref + c0 * sh.p, Mc, sh.nc_max, nullptr,
                   ws.cand, ws, s) != cudaSuccess)
      return LAGP_ERR_CUDA;
    // stage 1: the design at theta0, then theta-hat on it (and the prediction there)
    const Call c{design, y, xref, theta0, g, nullptr, nullptr, mean, s2, nullptr, nullptr,
                 nullptr, nullptr};
    DesignArgs a = chunk_args(sh, c, ws, c0, Mc, t);
    a.selected = selected ? selected + c0 * n : selbuf;
    double* th = theta_out + c0;
    if (run_design(a, sh.search, sh.precision, false, s) != cudaSuccess) return LAGP_ERR_CUDA;
    if (launch_mle(design, y, sh.N, sh.p, a.xref, Mc, a.selected, n, theta0, nullptr, g, tmin,
                   tmax, th, a.mean, a.s2, nullptr, ws.status, s) != cudaSuccess)
      return LAGP_ERR_CUDA;
    if (stages == 2) {
      // stage 2: a new design at each location's estimate, and the estimate
      // again from there
      a.theta_loc = th;
      if (run_design(a, sh.search, sh.precision, false, s) != cudaSuccess) return LAGP_ERR_CUDA;
      if (launch_mle(design, y, sh.N, sh.p, a.xref, Mc, a.selected, n, theta0, th, g, tmin,
                     tmax, th, a.mean, a.s2, nullptr, ws.status, s) != cudaSuccess)
        return LAGP_ERR_CUDA;
    }
  }
  return LAGP_OK;
}
