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
  if (search == LAGP_EXHAUSTIVE) cap = (precision == LAGP_FP64) ? 16384 : 32768;
  const int64_t per_loc = (int64_t)8 * knn_cap(nc_max);
  const int64_t by_mem = ((int64_t)16 << 30) / per_loc;
  if (by_mem < cap) cap = by_mem > 128 ? by_mem : 128;
  return M < cap ? (M > 0 ? M : 1) : cap;
}

size_t layout_workspace(const Shape& sh, void* base, Workspace* ws) {
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* ptr = b ? b + off : nullptr;
    off += align256(bytes);
    return ptr;
  };
  Workspace w;
  std::memset(&w, 0, sizeof(w));
  unsigned* words = static_cast<unsigned*>(take(2 * sizeof(unsigned)));
  w.status = words;
  w.maxn2 = words ? words + 1 : nullptr;
  w.bbox_part = static_cast<double*>(take(sizeof(double) * 64 * 2 * sh.p));
  w.lo = static_cast<double*>(take(sizeof(double) * sh.p));
  w.hi = static_cast<double*>(take(sizeof(double) * sh.p));
  w.center = static_cast<double*>(take(sizeof(double) * sh.p));
  w.Xf = static_cast<float*>(take(sizeof(float) * sh.Npad * sh.PP));
  w.nx = static_cast<float*>(take(sizeof(float) * sh.Npad));
  const int64_t c = sh.chunk;
  w.knn_buf = take((size_t)8 * c * knn_cap(sh.nc_max));
  w.knn_cnt = static_cast<int32_t*>(take(sizeof(int32_t) * c));
  w.cand = static_cast<int32_t*>(take(sizeof(int32_t) * c * sh.nc_max));
  size_t s64 = 0, s32 = 0;
  if (sh.precision == LAGP_FP64) {
    if (sh.search == LAGP_EXHAUSTIVE) s64 = sizeof(double) * c * sh.n_max * sh.nc_max;
  } else {
    const size_t per = (size_t)sh.n_max * sh.n_max > ray32_g64_doubles(sh.n_max)
                           ? (size_t)sh.n_max * sh.n_max
                           : ray32_g64_doubles(sh.n_max);
    s64 = sizeof(double) * c * per;
    if (sh.search == LAGP_EXHAUSTIVE) s32 = sizeof(float) * c * sh.n_max * sh.nc_max;
  }
  w.state64 = static_cast<double*>(take(s64));
  w.state32 = static_cast<float*>(take(s32));
  w.chunk = c;
  if (ws) *ws = w;
  return off;
}

static bool make_shape(int64_t N, int p, int64_t M, int n0, int n, int N_close, int nrays,
                       int search, int precision, Shape* sh, bool knn_only = false) {
  if (p < 1 || p > LAGP_MAX_P || N < 1 || M < 0) return false;
  if (n0 < 1 || n0 > n || n > LAGP_MAX_N || n > N_close || N_close > N || N_close > 4096)
    return false;
  if (search != LAGP_EXHAUSTIVE && search != LAGP_RAY) return false;
  if (precision != LAGP_FP64 && precision != LAGP_FP32_SCORE) return false;
  if (N > (int64_t)0x7fffff00) return false;   // int32 design indices
  int R = nrays <= 0 ? p : nrays;
  if (!knn_only && search == LAGP_RAY && (R > LAGP_MAX_RAYS || R > N_close - n)) return false;
  sh->N = N;
  sh->p = p;
  sh->PP = (p + 3) / 4 * 4;
  sh->Npad = (N + LAGP_KNN_TILE - 1) / LAGP_KNN_TILE * LAGP_KNN_TILE;
  sh->M = M;
  sh->n0 = n0;
  sh->n_max = n;
  sh->nc_max = N_close;
  sh->nrays = (search == LAGP_RAY) ? R : 1;
  sh->search = search;
  sh->precision = precision;
  sh->chunk = chunk_for(M, search, precision, N_close, N);
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

extern "C" int laGP_build_and_predict(const double* design, const double* y, int64_t N, int p,
                                      const double* xref, int64_t M, int n0, int n, int N_close,
                                      double theta, double g, int search, int nrays,
                                      int precision, const int32_t* n_loc,
                                      const int32_t* nclose_loc, double* mean, double* s2,
                                      int32_t* selected, double* tie_gap, int32_t* nevals,
                                      void* workspace, size_t workspace_bytes, void* stream) {
  Shape sh;
  if (!make_shape(N, p, M, n0, n, N_close, nrays, search, precision, &sh)) return LAGP_ERR_INVALID;
  if (!(theta > 0.0) || !(g >= 0.0) || theta != theta) return LAGP_ERR_INVALID;
  if (M == 0) return LAGP_OK;
  if (!design || !y || !xref || !mean || !s2 || !workspace) return LAGP_ERR_INVALID;
  Workspace ws;
  const size_t need = layout_workspace(sh, workspace, &ws);
  if (workspace_bytes < need) return LAGP_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(ws.status, 0, sizeof(unsigned), s) != cudaSuccess) return LAGP_ERR_CUDA;
  if (launch_prepare(design, N, p, sh.PP, sh.Npad, ws, s) != cudaSuccess) return LAGP_ERR_CUDA;
  for (int64_t c0 = 0; c0 < M; c0 += sh.chunk) {
    const int64_t Mc = (M - c0 < sh.chunk) ? M - c0 : sh.chunk;
    const int32_t* ncl = nclose_loc ? nclose_loc + c0 : nullptr;
    if (launch_knn(design, N, p, sh.PP, sh.Npad, xref + c0 * p, Mc, N_close, ncl, ws.cand, ws,
                   s) != cudaSuccess)
      return LAGP_ERR_CUDA;
    DesignArgs a;
    a.X = design; a.Y = y; a.N = N; a.p = p; a.PP = sh.PP; a.xref = xref + c0 * p; a.M = Mc;
    a.cand = ws.cand; a.nc_max = N_close; a.nc_loc = ncl; a.n0 = n0; a.n_max = n;
    a.n_loc = n_loc ? n_loc + c0 : nullptr; a.theta = theta; a.g = g; a.nrays = sh.nrays;
    a.mean = mean + c0; a.s2 = s2 + c0;
    a.selected = selected ? selected + c0 * n : nullptr;
    a.tie_gap = tie_gap ? tie_gap + c0 * n : nullptr;
    a.nevals = nevals ? nevals + c0 * n : nullptr;
    a.ws = &ws;
    cudaError_t e = (precision == LAGP_FP64) ? launch_design_fp64(a, search, s)
                                             : launch_design_fp32(a, search, s);
    if (e != cudaSuccess) return LAGP_ERR_CUDA;
  }
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
  if (cudaMemsetAsync(ws.status, 0, sizeof(unsigned), s) != cudaSuccess) return LAGP_ERR_CUDA;
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
