// serve.cu -- captured launch plans (CUDA graphs) and the serving context.
//
// Plan.  laGP_plan_create records the whole launch sequence of one call (the
// same sequence laGP_build_and_predict enqueues, with the launch choices fixed
// at capture) into a CUDA graph; laGP_plan_launch replays it on any stream.
// The plan keeps the caller's pointers: refilling xref (or n_loc) in place and
// launching again predicts at the new locations.
//
// Serving context.  A context keeps one device-resident design (its bounding
// box and centred FP32 copy prepared once) in a caller-provided device arena.
// Each submitted request takes an in-flight slot (its own stream) and a region
// of the arena (its inputs, outputs and request workspace); when no slot or no
// region of the size it needs is free, submit answers LAGP_BUSY and the caller
// retries after a completed request has been polled.  Requests in different
// slots run concurrently on the device; each one's results depend on its own
// locations only, so a location's prediction is the same alone and in a mix.
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/lagp.h"
#include "common.cuh"
#include "lagp_internal.h"

using namespace lagp;

// ----- plans ------------------------------------------------------------------------
struct laGP_plan {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" int laGP_plan_create(const double* design, const double* y, int64_t N, int p,
                                const double* xref, int64_t M, int n0, int n, int N_close,
                                double theta, double g, int search, int nrays, int precision,
                                const int32_t* n_loc, const int32_t* nclose_loc, double* mean,
                                double* s2, int32_t* selected, double* tie_gap, int32_t* nevals,
                                void* workspace, size_t workspace_bytes, laGP_plan** plan) {
  if (!plan) return LAGP_ERR_INVALID;
  *plan = nullptr;
  Shape sh;
  if (!make_shape(N, p, M, n0, n, N_close, nrays, search, precision, &sh) || M < 1)
    return LAGP_ERR_INVALID;
  if (!(theta > 0.0) || !(g >= 0.0) || theta != theta) return LAGP_ERR_INVALID;
  if (!design || !y || !xref || !mean || !s2 || !workspace) return LAGP_ERR_INVALID;
  Workspace ws;
  if (workspace_bytes < layout_workspace(sh, workspace, &ws)) return LAGP_ERR_WORKSPACE;
  const Call c{design, y, xref, theta, g, n_loc, nclose_loc, mean, s2, selected, tie_gap, nevals};
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return LAGP_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  prof_suspend(true);
  int rc = LAGP_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    rc = LAGP_ERR_CUDA;
  } else {
    rc = enqueue(sh, c, ws, tune_for(sh, n_loc || nclose_loc), cs, false);
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (rc == LAGP_OK && e != cudaSuccess) rc = LAGP_ERR_CUDA;
  }
  prof_suspend(false);
  cudaStreamDestroy(cs);
  if (rc != LAGP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return LAGP_ERR_CUDA;
  }
  *plan = new laGP_plan{graph, exec};
  return LAGP_OK;
}

extern "C" int laGP_plan_launch(laGP_plan* plan, void* stream) {
  if (!plan) return LAGP_ERR_INVALID;
  return cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LAGP_OK
             : LAGP_ERR_CUDA;
}

extern "C" int laGP_plan_destroy(laGP_plan* plan) {
  if (!plan) return LAGP_ERR_INVALID;
  cudaGraphExecDestroy(plan->exec);
  cudaGraphDestroy(plan->graph);
  delete plan;
  return LAGP_OK;
}

// ----- serving context ---------------------------------------------------------------
namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Region {
  size_t off, bytes;
};

// One request's device region: [request workspace | xref | n_loc | mean | s2 | selected]
struct ReqLayout {
  size_t ws, xref, nloc, mean, s2, sel, total;
};

ReqLayout req_layout(const Shape& sh, bool want_sel) {
  ReqLayout r;
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off += up256(b); return o; };
  r.ws = take(layout_request(sh, nullptr, nullptr) + 0);
  r.xref = take(sizeof(double) * sh.M * sh.p);
  r.nloc = take(sizeof(int32_t) * sh.M);
  r.mean = take(sizeof(double) * sh.M);
  r.s2 = take(sizeof(double) * sh.M);
  r.sel = take(want_sel ? sizeof(int32_t) * sh.M * sh.n_max : 0);
  r.total = off;
  return r;
}

struct Slot {
  cudaStream_t stream;
  cudaEvent_t done;
  bool busy;
  int64_t ticket;
  Region region;
};

}  // namespace

struct laGP_ctx {
  std::mutex mu;
  const double* design;
  const double* y;
  int64_t N;
  int p, PP;
  int64_t Npad;
  double theta, g;
  int n0, N_close, search, nrays, precision;
  char* arena;
  size_t arena_bytes;
  size_t design_bytes;
  Workspace dws;               // design part (prepared once)
  std::vector<Slot> slots;
  std::vector<Region> used;    // allocated regions, sorted by offset
  unsigned* host_status;       // page-locked, one word per slot
  int64_t next_ticket;
};

namespace {

// first fit in [design_bytes, arena_bytes) between the allocated regions
bool arena_alloc(laGP_ctx* c, size_t bytes, Region* out) {
  size_t at = up256(c->design_bytes);
  size_t i = 0;
  for (; i < c->used.size(); ++i) {
    if (c->used[i].off >= at + bytes) break;
    const size_t end = up256(c->used[i].off + c->used[i].bytes);
    if (end > at) at = end;
  }
  if (at + bytes > c->arena_bytes) return false;
  *out = Region{at, bytes};
  c->used.insert(c->used.begin() + i, *out);
  return true;
}

void arena_free(laGP_ctx* c, const Region& r) {
  for (size_t i = 0; i < c->used.size(); ++i)
    if (c->used[i].off == r.off) {
      c->used.erase(c->used.begin() + i);
      return;
    }
}

Shape ctx_shape(const laGP_ctx* c, int64_t M, int n, bool* ok) {
  Shape sh;
  *ok = make_shape(c->N, c->p, M, c->n0, n, c->N_close, c->nrays, c->search, c->precision, &sh);
  return sh;
}

}  // namespace

extern "C" size_t laGP_ctx_design_bytes(int64_t N, int p) {
  Shape sh;
  if (!make_shape(N, p, 1, 1, 1, 1, 1, LAGP_EXHAUSTIVE, LAGP_FP64, &sh)) return 0;
  return up256(layout_design(sh, nullptr, nullptr));
}

extern "C" size_t laGP_ctx_request_bytes(int64_t N, int p, int64_t M, int n, int N_close,
                                         int nrays, int search, int precision,
                                         int want_selected) {
  Shape sh;
  if (M < 1 || !make_shape(N, p, M, 1, n, N_close, nrays, search, precision, &sh)) return 0;
  return req_layout(sh, want_selected != 0).total;
}

extern "C" int laGP_ctx_create(const double* design, const double* y, int64_t N, int p,
                               double theta, double g, int n0, int N_close, int search,
                               int nrays, int precision, void* arena, size_t arena_bytes,
                               int max_inflight, laGP_ctx** out) {
  if (!out) return LAGP_ERR_INVALID;
  *out = nullptr;
  Shape sh;
  if (!make_shape(N, p, 1, n0, n0, N_close, nrays, search, precision, &sh))
    return LAGP_ERR_INVALID;
  if (!(theta > 0.0) || !(g >= 0.0) || theta != theta) return LAGP_ERR_INVALID;
  if (!design || !y || !arena || max_inflight < 1 || max_inflight > 64) return LAGP_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(arena) & 255) return LAGP_ERR_INVALID;
  const size_t dbytes = up256(layout_design(sh, nullptr, nullptr));
  if (arena_bytes < dbytes) return LAGP_ERR_WORKSPACE;
  laGP_ctx* c = new laGP_ctx();
  c->design = design; c->y = y; c->N = N; c->p = p; c->PP = sh.PP; c->Npad = sh.Npad;
  c->theta = theta; c->g = g; c->n0 = n0; c->N_close = N_close; c->search = search;
  c->nrays = nrays; c->precision = precision;
  c->arena = static_cast<char*>(arena); c->arena_bytes = arena_bytes; c->design_bytes = dbytes;
  c->next_ticket = 1;
  std::memset(&c->dws, 0, sizeof(c->dws));
  layout_design(sh, c->arena, &c->dws);
  int rc = LAGP_OK;
  if (cudaHostAlloc(&c->host_status, sizeof(unsigned) * max_inflight, cudaHostAllocDefault) !=
      cudaSuccess) {
    delete c;
    return LAGP_ERR_CUDA;
  }
  for (int i = 0; i < max_inflight && rc == LAGP_OK; ++i) {
    Slot s{};
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = LAGP_ERR_CUDA;
      break;
    }
    if (cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(s.stream);
      rc = LAGP_ERR_CUDA;
      break;
    }
    c->slots.push_back(s);
  }
  // prepare the design once, on the first slot's stream
  if (rc == LAGP_OK &&
      (launch_prepare(design, N, p, sh.PP, sh.Npad, c->dws, c->slots[0].stream) != cudaSuccess ||
       cudaStreamSynchronize(c->slots[0].stream) != cudaSuccess))
    rc = LAGP_ERR_CUDA;
  if (rc != LAGP_OK) {
    laGP_ctx_destroy(c);
    return rc;
  }
  *out = c;
  return LAGP_OK;
}

extern "C" int laGP_ctx_submit(laGP_ctx* c, const double* xref, int64_t M, int n,
                               const int32_t* n_loc, double* mean, double* s2,
                               int32_t* selected, int64_t* ticket) {
  if (!c || !xref || !mean || !s2 || !ticket || M < 1) return LAGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  bool ok = false;
  const Shape sh = ctx_shape(c, M, n, &ok);
  if (!ok) return LAGP_ERR_INVALID;
  int si = -1;
  for (size_t i = 0; i < c->slots.size(); ++i)
    if (!c->slots[i].busy) { si = (int)i; break; }
  if (si < 0) return LAGP_BUSY;
  const ReqLayout L = req_layout(sh, selected != nullptr);
  Region reg;
  if (!arena_alloc(c, L.total, &reg)) return LAGP_BUSY;
  Slot& s = c->slots[si];
  char* b = c->arena + reg.off;
  Workspace ws = c->dws;
  layout_request(sh, b + L.ws, &ws);
  const cudaStream_t st = s.stream;
  int rc = LAGP_OK;
  if (cudaMemcpyAsync(b + L.xref, xref, sizeof(double) * M * c->p, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      (n_loc && cudaMemcpyAsync(b + L.nloc, n_loc, sizeof(int32_t) * M, cudaMemcpyHostToDevice,
                                st) != cudaSuccess))
    rc = LAGP_ERR_CUDA;
  if (rc == LAGP_OK) {
    const Call call{c->design, c->y, reinterpret_cast<const double*>(b + L.xref), c->theta, c->g,
                    n_loc ? reinterpret_cast<const int32_t*>(b + L.nloc) : nullptr, nullptr,
                    reinterpret_cast<double*>(b + L.mean), reinterpret_cast<double*>(b + L.s2),
                    selected ? reinterpret_cast<int32_t*>(b + L.sel) : nullptr, nullptr, nullptr};
    rc = enqueue(sh, call, ws, tune_for(sh, n_loc != nullptr), st, true);
  }
  if (rc == LAGP_OK &&
      (cudaMemcpyAsync(mean, b + L.mean, sizeof(double) * M, cudaMemcpyDeviceToHost, st) !=
           cudaSuccess ||
       cudaMemcpyAsync(s2, b + L.s2, sizeof(double) * M, cudaMemcpyDeviceToHost, st) !=
           cudaSuccess ||
       (selected && cudaMemcpyAsync(selected, b + L.sel, sizeof(int32_t) * M * n,
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
       cudaMemcpyAsync(c->host_status + si, ws.status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                       st) != cudaSuccess ||
       cudaEventRecord(s.done, st) != cudaSuccess))
    rc = LAGP_ERR_CUDA;
  if (rc != LAGP_OK) {
    cudaStreamSynchronize(st);   // nothing of this request may still use its region
    arena_free(c, reg);
    return rc;
  }
  s.busy = true;
  s.ticket = c->next_ticket++;
  s.region = reg;
  *ticket = s.ticket;
  return LAGP_OK;
}

extern "C" int laGP_ctx_poll(laGP_ctx* c, int64_t ticket, int* done) {
  if (!c || !done) return LAGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  for (size_t i = 0; i < c->slots.size(); ++i) {
    Slot& s = c->slots[i];
    if (!s.busy || s.ticket != ticket) continue;
    const cudaError_t q = cudaEventQuery(s.done);
    if (q == cudaErrorNotReady) {
      *done = 0;
      return LAGP_OK;
    }
    *done = 1;
    s.busy = false;
    arena_free(c, s.region);
    if (q != cudaSuccess) return LAGP_ERR_CUDA;
    return c->host_status[i] ? LAGP_ERR_DEVICE : LAGP_OK;
  }
  return LAGP_ERR_INVALID;   // unknown or already collected ticket
}

extern "C" int laGP_ctx_wait(laGP_ctx* c, int64_t ticket) {
  if (!c) return LAGP_ERR_INVALID;
  cudaEvent_t ev = nullptr;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto& s : c->slots)
      if (s.busy && s.ticket == ticket) ev = s.done;
  }
  if (!ev) return LAGP_ERR_INVALID;
  if (cudaEventSynchronize(ev) != cudaSuccess) return LAGP_ERR_CUDA;
  int done = 0;
  return laGP_ctx_poll(c, ticket, &done);
}

extern "C" int laGP_ctx_capacity(laGP_ctx* c, size_t* largest_free, int* free_slots) {
  if (!c || !largest_free || !free_slots) return LAGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  size_t at = up256(c->design_bytes), best = 0;
  for (const Region& r : c->used) {
    if (r.off > at && r.off - at > best) best = r.off - at;
    const size_t end = up256(r.off + r.bytes);
    if (end > at) at = end;
  }
  if (c->arena_bytes > at && c->arena_bytes - at > best) best = c->arena_bytes - at;
  int f = 0;
  for (const auto& s : c->slots) f += s.busy ? 0 : 1;
  *largest_free = best;
  *free_slots = f;
  return LAGP_OK;
}

extern "C" int laGP_ctx_destroy(laGP_ctx* c) {
  if (!c) return LAGP_ERR_INVALID;
  for (auto& s : c->slots) {
    cudaStreamSynchronize(s.stream);
    cudaEventDestroy(s.done);
    cudaStreamDestroy(s.stream);
  }
  if (c->host_status) cudaFreeHost(c->host_status);
  delete c;
  return LAGP_OK;
}
