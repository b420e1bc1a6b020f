// knn_noalloc.cu -- laGP_knn_noalloc: the kNN candidate search (the same
// kernels as laGP_knn) with its scratch space in a fixed device array that is
// part of the library image, so the caller needs no workspace allocation.
//
// Who needs this: code that may not allocate device memory at run time.
// Examples are plug-ins whose host framework owns every device byte through
// its own pool, serving loops where cudaMalloc's implicit device-wide
// synchronisation would stall unrelated streams, and embedded deployments
// with a fixed memory budget decided at load time.
#include <cuda.h>

#include <cstdint>
#include <mutex>

#include "../../include/lagp.h"

// The scratch array.  Every GPU that loads the library reserves this much
// device memory until the process exits.
static __device__ __align__(256) unsigned char g_knn_scratch[LAGP_KNN_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;

// g_knn_scratch's device address on each device, with the id of the context
// it was looked up in.  In host code the array's name is only a host-side
// stand-in, so the address is looked up with the device current: once per
// device, and again whenever the device's context has changed (after a
// cudaDeviceReset the module is loaded anew and the array may move).
struct Slot {
  void* addr;
  unsigned long long ctx_id;
};
Slot g_slots[kMaxDevices] = {};
std::mutex g_setup_mu;

// Driver entry points for the current context's unique id, found through the
// runtime (no link-time dependency on the driver library).
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);
ctx_get_current_fn g_get_current = nullptr;
ctx_get_id_fn g_get_id = nullptr;
bool g_entry_looked_up = false;

// Id of the calling thread's current context, or 0 when it cannot be told.
unsigned long long current_ctx_id() {
  if (!g_entry_looked_up) {
    g_entry_looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_get_current = reinterpret_cast<ctx_get_current_fn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_get_id = reinterpret_cast<ctx_get_id_fn>(f);
  }
  if (!g_get_current || !g_get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (g_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LAGP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  Slot& s = g_slots[dev];
  unsigned long long id = current_ctx_id();
  // without a context id every call looks the address up again
  if (!s.addr || id == 0 || id != s.ctx_id) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_knn_scratch) != cudaSuccess || !addr) return LAGP_ERR_CUDA;
    // the lookup initialises the context if it was not yet: read its id now
    s.addr = addr;
    s.ctx_id = current_ctx_id();
  }
  *out = s.addr;
  return LAGP_OK;
}
}  // namespace

extern "C" int laGP_knn_noalloc(const double* design, int64_t N, int p, const double* xref,
                                int64_t M, int N_close, int32_t* cand, unsigned* status,
                                void* stream) {
  const size_t need = laGP_knn_workspace_bytes(N, p, M, N_close);
  if (need == 0) return LAGP_ERR_INVALID;
  if (need > (size_t)LAGP_KNN_NOALLOC_SCRATCH_BYTES) return LAGP_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (M == 0) {
    // nothing to search; the caller's status word still reports this call
    if (status && cudaMemsetAsync(status, 0, sizeof(unsigned), s) != cudaSuccess)
      return LAGP_ERR_CUDA;
    return LAGP_OK;
  }
  if (!design || !xref || !cand) return LAGP_ERR_INVALID;
  void* ws = nullptr;
  int rc = scratch_for_current_device(&ws);
  if (rc != LAGP_OK) return rc;
  // laGP_knn clears the status word and rewrites every scratch region it reads.
  rc = laGP_knn(design, N, p, xref, M, N_close, cand, ws, need, stream);
  if (rc != LAGP_OK) return rc;
  if (status) {
    // the status word leads the scratch layout
    if (cudaMemcpyAsync(status, ws, sizeof(unsigned), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return LAGP_ERR_CUDA;
  }
  return LAGP_OK;
}
