// knn_noalloc.cu -- laGP_knn_noalloc: the kNN candidate search (the same
// kernels as laGP_knn) with its scratch space in a fixed device array that is
// part of the library image, so the caller needs no workspace allocation.
//
// Who needs this: code that may not allocate device memory at run time.
// Examples are plug-ins whose host framework owns every device byte through
// its own pool, serving loops where cudaMalloc's implicit device-wide
// synchronisation would stall unrelated streams, and embedded deployments
// with a fixed memory budget decided at load time.
#include <cstdint>
#include <mutex>

#include "../../include/lagp.h"

// The scratch array.  Every GPU that loads the library reserves this much
// device memory until the process exits.
static __device__ __align__(256) unsigned char g_knn_scratch[LAGP_KNN_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
// g_knn_scratch's device address on each device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device with that device current.
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mu;

int scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LAGP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_knn_scratch) != cudaSuccess || !addr) return LAGP_ERR_CUDA;
    g_scratch_addr[dev] = addr;
  }
  *out = g_scratch_addr[dev];
  return LAGP_OK;
}
}  // namespace

extern "C" int laGP_knn_noalloc(const double* design, int64_t N, int p, const double* xref,
                                int64_t M, int N_close, int32_t* cand, unsigned* status,
                                void* stream) {
  const size_t need = laGP_knn_workspace_bytes(N, p, M, N_close);
  if (need == 0) return LAGP_ERR_INVALID;
  if (need > (size_t)LAGP_KNN_NOALLOC_SCRATCH_BYTES) return LAGP_ERR_WORKSPACE;
  if (M == 0) return LAGP_OK;
  if (!design || !xref || !cand) return LAGP_ERR_INVALID;
  void* ws = nullptr;
  int rc = scratch_for_current_device(&ws);
  if (rc != LAGP_OK) return rc;
  // laGP_knn clears the status word and rewrites every scratch region it reads.
  rc = laGP_knn(design, N, p, xref, M, N_close, cand, ws, need, stream);
  if (rc != LAGP_OK) return rc;
  if (status) {
    // the status word leads the scratch layout
    if (cudaMemcpyAsync(status, ws, sizeof(unsigned), cudaMemcpyDeviceToDevice,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
      return LAGP_ERR_CUDA;
  }
  return LAGP_OK;
}
