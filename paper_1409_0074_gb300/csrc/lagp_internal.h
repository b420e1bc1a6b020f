// lagp_internal.h -- workspace layout and kernel launchers shared by the
// translation units of the library (not part of the public C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lagp {

// Device buffers carved out of the caller's workspace.  Per-location arrays
// cover one chunk of at most `chunk` predictive locations; chunks run in
// sequence on the caller's stream.
struct Workspace {
  unsigned* status;     // device status word (LAGP_DEV_* bits)
  unsigned* maxn2;      // largest squared norm of the centred FP32 design (bits)
  double* bbox_part;    // [64][2p] partial bounding boxes
  double* lo;           // [p] bounding box of the design
  double* hi;           // [p]
  double* center;       // [p] box centre, origin of the FP32 coordinates
  float* Xf;            // [Npad][PP] centred FP32 design, PP = p rounded up to 4
  float* nx;            // [Npad] squared norms of Xf rows
  void* knn_buf;        // [chunk][cap] (float d32, int32 index) candidate buffers
  int32_t* knn_cnt;     // [chunk] surviving buffer entries
  int32_t* cand;        // [chunk][nc_max] candidate design indices, nearest first
  double* state64;      // per-location FP64 state: FP64 form [chunk][nc_max][n_max]
                        // correlation cache (exhaustive); FP32 form [chunk][n_max][n_ld] L^{-1}
  float* state32;       // FP32 form, exhaustive: [chunk][n_max][nc_max] correlation cache
  int64_t chunk;
};

struct Shape {
  int64_t N;
  int p, PP;
  int64_t Npad;
  int64_t M;
  int n0, n_max, nc_max, nrays;
  int search, precision;
  int64_t chunk;
};

// Layout of the workspace for a shape; returns total bytes.  With base != null
// fills ws with pointers into [base, base + bytes).
size_t layout_workspace(const Shape& sh, void* base, Workspace* ws);

int knn_cap(int nc_max);
size_t knn_smem_stream(int PP);

cudaError_t launch_prepare(const double* X, int64_t N, int p, int PP, int64_t Npad,
                           const Workspace& ws, cudaStream_t s);
cudaError_t launch_knn(const double* X, int64_t N, int p, int PP, int64_t Npad,
                       const double* xref, int64_t M, int nc_max, const int32_t* nc_loc,
                       int32_t* cand, const Workspace& ws, cudaStream_t s);

// Greedy local design and prediction for one chunk of locations.
struct DesignArgs {
  const double* X;
  const double* Y;
  int64_t N;
  int p, PP;
  const double* xref;      // chunk-offset
  int64_t M;               // locations in this chunk
  const int32_t* cand;     // [M][nc_max]
  int nc_max;
  const int32_t* nc_loc;   // chunk-offset or null
  int n0, n_max;
  const int32_t* n_loc;    // chunk-offset or null
  double theta, g;
  int nrays;
  double* mean;            // chunk-offset outputs
  double* s2;
  int32_t* selected;       // [M][n_max] or null
  double* tie_gap;         // [M][n_max] or null
  int32_t* nevals;         // [M][n_max] or null
  const Workspace* ws;
};

// Opt-in per-kernel timing (CUDA events recorded on the launch stream around
// each kernel; off unless laGP_profile(1) was called).
void prof_begin(const char* name, cudaStream_t s);
void prof_end(cudaStream_t s);

cudaError_t launch_design_fp64(const DesignArgs& a, int search, cudaStream_t s);
// FP32-scoring ray search, one warp per location (ray32.cu); its per-location
// FP64 scratch in Workspace::state64 holds ray32_g64_doubles(n_max) doubles.
cudaError_t launch_ray32(const DesignArgs& a, cudaStream_t s);
// FP32-scoring exhaustive search with tensor-core scoring (exh_tc.cu), n_max <= 64.
bool exh_tc_supported(int n_max);
cudaError_t launch_exh_tc(const DesignArgs& a, cudaStream_t s);
size_t ray32_g64_doubles(int n_max);
cudaError_t launch_design_fp32(const DesignArgs& a, int search, cudaStream_t s);

}  // namespace lagp
