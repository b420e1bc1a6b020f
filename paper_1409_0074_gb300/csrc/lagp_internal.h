// lagp_internal.h -- workspace layout and kernel launchers shared by the
// translation units of the library (not part of the public C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "kdtree.cuh"

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
  float* Btc;           // design tiles of the tensor-core kNN filter (knn_tc.cu)
  void* knn_buf;        // [chunk][cap] (float d32, int32 index) candidate buffers
  int32_t* knn_cnt;     // [chunk] surviving buffer entries (-1: stream again)
  float* knn_thr;       // [chunk] pilot thresholds of the kNN stream
  int32_t* knn_seg;     // [chunk][4] entries per buffer quarter (tensor-core filter)
  int32_t* cand;        // [chunk][nc_max] candidate design indices, nearest first
  double* state64;      // FP64 state: FP64 form, exhaustive: [chunk][nc_max][n_max]
                        // correlation cache; FP32 form: per slot, L^{-1} and its vectors
  float* state32;       // FP32 form, exhaustive: [slots][n_max][nc_max] correlation cache
  float* crow;          // FP32 form, exhaustive: [CTA slots][nc_max][PP] candidate rows
  unsigned* queue;      // [4] work counters of the persistent kernels
  int32_t* order;       // [2][chunk] work order (largest local designs first), two parts
  unsigned* order_hist; // [2][256] cost-bucket counts, then offsets
  unsigned* order_count;// [2] items per part
  uint16_t* order_key;  // [chunk] part and cost bucket
  KdTree kd;            // k-d tree over the design (LAGP_RAY_FULL; kd.perm null otherwise)
  int32_t* promote;     // [chunk] locations handed to the binary64 re-solve (LAGP_PROMOTE);
                        // status[1] counts them per launch, status[2] per call
  double* promote64;    // exhaustive re-solve: [PROMOTE_SLOTS][n_max][nc_max] FP64 cache
  int64_t chunk;
};

// CTAs of the binary64 re-solve of promoted locations (each with its own slot
// of the exhaustive correlation cache).
#define PROMOTE_SLOTS 608

// Warp slots of the persistent ray kernel and CTA slots of the persistent
// exhaustive kernels: their FP64 / correlation scratch is per slot, so a
// launch holds at most this many locations' state at a time.
#define RAY_SLOTS 6144
#define EXH_SLOTS 1216
int ray32_slots(int64_t chunk);
int exh_slots(int64_t chunk);
// floats of the tensor-core scorer's correlation cache per CTA slot
size_t exh_tc_cache_floats(int nc_max);

// Launch choices of the FP32-scoring kernels (picked by laGP_autotune, else
// the defaults).  They schedule work only: no choice changes any result.
struct Tune {
  int ray_warps;     // locations (warps) per CTA of the ray kernel: 1, 2 or 4
  int lpt;           // order uneven work largest-first (1) or by bucket-free scatter (0)
  int exh_occ;       // exhaustive kernels keep 1/exh_occ of the resident CTAs per SM: 1 or 2
};
Tune default_tune();
Tune lookup_tune(int p, int n_max, int nc_max, int nrays, int search, int uneven);
void store_tune(int p, int n_max, int nc_max, int nrays, int search, int uneven, const Tune& t);
int encode_tune(const Tune& t);
bool decode_tune(int code, Tune* t);

// CTAs of `kernel` that fit on one SM by its registers, threads and shared
// memory (dynamic `smem` plus static, plus the per-CTA reservation).
int ctas_per_sm(const void* kernel, int threads, size_t smem);

// Grid of a persistent kernel: CTAs resident at once on the device, at most
// ceil(items / per_cta) and at most slots / per_cta, so that CTA b's slots
// b * per_cta .. b * per_cta + per_cta - 1 all exist (returns -1 on a CUDA
// error or when not even one CTA has its slots).
// Residency is the larger of the runtime's occupancy figure and the count
// from the kernel's resources: a grid above residency is still correct (the
// extra CTAs start late and find less work), one below it idles SMs.
template <typename K>
int64_t persistent_grid(K kernel, int threads, size_t smem, int64_t items, int64_t slots,
                        int per_cta = 1, int occ_div = 1) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
    return -1;
  const int own = ctas_per_sm(reinterpret_cast<const void*>(kernel), threads, smem);
  if (own > per_sm) per_sm = own;
  const int64_t cap = slots / per_cta;
  if (cap < 1) return -1;
  int64_t grid = (items + per_cta - 1) / per_cta;
  int keep = per_sm / (occ_div > 0 ? occ_div : 1);
  const int64_t resident = (int64_t)sms * (keep > 0 ? keep : 1);
  if (grid > resident) grid = resident;
  if (grid > cap) grid = cap;
  return grid < 1 ? 1 : grid;
}

struct Shape {
  int64_t N;
  int p, PP;
  int64_t Npad;
  int64_t M;
  int n0, n_max, nc_max, nrays;
  int search, precision;      // precision: the form, LAGP_PROMOTE stripped
  bool promote;               // FP32 forms with LAGP_PROMOTE
  int64_t chunk;
};

// Layout of the workspace for a shape; returns total bytes.  With base != null
// fills ws with pointers into [base, base + bytes).  The workspace is the
// request part (status word first) followed by the design part; a serving
// context keeps one design part and gives each request its own request part.
size_t layout_workspace(const Shape& sh, void* base, Workspace* ws);
size_t layout_request(const Shape& sh, void* base, Workspace* ws);
size_t layout_design(const Shape& sh, void* base, Workspace* ws);

int knn_cap(int nc_max);
size_t knn_smem_stream(int PP);

cudaError_t launch_prepare(const double* X, int64_t N, int p, int PP, int64_t Npad,
                           const Workspace& ws, cudaStream_t s);
size_t knn_tc_tile_floats(int64_t Npad, int p);
cudaError_t launch_design_to_tc(int64_t N, int p, int PP, int64_t Npad, const Workspace& ws,
                                cudaStream_t s);
cudaError_t launch_knn_tc(int64_t Npad, int p, const double* xref, int64_t M, int nc_max,
                          const int32_t* nc_loc, int cap, const Workspace& ws, cudaStream_t s);
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
  const double* theta_loc; // chunk-offset per-location lengthscale, or null (theta)
  int nrays;
  int full_scope;          // ray snaps over all of X_N (LAGP_RAY_FULL)
  double* mean;            // chunk-offset outputs
  double* s2;
  int32_t* selected;       // [M][n_max] or null
  double* tie_gap;         // [M][n_max] or null
  int32_t* nevals;         // [M][n_max] or null
  const Workspace* ws;
  const int32_t* order;    // work order of the launch (device) or null
  const unsigned* count;   // items in `order` (device) or null
  bool promote;            // FP32 forms: list ill-conditioned locations in ws->promote
  Tune tune;
};

// Work order for uneven local designs: counting sort of the chunk's locations
// by descending cost bucket, split into part 0 (n <= split_n, or all when
// split_n <= 0) and part 1 (n > split_n).  Fills ws.order and ws.order_count.
cudaError_t launch_order(const DesignArgs& a, int search, int split_n, int lpt, cudaStream_t s);

// Validated shape of a call (false if an argument is out of range).
bool make_shape(int64_t N, int p, int64_t M, int n0, int n, int N_close, int nrays, int search,
                int precision, Shape* sh, bool knn_only = false);

// Arguments of one predictive call (device pointers).
struct Call {
  const double* design;
  const double* y;
  const double* xref;
  double theta, g;
  const int32_t* n_loc;
  const int32_t* nclose_loc;
  double* mean;
  double* s2;
  int32_t* selected;
  double* tie_gap;
  int32_t* nevals;
  const double* theta_loc;   // per-location lengthscale [M] or null (theta for all)
};

// Enqueues the whole path for a call on stream s: (design preparation unless
// `prepared`), then per chunk kNN, greedy design and prediction.  Returns an
// LAGP_* code.
int enqueue(const Shape& sh, const Call& c, const Workspace& ws, const Tune& t, cudaStream_t s,
            bool prepared);
Tune tune_for(const Shape& sh, bool uneven);

// Opt-in per-kernel timing (CUDA events recorded on the launch stream around
// each kernel; off unless laGP_profile(1) was called).  Suspended while a
// launch sequence is being captured into a CUDA graph.
void prof_begin(const char* name, cudaStream_t s);
void prof_end(cudaStream_t s);
void prof_suspend(bool on);

// Binary64 greedy design and prediction (design_fp64.cu): every location of
// the chunk, or with `list` the *count locations list[0 ..] (device count) on
// at most grid_cap CTAs, each with its slot of kc_slots for the exhaustive
// correlation cache.
cudaError_t launch_design_fp64(const DesignArgs& a, int search, cudaStream_t s,
                               const int32_t* list = nullptr, const unsigned* count = nullptr,
                               double* kc_slots = nullptr, int grid_cap = 0);
// Local maximum-likelihood lengthscale on the designs sel [M][n] and the
// predictive equations at it (mle.cu); the start is theta0_loc[m] when given.
bool mle_shape_ok(int p, int n);
cudaError_t launch_mle(const double* X, const double* Y, int64_t N, int p, const double* xref,
                       int64_t M, const int32_t* sel, int n, double theta0,
                       const double* theta0_loc, double g, double tmin, double tmax,
                       double* theta_out, double* mean, double* s2, int32_t* iters,
                       unsigned* status, cudaStream_t s);
// FP32-scoring ray search, one warp per location (ray32.cu); its per-location
// FP64 scratch in Workspace::state64 holds ray32_g64_doubles(n_max) doubles.
cudaError_t launch_ray32(const DesignArgs& a, cudaStream_t s);
// Exhaustive search of the LAGP_FP32_SCORE_TC form, tensor-core scoring
// (exh_tc.cu), for the locations with n <= exh_tc_max_n().
int exh_tc_max_n();
cudaError_t launch_exh_tc(const DesignArgs& a, cudaStream_t s);
size_t ray32_g64_doubles(int n_max);
// warps per CTA of the ray kernel when no launch choice is stored for a shape
int ray32_default_warps(int p, int n_max, int nc_max, int nrays);
// FP32-scoring exhaustive search with incremental CUDA-core scoring
// (design_fp32.cu), n_max <= 128: every location of the LAGP_FP32_SCORE form,
// the n > exh_tc_max_n() locations of LAGP_FP32_SCORE_TC.
cudaError_t launch_exh32(const DesignArgs& a, cudaStream_t s);

}  // namespace lagp
