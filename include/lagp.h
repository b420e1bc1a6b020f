/*
 * lagp.h -- C ABI of the GB300 (sm_103a) library for local approximate
 * Gaussian process prediction with greedy ALC local designs.
 *
 * Method: Gramacy & Haaland, "Speeding up neighborhood search in local
 * Gaussian process prediction" (arXiv:1409.0074).  For every predictive
 * location x:
 *   1. the N_close nearest design points are the candidates (Sec 2.2);
 *   2. the local design starts from the n0 nearest candidates;
 *   3. for j = n0 .. n-1 one candidate is added, the one maximising the
 *      reduction in predictive variance at x (ALC, the integrand of Eq. alc),
 *      found by exhaustive scoring of every unselected candidate (Sec 2.2) or
 *      by the ray search of Sec 4 (Brent line searches along rays leaving x,
 *      the best point snapped to the nearest unselected candidate); K_j^{-1}
 *      is extended by the partitioned-inverse update (Sec 2.2);
 *   4. the predictive mean and scale of Eq. predgp and Eq. preds2 are returned
 *      (Student-t with n degrees of freedom).
 * Correlation: isotropic Gaussian exp(-||x - x'||^2 / theta) with nugget g on
 * self-correlations (Sec 2.1).
 *
 * Conventions for every entry point below:
 *   - Pointers marked "device" are CUDA device pointers; "host" are host
 *     pointers.  Arrays are dense, row-major, binary64 unless stated.
 *   - The caller owns every buffer.  The library allocates no device memory:
 *     scratch space comes from the caller's `workspace`, sized by
 *     laGP_workspace_bytes (a serving context sub-allocates from a
 *     caller-provided arena).  The library never frees caller memory.  Plans
 *     and serving contexts own CUDA objects (a graph; streams, events and a
 *     small page-locked status array) until they are destroyed.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device entry
 *     points only enqueue work; a return of LAGP_OK means "enqueued".  Errors
 *     found on the device are collected in a status word inside the workspace,
 *     read by laGP_status.
 *   - Errors are returned as negative codes; nothing is printed.
 */
#ifndef LAGP_H
#define LAGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Search for the next design point (Sec 2.2 exhaustive, Sec 4 rays).
 * LAGP_RAY snaps a ray step's best point to the nearest unselected candidate
 * (the N_close nearest design points).  LAGP_RAY_FULL snaps it to the nearest
 * point of the whole design X_N outside the local design (Sec 5 places no N'
 * limit on ray searches), through a k-d tree over X_N built with the design's
 * preparation; ray starts still come from the candidates, and ties go to the
 * point nearer x, then to the lower design index. */
#define LAGP_EXHAUSTIVE 0
#define LAGP_RAY 1
#define LAGP_RAY_FULL 2

/* Arithmetic of the greedy loop.
 * LAGP_FP64: every step in binary64 with the paper's explicit K_j^{-1} and
 *   partitioned-inverse update, in a fixed operation order (the parity form).
 * LAGP_FP32_SCORE: candidate and ray scoring in FP32 through the inverse
 *   Cholesky factor L_j^{-1} (k^T K^{-1} k = |L^{-1} k|^2); the factor update,
 *   its Schur complement and the predictive equations stay in binary64.
 *   Exhaustive search keeps every candidate's running |L^{-1} k|^2 and
 *   (L^{-1} k) . (L^{-1} k(x)), extended by one term per step (the factor
 *   only gains a row), on the FP32 CUDA cores.
 * LAGP_FP32_SCORE_TC: as LAGP_FP32_SCORE, but exhaustive search forms all of
 *   W = Kc L_j^{-T} at every step as a dense contraction on the tensor cores
 *   (3xTF32 split products, FP32 accumulation) for local designs up to 64
 *   points (larger ones as LAGP_FP32_SCORE).  Same method and tolerances,
 *   other rounding; ray search is the same as LAGP_FP32_SCORE.
 *
 * LAGP_PROMOTE, OR-ed into either FP32 form: precision promotion.  Every form
 * computes the Schur complements v = 1 + g - k^T K_j^{-1} k of the points a
 * location adds (the pivots of the partitioned update, Sec 2.2) in binary64.
 * The FP32 estimate of a candidate's v carries an absolute error of a few
 * 1e-7 (FP32 rounding of the correlations and of L_j^{-1}), so once a local
 * design's pivots fall to a few 1e-5 the FP32 scores no longer rank the
 * candidates.  With LAGP_PROMOTE, a location whose smallest pivot is below
 * LAGP_PROMOTE_PIVOT is solved again within the same call by the binary64
 * kernels (its results then equal those of LAGP_FP64) and its FP32 results
 * are overwritten.  Measured on seeded uniform designs: the 8-d, N = 1e6,
 * theta = 1 workload meets the FP32 accuracy bar without it and would promote
 * about 3 in 10,000 ray locations (a binary64 ray location takes ~29 ms on
 * its own, a tail added to the call); the 4-d, N = 1e5, theta = 0.25 workload
 * has smallest pivots of 1.5e-6 .. 8.4e-6, where the FP32 choice differed
 * from the binary64 one at 17 to 29 of the 44 greedy steps of every location,
 * and is promoted whole.  laGP_promoted reports how many locations the last
 * call promoted. */
#define LAGP_FP64 0
#define LAGP_FP32_SCORE 1
#define LAGP_FP32_SCORE_TC 2
#define LAGP_PROMOTE 16
#define LAGP_PROMOTE_PIVOT 3e-5

/* Return codes. */
#define LAGP_OK 0
#define LAGP_ERR_INVALID (-1)   /* an argument is out of range or a pointer is NULL */
#define LAGP_ERR_WORKSPACE (-2) /* workspace_bytes is below laGP_workspace_bytes */
#define LAGP_ERR_CUDA (-3)      /* a CUDA call or kernel launch failed */
#define LAGP_ERR_DEVICE (-4)    /* laGP_status: the device reported a failure */
#define LAGP_BUSY 1             /* laGP_ctx_submit: no free slot or arena region now */

/* Device status bits reported by laGP_status. */
#define LAGP_STATUS_TIMEOUT 1u      /* a bounded on-device wait ran out */
#define LAGP_STATUS_CAPACITY 2u     /* too many exactly tied kNN distances */
#define LAGP_STATUS_NUMERIC 4u      /* a Schur complement v <= 0: that location's
                                       mean and s2 are NaN */

/*
 * Bytes of device workspace laGP_build_and_predict needs for these sizes.
 * Arguments as in laGP_build_and_predict (n and N_close are the maxima when
 * per-location arrays are used).  Returns 0 when the sizes are invalid.
 */
size_t laGP_workspace_bytes(int64_t N, int p, int64_t M, int n, int N_close, int nrays,
                            int search, int precision);

/*
 * Local approximate GP prediction at M locations (steps 1-4 above).
 *
 *   design    device [N][p]   design X_N
 *   y         device [N]      responses Y_N
 *   N, p      design size (N >= N_close) and input dimension (1 <= p <= 16)
 *   xref      device [M][p]   predictive locations
 *   M         number of locations (>= 0; 0 is a no-op)
 *   n0        starting design size (1 <= n0 <= n)
 *   n         final local design size (n <= N_close, n <= 128)
 *   N_close   candidates per location (n <= N_close <= min(N, 4096))
 *   theta     lengthscale (> 0)
 *   g         nugget (>= 0)
 *   search    LAGP_EXHAUSTIVE, LAGP_RAY or LAGP_RAY_FULL
 *   nrays     rays per step of a ray search (<= 0 selects p; at most 16 and at
 *             most N_close - n); ignored for LAGP_EXHAUSTIVE
 *   precision LAGP_FP64, LAGP_FP32_SCORE or LAGP_FP32_SCORE_TC, the FP32 forms
 *             optionally OR-ed with LAGP_PROMOTE
 *   n_loc     device [M] int32 or NULL: per-location final size (each in
 *             [n0, n]); NULL gives every location n
 *   nclose_loc device [M] int32 or NULL: per-location N_close (each in
 *             [that location's n, N_close]); NULL gives N_close
 *   mean      device [M] out: predictive mean, Eq. predgp
 *   s2        device [M] out: predictive scale sigma^2, Eq. preds2, with
 *             K(x,x) = 1 + g; the degrees of freedom are the location's n and
 *             the predictive variance is s2 * n / (n - 2)
 *   selected  device [M][n] int32 out or NULL: design indices in selection
 *             order (the n0 nearest first); entries past a location's n are -1
 *             (with LAGP_RAY_FULL a design may hold points outside the
 *             candidates)
 *   tie_gap   device [M][n] out or NULL: entry j - n0 holds the smallest
 *             relative gap among the comparisons that decided step j (argmax
 *             of ALC; for rays also Brent's comparisons, the s = 0 check and
 *             the snap); 0 elsewhere
 *   nevals    device [M][n] int32 out or NULL: ALC evaluations of ray step j
 *             at entry j - n0 (0 for the exhaustive search)
 *   workspace device scratch of workspace_bytes >= laGP_workspace_bytes(...)
 *   stream    cudaStream_t
 *
 * A location whose update meets v <= 0 gets NaN in mean and s2 and sets
 * LAGP_STATUS_NUMERIC; the other locations are unaffected.
 */
int laGP_build_and_predict(const double* design, const double* y, int64_t N, int p,
                           const double* xref, int64_t M, int n0, int n, int N_close,
                           double theta, double g, int search, int nrays, int precision,
                           const int32_t* n_loc, const int32_t* nclose_loc, double* mean,
                           double* s2, int32_t* selected, double* tie_gap, int32_t* nevals,
                           void* workspace, size_t workspace_bytes, void* stream);

/*
 * Step 1 alone (Sec 2.2): the N_close nearest design points of each location,
 * ordered by squared Euclidean distance computed in binary64 as
 * sum_k (X_ik - x_k)^2 (ascending k), ties to the lower index.
 *   cand      device [M][N_close] int32 out.  When a location's search ends
 *             with LAGP_STATUS_CAPACITY or LAGP_STATUS_TIMEOUT, its list may be
 *             incomplete; the missing ranks repeat an index of the design.
 *   workspace sized by laGP_knn_workspace_bytes(N, p, M, N_close)
 */
size_t laGP_knn_workspace_bytes(int64_t N, int p, int64_t M, int N_close);
int laGP_knn(const double* design, int64_t N, int p, const double* xref, int64_t M,
             int N_close, int32_t* cand, void* workspace, size_t workspace_bytes, void* stream);

/*
 * laGP_knn without a workspace: the same candidate search, with its scratch
 * space in a fixed device array inside the library instead of caller memory.
 * It serves callers that may not allocate device memory while they run (a
 * host framework that owns all device memory through its own pool, a serving
 * loop that cannot afford cudaMalloc's implicit device synchronisation, a
 * deployment with a memory budget fixed at load time).  The paper has no
 * counterpart; this is a deployment variant of step 1.
 *
 *   design, N, p, xref, M, N_close, cand: as in laGP_knn (device pointers)
 *   status    device unsigned* or NULL: receives the LAGP_STATUS_* bits of
 *             this call once the stream reaches the end of it (0 when M = 0)
 *   stream    cudaStream_t
 * Limits: the scratch needed, laGP_knn_workspace_bytes(N, p, M, N_close),
 * must not exceed LAGP_KNN_NOALLOC_SCRATCH_BYTES (64 MiB); larger requests
 * return LAGP_ERR_WORKSPACE before any device work.  Every GPU that loads the
 * library holds that array until the process exits.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  A call
 * that finds the device under a new context (after cudaDeviceReset) looks the
 * address up again, so it too belongs outside a stream capture.  All calls
 * share the one array and each overwrites it: calls that overlap on the GPU
 * (concurrent streams, threads or devices sharing a context) race, so
 * serialise them.  No device memory is allocated or freed.
 */
#define LAGP_KNN_NOALLOC_SCRATCH_BYTES (64u << 20)
int laGP_knn_noalloc(const double* design, int64_t N, int p, const double* xref, int64_t M,
                     int N_close, int32_t* cand, unsigned* status, void* stream);

/*
 * Local inference for the lengthscale on given local designs (Sec 5: local
 * designs are coupled with Newton-like maximisation of the local posterior of
 * theta; Sec 2.1, Eq. gpk), then the predictive equations (Eq. predgp,
 * preds2) at the estimate.  Binary64.  For location m the design is the rows
 * sel[m][0..n-1] of `design`.  theta maximises the marginal likelihood of Eq.
 * gpk (reference prior on tau^2, flat prior on theta over [tmin, tmax], nugget
 * g fixed, 1 + g on the diagonal of K) by Newton's method from theta0,
 * safeguarded by a bracket kept from the sign of the derivative (midpoint
 * steps where Newton's would leave it or the curvature is not negative), to a
 * relative step or bracket of 1e-10, 200 iterations at most.  With `sel` the
 * selected output of laGP_build_and_predict at theta0 this is the first stage
 * of a local design coupled with local inference; a second stage calls
 * laGP_build_and_predict again at the estimate.
 *   design, y   device [N][p], [N] binary64
 *   xref        device [M][p] binary64
 *   sel         device [M][n] int32 design indices (each in [0, N))
 *   n           local design size, 1 <= n <= 64 (n <= N); 1 <= p <= 16
 *   theta0, g   start (theta0 > 0, clamped to the range) and nugget (g >= 0)
 *   tmin, tmax  the range, 0 < tmin < tmax
 *   theta_out, mean, s2  device [M] binary64 out; iters device [M] int32 out or NULL
 *   status      device unsigned*, cleared by the call; LAGP_STATUS_NUMERIC when
 *               a location's K is not positive definite at its estimate or an
 *               index in sel is out of range (that location's outputs are NaN)
 * Asynchronous on `stream`.  Returns LAGP_OK, LAGP_ERR_INVALID (before any
 * device work) or LAGP_ERR_CUDA.  No device memory is allocated.
 */
int laGP_mle_predict(const double* design, const double* y, int64_t N, int p,
                     const double* xref, int64_t M, const int32_t* sel, int n, double theta0,
                     double g, double tmin, double tmax, double* theta_out, double* mean,
                     double* s2, int32_t* iters, unsigned* status, void* stream);

/*
 * Local designs coupled with local inference for the lengthscale, in one call
 * (Sec 5: every local design is paired with Newton-like maximisation of the
 * local posterior of theta, and a second stage may redesign at the estimate;
 * Sec 2.1, Eq. gpk).  For each location, after the kNN candidates:
 *   stage 1: the greedy design at theta0 (as laGP_build_and_predict), then
 *            theta-hat_1 on it (as laGP_mle_predict, started at theta0);
 *   stage 2 (stages = 2): a new greedy design at the location's own
 *            theta-hat_1, then theta-hat_2 on it, started at theta-hat_1.
 * mean and s2 are the predictive equations at the last estimate on the last
 * design (Eq. predgp, preds2; df = n).
 *   design, y, N, p, xref, M, n0, n, N_close, g, search, nrays, precision: as in
 *             laGP_build_and_predict, with 1 <= n <= 64 and every location of
 *             size n
 *   theta0    start of the estimate and lengthscale of the first design (> 0)
 *   tmin, tmax the range of theta (0 < tmin < tmax)
 *   stages    1 or 2
 *   theta_out device [M] out: the last estimate
 *   mean, s2  device [M] out
 *   selected  device [M][n] int32 out or NULL: the last design, in selection order
 *   workspace device scratch of at least laGP_mle_workspace_bytes(...) bytes
 * A location whose design or estimate fails gets NaN and sets
 * LAGP_STATUS_NUMERIC (read with laGP_status).  Asynchronous on `stream`.
 */
size_t laGP_mle_workspace_bytes(int64_t N, int p, int64_t M, int n, int N_close, int nrays,
                                int search, int precision);
int laGP_build_and_predict_mle(const double* design, const double* y, int64_t N, int p,
                               const double* xref, int64_t M, int n0, int n, int N_close,
                               double theta0, double g, double tmin, double tmax, int stages,
                               int search, int nrays, int precision, double* theta_out,
                               double* mean, double* s2, int32_t* selected, void* workspace,
                               size_t workspace_bytes, void* stream);

/*
 * Pre-scaled inputs (Sec 5.3, the subset table's "rays with pre-scaled
 * inputs"): a crude global analysis fits a separable Gaussian correlation
 * K_ab = exp(-sum_k (x_ak - x_bk)^2 / theta_k), diagonal 1 + g, to a random
 * subset of the design by maximum likelihood (the reference-prior likelihood
 * of Eq. gpk, as for the local lengthscale, with one theta per input), and
 * every input coordinate is then divided by sqrt(theta_k); the local
 * approximation runs on the scaled design and locations with theta = 1, the
 * global correlation in scaled coordinates.
 *
 * laGP_sep_mle_workspace_bytes: device workspace of laGP_sep_mle for a
 * subset of n_sub rows (2 <= n_sub <= 1024) in p <= 16 inputs (0 otherwise);
 * about 8 n_sub^2 bytes.
 *
 * laGP_sep_mle: the fit on the design rows subset[0 .. n_sub - 1].
 *   design, y  device [N][p], [N] (as in laGP_build_and_predict)
 *   subset     device [n_sub] int32 row indices (the caller's random draw)
 *   g          fixed nugget (>= 0)
 *   theta0     start, the same for every input (> 0)
 *   tmin, tmax the box of every theta_k (0 < tmin <= tmax)
 *   maxit      iterations at most (>= 1)
 *   theta_out  device [p]: the estimate
 *   info       device [3] int32 or NULL: iterations, likelihood evaluations,
 *              status (0 ok, 1 the start's K not positive definite, 2 a
 *              subset index outside [0, N))
 * Maximiser: BFGS on log theta from log theta0 with an Armijo line search
 * (halvings from a step capped at 2 per coordinate), projected on the box,
 * ending when a step moves no coordinate by more than 1e-9.  Each likelihood
 * evaluation inverts K by Gauss-Jordan elimination (K is positive definite;
 * its pivots give log|K|).  Unlike the other entry points this one blocks:
 * it synchronises `stream` after every evaluation to read the done flag.
 * Returns LAGP_OK, LAGP_ERR_INVALID / _WORKSPACE for bad arguments,
 * LAGP_ERR_CUDA, or LAGP_ERR_DEVICE when the status is not 0.
 *
 * laGP_prescale: X_out[r][k] = X[r][k] / sqrt(theta[k]) for rows r < rows
 * (device arrays; X_out may be X).  Returns LAGP_OK, LAGP_ERR_INVALID or
 * LAGP_ERR_CUDA.
 */
size_t laGP_sep_mle_workspace_bytes(int n_sub, int p);
int laGP_sep_mle(const double* design, const double* y, int64_t N, int p, const int32_t* subset,
                 int n_sub, double g, double theta0, double tmin, double tmax, int maxit,
                 double* theta_out, int32_t* info, void* workspace, size_t workspace_bytes,
                 void* stream);
int laGP_prescale(const double* X, int64_t rows, int p, const double* theta, double* X_out,
                  void* stream);

/*
 * Waits for `stream`, then reads and clears the device status word of the
 * workspace.  *status receives the LAGP_STATUS_* bits.  Returns LAGP_OK when
 * no bit was set, LAGP_ERR_DEVICE when one was, LAGP_ERR_CUDA when the wait
 * or the copy failed.
 */
int laGP_status(void* workspace, void* stream, unsigned* status);

/*
 * Waits for `stream`, then reads how many locations the last call on this
 * workspace (laGP_build_and_predict, its plan replay or host form,
 * laGP_build_and_predict_mle: every design pass counts) handed to the
 * binary64 re-solve of LAGP_PROMOTE (0 without the flag).  Each call resets
 * the count when it starts.  Returns LAGP_OK, or LAGP_ERR_INVALID for a NULL
 * argument, LAGP_ERR_CUDA when the copy failed.
 */
int laGP_promoted(void* workspace, void* stream, int64_t* count);

/*
 * Host-buffer form of laGP_build_and_predict: design, y, xref, n_loc,
 * nclose_loc, mean, s2, selected, tie_gap and nevals are HOST pointers (pinned
 * memory makes the copies asynchronous with respect to the host).  Inputs are
 * copied into the device workspace, the device path runs on `stream`, the
 * outputs are copied back and the stream is synchronised before returning;
 * device-side status bits are returned as LAGP_ERR_DEVICE.
 *   workspace device scratch of at least laGP_host_workspace_bytes(...)
 */
size_t laGP_host_workspace_bytes(int64_t N, int p, int64_t M, int n, int N_close, int nrays,
                                 int search, int precision);
int laGP_build_and_predict_host(const double* design, const double* y, int64_t N, int p,
                                const double* xref, int64_t M, int n0, int n, int N_close,
                                double theta, double g, int search, int nrays, int precision,
                                const int32_t* n_loc, const int32_t* nclose_loc, double* mean,
                                double* s2, int32_t* selected, double* tie_gap, int32_t* nevals,
                                void* workspace, size_t workspace_bytes, void* stream);

/*
 * Launch choices (FP32-scoring form).  The persistent kernels have launch
 * choices that change scheduling only, never a result: locations (warps) per
 * CTA of the ray kernel (1, 2 or 4), largest-first ordering of uneven work
 * (n_loc / nclose_loc given), and the fraction of resident CTAs per SM the
 * exhaustive kernels keep (1 or 1/2).  A process-wide table keyed by
 * (p, n, N_close, nrays, search, uneven) holds the choice; without an entry
 * the defaults are largest-first and all resident CTAs, with the ray kernel's
 * warps per CTA the choice that lets the most of its warps reside on an SM
 * at that shape (ties to 2, then 4, then 1; 2 when no device can be queried).
 *
 * laGP_autotune times every choice that applies to these arguments on the
 * first min(M, chunk) locations (one kNN pass, then for each choice one
 * untimed and one timed design launch on `stream`), stores the fastest in the
 * table and returns its code in *choice.  It synchronises `stream` and
 * overwrites mean and s2.  Arguments as in laGP_build_and_predict.
 * laGP_tune_get / laGP_tune_set read and install a code for a shape (so a
 * tuned choice can be saved and restored); `uneven` is 1 for calls with
 * n_loc or nclose_loc.  Code: ray_warps | lpt << 4 | (exh_occ - 1) << 5.
 */
int laGP_autotune(const double* design, const double* y, int64_t N, int p, const double* xref,
                  int64_t M, int n0, int n, int N_close, double theta, double g, int search,
                  int nrays, int precision, const int32_t* n_loc, const int32_t* nclose_loc,
                  double* mean, double* s2, void* workspace, size_t workspace_bytes,
                  void* stream, int* choice);
int laGP_tune_get(int p, int n, int N_close, int nrays, int search, int uneven, int* choice);
int laGP_tune_set(int p, int n, int N_close, int nrays, int search, int uneven, int choice);

/*
 * Captured plans.  laGP_plan_create records the complete launch sequence of
 * laGP_build_and_predict for these arguments (same meaning and checks; the
 * launch choices in force at creation are fixed into the plan) into a CUDA
 * graph and instantiates it; nothing runs at creation.  laGP_plan_launch
 * replays it on `stream`: the device reads the buffers behind the pointers
 * given at creation when the replay runs, so refilling xref (or n_loc,
 * nclose_loc) in place and launching again predicts at the new contents.
 * The buffers must stay allocated while the plan exists.  Device status:
 * laGP_status(workspace, ...) as for a direct call.
 */
typedef struct laGP_plan laGP_plan;
int laGP_plan_create(const double* design, const double* y, int64_t N, int p,
                     const double* xref, int64_t M, int n0, int n, int N_close, double theta,
                     double g, int search, int nrays, int precision, const int32_t* n_loc,
                     const int32_t* nclose_loc, double* mean, double* s2, int32_t* selected,
                     double* tie_gap, int32_t* nevals, void* workspace, size_t workspace_bytes,
                     laGP_plan** plan);
int laGP_plan_launch(laGP_plan* plan, void* stream);
int laGP_plan_destroy(laGP_plan* plan);

/*
 * Serving context: a device-resident design and continuous admission of
 * prediction requests (a deployment form of steps 1-4; the paper's own
 * implementation is a batch program).
 *
 * laGP_ctx_create keeps the device pointers design [N][p] and y [N] (which
 * must stay valid) with the fixed method settings (theta, g, n0, N_close,
 * search, nrays, precision), lays out the design part (bounding box, centred
 * FP32 copy: laGP_ctx_design_bytes(N, p)) at the start of `arena` (device,
 * 256-byte aligned, arena_bytes long), prepares it (synchronously) and creates
 * max_inflight (1..64) slots, each with its own stream.
 *
 * laGP_ctx_submit admits one request of M locations: xref [M][p] host, an
 * optional per-location final size n_loc [M] host (each in [n0, n]; NULL:
 * all n), outputs mean [M], s2 [M] and optionally selected [M][n] (host).  The
 * request takes a free slot and a first-fit region of the arena of
 * laGP_ctx_request_bytes(N, p, M, n, N_close, nrays, search, precision,
 * selected != NULL) bytes; it copies the inputs, enqueues the path on the
 * slot's stream, queues the copies of the outputs and returns LAGP_OK with a
 * ticket.  Without a free slot or region it returns LAGP_BUSY and does
 * nothing.  Host buffers should be page-locked: a pageable output makes the
 * call wait for the request to finish.  Results of a location do not depend
 * on the other locations of its request nor on concurrent requests.
 *
 * laGP_ctx_poll sets *done = 1 once the request's outputs are in its host
 * buffers; the first poll that finds it done releases its slot and region and
 * returns its device status (LAGP_OK or LAGP_ERR_DEVICE); a ticket is
 * collected once (later polls return LAGP_ERR_INVALID).  laGP_ctx_wait blocks
 * until the request is done, then polls it.  laGP_ctx_capacity reports the
 * largest free arena region and the number of free slots.  laGP_ctx_destroy
 * waits for every slot and releases the context's CUDA objects (the arena is
 * the caller's).  Calls on one context are serialised by the context.
 */
typedef struct laGP_ctx laGP_ctx;
size_t laGP_ctx_design_bytes(int64_t N, int p);
size_t laGP_ctx_request_bytes(int64_t N, int p, int64_t M, int n, int N_close, int nrays,
                              int search, int precision, int want_selected);
int laGP_ctx_create(const double* design, const double* y, int64_t N, int p, double theta,
                    double g, int n0, int N_close, int search, int nrays, int precision,
                    void* arena, size_t arena_bytes, int max_inflight, laGP_ctx** ctx);
int laGP_ctx_submit(laGP_ctx* ctx, const double* xref, int64_t M, int n, const int32_t* n_loc,
                    double* mean, double* s2, int32_t* selected, int64_t* ticket);
int laGP_ctx_poll(laGP_ctx* ctx, int64_t ticket, int* done);
int laGP_ctx_wait(laGP_ctx* ctx, int64_t ticket);
int laGP_ctx_capacity(laGP_ctx* ctx, size_t* largest_free, int* free_slots);
int laGP_ctx_destroy(laGP_ctx* ctx);

/*
 * Opt-in kernel timing.  laGP_profile(1) clears earlier records and makes
 * every later call record a pair of CUDA events on its stream around each
 * kernel it launches; laGP_profile(0) stops recording.  Not thread-safe
 * against concurrent callers of the other entry points.
 * laGP_profile_read waits for the recorded events and aggregates them by
 * kernel name: names [max_kernels][32] (NUL-terminated), total_ms and
 * launches [max_kernels].  Returns the number of kernels filled in, or a
 * negative error code.
 */
int laGP_profile(int enable);
int laGP_profile_read(int max_kernels, char* names, double* total_ms, int32_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* LAGP_H */
