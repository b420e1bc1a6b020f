// prescale.cu -- pre-scaled inputs (Sec 5.3): a crude global analysis fits a
// separable Gaussian correlation K_ab = exp(-sum_k (x_ak - x_bk)^2 / theta_k)
// (diagonal 1 + g) to a random subset of the design by maximum likelihood,
// and the inputs are divided by sqrt(theta_k) before the local approximation
// runs on them.
//
// Likelihood (the reference-prior form of Eq. gpk, as for the local
// lengthscale, with a vector theta):
//   l = lgamma(n/2) - (n/2) log(2 pi) - (1/2) log|K| - (n/2) log(psi / 2),
//   psi = y^T K^{-1} y,  alpha = K^{-1} y,
//   dl/dtheta_k = -(1/2) tr(K^{-1} K_k) + (n/2) (alpha^T K_k alpha) / psi,
//   K_k,ab = K_ab (x_ak - x_bk)^2 / theta_k^2.
// One evaluation: the gathered subset rows -> K (n x n, binary64) -> K^{-1}
// in place by Gauss-Jordan elimination without pivoting (K is symmetric
// positive definite; the pivots are the successive Schur complements, so
// their logs sum to log|K|), one launch per pivot with the pivot's row,
// column and reciprocal double-buffered so that no launch reads what it
// writes -> alpha ->
// per-row partial sums of the trace and quadratic-form terms (one warp per
// row, fixed order) -> the likelihood and its gradient in eta = log theta on
// one thread, which also advances the maximiser.
//
// Maximiser: BFGS on eta from eta0 = log theta0 (inverse curvature H = I at
// the start), ascent direction d = H grad scaled so that no coordinate moves
// more than 2, trial points projected on [log tmin, log tmax]^p, steps
// t = 1, 1/2, ... (at most 41 trials) until l(eta_t) >= l(eta) + 1e-4 grad .
// (eta_t - eta); the H update is skipped unless s . y > 1e-12 |s| |y| (y the
// change of the negated gradient); the fit ends when a trial moves no
// coordinate by more than 1e-9, when no trial is accepted, or after maxit
// iterations.  The state machine runs on the device; the host only enqueues
// evaluations and reads a done flag after each.
#include <cmath>
#include <cstdint>

#include "../../include/lagp.h"
#include "common.cuh"
#include "lagp_internal.h"

namespace lagp {

#define SEP_MAX_N 1024
#define SEP_MAX_P 16
#define SEP_TOL 1e-9

enum { SEP_INIT = 0, SEP_TRIAL = 1 };

struct SepState {
  double eta[SEP_MAX_P];      // current point (log theta)
  double gr[SEP_MAX_P];       // gradient at eta
  double d[SEP_MAX_P];        // search direction
  double eta_t[SEP_MAX_P];    // point being evaluated
  double H[SEP_MAX_P * SEP_MAX_P];
  double l, t;
  int phase, it, trials, evals, done, status;
};

struct SepWork {
  double* S;       // [n][p] subset rows
  double* ys;      // [n]
  double* A;       // [n][n] K, then K^{-1}
  double* snap;    // [2][2][n] pivot column / row of the current and next step, then
                   // [2] the reciprocal pivot of the current and next step
  double* piv;     // [n]
  double* alpha;   // [n]
  double* part;    // [n][2p] per-row partial sums
  SepState* st;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t sep_layout(int n, int p, char* base, SepWork* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* q = base ? base + off : nullptr;
    off += align256(bytes);
    return q;
  };
  SepWork t;
  t.S = reinterpret_cast<double*>(take(sizeof(double) * n * p));
  t.ys = reinterpret_cast<double*>(take(sizeof(double) * n));
  t.A = reinterpret_cast<double*>(take(sizeof(double) * n * n));
  t.snap = reinterpret_cast<double*>(take(sizeof(double) * (4 * n + 2)));
  t.piv = reinterpret_cast<double*>(take(sizeof(double) * n));
  t.alpha = reinterpret_cast<double*>(take(sizeof(double) * n));
  t.part = reinterpret_cast<double*>(take(sizeof(double) * n * 2 * p));
  t.st = reinterpret_cast<SepState*>(take(sizeof(SepState)));
  if (w) *w = t;
  return off;
}

// subset rows and responses; an index outside [0, N) is reported and skipped
__global__ void sep_gather(const double* X, const double* Y, int64_t N, int p,
                           const int32_t* subset, int n, double theta0, double tmin, double tmax,
                           SepWork w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    SepState* s = w.st;
    const double e0 = log(fmin(fmax(theta0, tmin), tmax));
    for (int k = 0; k < p; ++k) { s->eta[k] = e0; s->eta_t[k] = e0; }
    s->phase = SEP_INIT;
    s->it = 0; s->trials = 0; s->evals = 0; s->done = 0; s->status = 0;
  }
  if (i >= n) return;
  const int32_t r = subset[i];
  if (r < 0 || (int64_t)r >= N) {
    atomicOr(reinterpret_cast<int*>(&w.st->status), 2);
    return;
  }
  for (int k = 0; k < p; ++k) w.S[(int64_t)i * p + k] = X[(int64_t)r * p + k];
  w.ys[i] = Y[r];
}

__device__ __forceinline__ double sep_corr(const double* a, const double* b, int p,
                                           const double* ith) {
  double s = 0.0;
  for (int k = 0; k < p; ++k) {
    const double d = a[k] - b[k];
    s += d * d * ith[k];
  }
  return exp(-s);
}

// K at theta = exp(eta_t), and the first pivot row / column
__global__ void sep_build(int n, int p, double g, SepWork w) {
  if (w.st->done) return;
  double ith[SEP_MAX_P];
  for (int k = 0; k < p; ++k) ith[k] = exp(-w.st->eta_t[k]);
  const int b = blockIdx.x * blockDim.x + threadIdx.x, a = blockIdx.y * blockDim.y + threadIdx.y;
  if (a >= n || b >= n) return;
  const double v = (a == b) ? 1.0 + g : sep_corr(w.S + (int64_t)a * p, w.S + (int64_t)b * p, p, ith);
  w.A[(int64_t)a * n + b] = v;
  if (b == 0) w.snap[a] = v;            // column 0
  if (a == 0) w.snap[n + b] = v;        // row 0
  if (a == 0 && b == 0) w.snap[4 * n] = 1.0 / v;
}

// Gauss-Jordan step k: every element from its own value and the pivot's
// column (cin) and row (rin) as they were before the step, with the pivot's
// reciprocal computed once by the previous step; the new column and row
// k + 1 go to cout / rout, and the thread that forms the next pivot also
// forms its reciprocal, for the next step.
__global__ void gj_step(int n, int k, SepWork w) {
  if (w.st->done) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const double* cin = w.snap + (k & 1) * 2 * n;
  const double* rin = cin + n;
  double* cout = w.snap + ((k + 1) & 1) * 2 * n;
  double* rout = cout + n;
  const double pi = w.snap[4 * n + (k & 1)];
  double v;
  if (i == k && j == k) {
    v = pi;
    w.piv[k] = rin[k];
  } else if (j == k) {
    v = -cin[i] * pi;
  } else if (i == k) {
    v = rin[j] * pi;
  } else {
    v = fma(-cin[i] * pi, rin[j], w.A[(int64_t)i * n + j]);
  }
  w.A[(int64_t)i * n + j] = v;
  if (j == k + 1) cout[i] = v;
  if (i == k + 1) rout[j] = v;
  if (i == k + 1 && j == k + 1) w.snap[4 * n + ((k + 1) & 1)] = 1.0 / v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// alpha = K^{-1} y, one warp per row
__global__ void sep_alpha(int n, SepWork w) {
  if (w.st->done) return;
  const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= n) return;
  double s = 0.0;
  for (int b = lane; b < n; b += 32) s += w.A[(int64_t)a * n + b] * w.ys[b];
  s = warp_sum_d(s);
  if (lane == 0) w.alpha[a] = s;
}

// row a's sums: T_k = sum_b Kinv_ab K_ab d_abk and U_k = sum_b K_ab d_abk alpha_b
__global__ void sep_rows(int n, int p, SepWork w) {
  if (w.st->done) return;
  const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= n) return;
  double ith[SEP_MAX_P], T[SEP_MAX_P], U[SEP_MAX_P];
  for (int k = 0; k < p; ++k) { ith[k] = exp(-w.st->eta_t[k]); T[k] = 0.0; U[k] = 0.0; }
  const double* xa = w.S + (int64_t)a * p;
  for (int b = lane; b < n; b += 32) {
    if (b == a) continue;
    const double* xb = w.S + (int64_t)b * p;
    const double kab = sep_corr(xa, xb, p, ith);
    const double ki = w.A[(int64_t)a * n + b] * kab, ka = kab * w.alpha[b];
    for (int k = 0; k < p; ++k) {
      const double d = xa[k] - xb[k], dd = d * d;
      T[k] += ki * dd;
      U[k] += ka * dd;
    }
  }
  for (int k = 0; k < p; ++k) {
    const double tk = warp_sum_d(T[k]), uk = warp_sum_d(U[k]);
    if (lane == 0) {
      w.part[(int64_t)a * 2 * p + k] = tk;
      w.part[(int64_t)a * 2 * p + p + k] = uk;
    }
  }
}

__device__ void sep_propose(SepState* s, int p, double lo, double hi, int maxit, bool new_iter) {
  for (;;) {
    if (new_iter) {
      if (s->it >= maxit) { s->done = 1; return; }
      ++s->it;
      double m = 0.0;
      for (int k = 0; k < p; ++k) {
        double v = 0.0;
        for (int c = 0; c < p; ++c) v += s->H[k * SEP_MAX_P + c] * s->gr[c];
        s->d[k] = v;
        m = fmax(m, fabs(v));
      }
      if (m > 2.0)
        for (int k = 0; k < p; ++k) s->d[k] *= 2.0 / m;
      s->t = 1.0;
      s->trials = 0;
    }
    double ms = 0.0;
    for (int k = 0; k < p; ++k) {
      const double e = fmin(fmax(s->eta[k] + s->t * s->d[k], lo), hi);
      s->eta_t[k] = e;
      ms = fmax(ms, fabs(e - s->eta[k]));
    }
    ++s->trials;
    if (!(ms > SEP_TOL)) { s->done = 1; return; }     // the trial does not move: stalled
    s->phase = SEP_TRIAL;
    return;
  }
}

// Likelihood and gradient at eta_t from the partial sums; then one move of
// the BFGS state machine (one thread).
__global__ void sep_finish(int n, int p, double lo, double hi, int maxit, SepWork w) {
  SepState* s = w.st;
  if (s->done) return;
  __shared__ double red[2];
  const int lane = threadIdx.x;
  double ps = 0.0, ld = 0.0;
  for (int a = lane; a < n; a += 32) {
    ps += w.ys[a] * w.alpha[a];
    ld += log(w.piv[a]);
  }
  ps = warp_sum_d(ps);
  ld = warp_sum_d(ld);
  if (lane == 0) { red[0] = ps; red[1] = ld; }
  __syncwarp();
  if (lane != 0) return;
  const double psi = red[0], logdet = red[1], hn = 0.5 * n;
  double l = lgamma(hn) - hn * log(2.0 * M_PI) - 0.5 * logdet - hn * log(psi / 2.0);
  if (!(psi > 0.0)) l = NAN;
  double gt[SEP_MAX_P];
  for (int k = 0; k < p; ++k) {
    double tr = 0.0, q = 0.0;
    for (int a = 0; a < n; ++a) {
      tr += w.part[(int64_t)a * 2 * p + k];
      q += w.alpha[a] * w.part[(int64_t)a * 2 * p + p + k];
    }
    const double th = exp(s->eta_t[k]);
    // dl/dtheta_k times theta_k (the gradient in eta)
    gt[k] = (-0.5 * tr + hn * q / psi) / th;
  }
  ++s->evals;
  if (s->phase == SEP_INIT) {
    if (!(l == l)) { s->done = 1; s->status |= 1; return; }
    s->l = l;
    for (int k = 0; k < p; ++k) s->gr[k] = gt[k];
    for (int k = 0; k < SEP_MAX_P * SEP_MAX_P; ++k) s->H[k] = 0.0;
    for (int k = 0; k < p; ++k) s->H[k * SEP_MAX_P + k] = 1.0;
    sep_propose(s, p, lo, hi, maxit, true);
    return;
  }
  double gs = 0.0;
  for (int k = 0; k < p; ++k) gs += s->gr[k] * (s->eta_t[k] - s->eta[k]);
  if (l == l && l >= s->l + 1e-4 * gs) {
    double sv[SEP_MAX_P], yv[SEP_MAX_P], sy = 0.0, ns = 0.0, ny = 0.0;
    for (int k = 0; k < p; ++k) {
      sv[k] = s->eta_t[k] - s->eta[k];
      yv[k] = s->gr[k] - gt[k];
      sy += sv[k] * yv[k];
      ns += sv[k] * sv[k];
      ny += yv[k] * yv[k];
    }
    if (sy > 1e-12 * sqrt(ns) * sqrt(ny)) {
      // H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T
      const double rho = 1.0 / sy;
      double Hy[SEP_MAX_P], yH[SEP_MAX_P], yHy = 0.0;
      for (int r = 0; r < p; ++r) {
        double a = 0.0, b = 0.0;
        for (int c = 0; c < p; ++c) {
          a += s->H[r * SEP_MAX_P + c] * yv[c];
          b += yv[c] * s->H[c * SEP_MAX_P + r];
        }
        Hy[r] = a;
        yH[r] = b;
      }
      for (int c = 0; c < p; ++c) yHy += yv[c] * Hy[c];
      for (int r = 0; r < p; ++r)
        for (int c = 0; c < p; ++c)
          s->H[r * SEP_MAX_P + c] += -rho * (sv[r] * yH[c] + Hy[r] * sv[c]) +
                                     (rho * rho * yHy + rho) * sv[r] * sv[c];
    }
    for (int k = 0; k < p; ++k) { s->eta[k] = s->eta_t[k]; s->gr[k] = gt[k]; }
    s->l = l;
    sep_propose(s, p, lo, hi, maxit, true);
  } else {
    if (s->trials >= 41) { s->done = 1; return; }   // no accepted trial
    s->t *= 0.5;
    sep_propose(s, p, lo, hi, maxit, false);
  }
}

__global__ void sep_out(int p, SepWork w, double* theta_out, int32_t* info) {
  const int k = threadIdx.x;
  if (k < p) theta_out[k] = exp(w.st->eta[k]);
  if (k == 0 && info) {
    info[0] = w.st->it;
    info[1] = w.st->evals;
    info[2] = w.st->status;
  }
}

__global__ void prescale_kernel(const double* X, int64_t rows, int p, const double* theta,
                                double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * p) return;
  out[e] = X[e] / sqrt(theta[e % p]);
}

}  // namespace lagp

using namespace lagp;

extern "C" size_t laGP_sep_mle_workspace_bytes(int n_sub, int p) {
  if (n_sub < 2 || n_sub > SEP_MAX_N || p < 1 || p > SEP_MAX_P) return 0;
  return sep_layout(n_sub, p, nullptr, nullptr);
}

extern "C" int laGP_sep_mle(const double* design, const double* y, int64_t N, int p,
                            const int32_t* subset, int n_sub, double g, double theta0,
                            double tmin, double tmax, int maxit, double* theta_out,
                            int32_t* info, void* workspace, size_t workspace_bytes,
                            void* stream) {
  if (!design || !y || !subset || !theta_out || !workspace) return LAGP_ERR_INVALID;
  if (n_sub < 2 || n_sub > SEP_MAX_N || p < 1 || p > SEP_MAX_P || N < n_sub) return LAGP_ERR_INVALID;
  if (!(g >= 0.0) || !(tmin > 0.0) || !(tmax >= tmin) || !(theta0 > 0.0) || maxit < 1)
    return LAGP_ERR_INVALID;
  if (workspace_bytes < sep_layout(n_sub, p, nullptr, nullptr)) return LAGP_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SepWork w;
  sep_layout(n_sub, p, static_cast<char*>(workspace), &w);
  const int n = n_sub;
  const double lo = log(tmin), hi = log(tmax);
  sep_gather<<<(n + 127) / 128, 128, 0, s>>>(design, y, N, p, subset, n, theta0, tmin, tmax, w);
  if (cudaGetLastError() != cudaSuccess) return LAGP_ERR_CUDA;
  const dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  const int rows_grid = (n + 7) / 8;
  // at most maxit iterations of at most 41 trials each, plus the first evaluation
  const int64_t max_evals = (int64_t)maxit * 41 + 1;
  for (int64_t e = 0; e < max_evals; ++e) {
    sep_build<<<grd, blk, 0, s>>>(n, p, g, w);
    for (int k = 0; k < n; ++k) gj_step<<<grd, blk, 0, s>>>(n, k, w);
    sep_alpha<<<rows_grid, 256, 0, s>>>(n, w);
    sep_rows<<<rows_grid, 256, 0, s>>>(n, p, w);
    sep_finish<<<1, 32, 0, s>>>(n, p, lo, hi, maxit, w);
    if (cudaGetLastError() != cudaSuccess) return LAGP_ERR_CUDA;
    int done = 0;
    if (cudaMemcpyAsync(&done, &w.st->done, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return LAGP_ERR_CUDA;
    if (done) break;
  }
  sep_out<<<1, 32, 0, s>>>(p, w, theta_out, info);
  if (cudaGetLastError() != cudaSuccess) return LAGP_ERR_CUDA;
  int st = 0;
  if (cudaMemcpyAsync(&st, &w.st->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LAGP_ERR_CUDA;
  return st ? LAGP_ERR_DEVICE : LAGP_OK;
}

extern "C" int laGP_prescale(const double* X, int64_t rows, int p, const double* theta,
                             double* X_out, void* stream) {
  if (rows < 0 || p < 1 || p > LAGP_MAX_P) return LAGP_ERR_INVALID;
  if (rows == 0) return LAGP_OK;
  if (!X || !theta || !X_out) return LAGP_ERR_INVALID;
  const int64_t e = rows * p;
  prescale_kernel<<<(unsigned)((e + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      X, rows, p, theta, X_out);
  return cudaGetLastError() == cudaSuccess ? LAGP_OK : LAGP_ERR_CUDA;
}
