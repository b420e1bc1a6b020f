// mle.cu -- local inference for the lengthscale on a given local design
// (Gramacy & Haaland, Sec 5: local designs are coupled with Newton-like
// maximisation of the local posterior of theta; Sec 2.1, Eq. gpk), then the
// predictive equations (Eq. predgp, preds2) at the estimate.  Binary64, one CTA
// of 128 threads per predictive location, the local matrices in shared memory
// (n <= 64).
//
// Objective (readings M1, M2): the log marginal likelihood of Eq. gpk with the
// reference prior on tau^2 and a flat prior on theta over [tmin, tmax],
//   l(theta) = log Gamma(n/2) - (n/2) log(2 pi) - (1/2) log|K| - (n/2) log(psi/2),
//   psi = y^T K^{-1} y,  K_ab = exp(-d_ab / theta) off the diagonal, 1 + g on it,
// with exact derivatives in theta (K' = K d / theta^2 off the diagonal,
// K'' = K' (d / theta^2 - 2 / theta)):
//   l'  = -(1/2) tr(K^{-1} K') - (n/2) psi' / psi,
//   l'' = -(1/2) [tr(K^{-1} K'') - tr(K^{-1} K' K^{-1} K')] - (n/2) [psi''/psi - (psi'/psi)^2],
//   psi' = -alpha^T K' alpha, psi'' = 2 (K' alpha)^T K^{-1} (K' alpha) - alpha^T K'' alpha,
//   alpha = K^{-1} y.
// Each evaluation factors K = C C^T (Cholesky, by columns), forms C^{-1} and
// K^{-1} = C^{-T} C^{-1}, then K^{-1} K'.  The constant log Gamma(n/2) and
// -(n/2) log(2 pi) do not move the maximiser and are left out.
//
// Maximiser (reading M3): Newton's method from theta0, safeguarded by a bracket
// [a, b] kept from the sign of l'; a step outside the bracket, or taken where
// l'' >= 0, is replaced by the bracket's midpoint; it stops when a step or the
// bracket falls below tol * theta, or after maxit iterations.  Every thread
// evaluates the scalar recurrence on the same block sums, so control flow is
// uniform.  No loop waits on another thread or block.
#include <cstdint>

#include "../../include/lagp.h"
#include "common.cuh"
#include "lagp_internal.h"

namespace lagp {

#define MLE_THREADS 128
#define MLE_WARPS (MLE_THREADS / 32)
#define MLE_NMAX 64
#define MLE_PMAX 16

struct MleParams {
  const double* X;
  const double* Y;
  int64_t N;
  int p;
  const double* xref;
  int64_t M;
  const int32_t* sel;   // [M][n] design indices of each local design
  int n;
  double theta0, g, tmin, tmax, tol;
  const double* theta0_loc;   // per-location start [M] or null (theta0)
  int maxit;
  double* theta_out;
  double* mean;
  double* s2;
  int32_t* iters;       // or null
  unsigned* status;
};

// Sum over the block; every thread returns the same value (the four warp
// totals are added in warp order by every thread).
__device__ __forceinline__ double mle_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();   // earlier readers of red are done
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < MLE_WARPS; ++w) t += red[w];
  return t;
}

struct MleEval {
  double ll, d1, d2, psi;
  bool ok;
};

// Log-likelihood (without its theta-free constant) and derivatives at theta.
// Leaves C (Cholesky factor, lower triangle), Ki = K^{-1} and al = K^{-1} y.
__device__ MleEval mle_eval(int n, double theta, double g, const double* D, const double* y,
                            double* Cm, double* Ki, double* K1, double* A, double* al,
                            double* u, double* red, int* flag) {
  const int tid = threadIdx.x;
  const int nn = n * n;
  const double th2 = theta * theta;
  MleEval r;
  r.ok = false;
  r.ll = r.d1 = r.d2 = r.psi = 0.0;
  for (int e = tid; e < nn; e += MLE_THREADS) {
    const int a = e / n, b = e - a * n;
    const double d = D[e];
    const double k = exp_neg_fma(-(d / theta));
    Cm[e] = (a == b) ? 1.0 + g : k;
    K1[e] = (a == b) ? 0.0 : k * d / th2;
  }
  if (tid == 0) *flag = 0;
  __syncthreads();
  // Cholesky by columns: warp 0 forms the pivot, all threads the column below it
  for (int j = 0; j < n; ++j) {
    if (tid < 32) {
      double s = 0.0;
      for (int k = tid; k < j; k += 32) s = fma(Cm[j * n + k], Cm[j * n + k], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (tid == 0) {
        const double piv = Cm[j * n + j] - s;
        if (!(piv > 0.0)) *flag = 1;
        Cm[j * n + j] = piv > 0.0 ? sqrt(piv) : 1.0;
      }
    }
    __syncthreads();
    const double cjj = Cm[j * n + j];
    for (int i = j + 1 + tid; i < n; i += MLE_THREADS) {
      double t = Cm[i * n + j];
      for (int k = 0; k < j; ++k) t = fma(-Cm[i * n + k], Cm[j * n + k], t);
      Cm[i * n + j] = t / cjj;
    }
    __syncthreads();
  }
  if (*flag) return r;
  // C^{-1} into A by columns (thread c: column c), then K^{-1} = C^{-T} C^{-1}
  for (int c = tid; c < n; c += MLE_THREADS) {
    for (int i = 0; i < c; ++i) A[i * n + c] = 0.0;
    for (int i = c; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) t = fma(-Cm[i * n + k], A[k * n + c], t);
      A[i * n + c] = t / Cm[i * n + i];
    }
  }
  __syncthreads();
  for (int e = tid; e < nn; e += MLE_THREADS) {
    const int i = e / n, j = e - i * n;
    double t = 0.0;
    for (int k = (i > j ? i : j); k < n; ++k) t = fma(A[k * n + i], A[k * n + j], t);
    Ki[e] = t;
  }
  __syncthreads();
  // log|K|, alpha = K^{-1} y, psi
  double ld = 0.0;
  for (int j = tid; j < n; j += MLE_THREADS) ld += log(Cm[j * n + j]);
  for (int i = tid; i < n; i += MLE_THREADS) {
    double t = 0.0;
    for (int k = 0; k < n; ++k) t = fma(Ki[i * n + k], y[k], t);
    al[i] = t;
  }
  const double logdet = 2.0 * mle_block_sum(ld, red);   // its barriers publish al
  double ps = 0.0;
  for (int i = tid; i < n; i += MLE_THREADS) ps = fma(y[i], al[i], ps);
  const double psi = mle_block_sum(ps, red);
  // A = K^{-1} K' (overwrites C^{-1}); u = K' alpha
  for (int e = tid; e < nn; e += MLE_THREADS) {
    const int i = e / n, j = e - i * n;
    double t = 0.0;
    for (int k = 0; k < n; ++k) t = fma(Ki[i * n + k], K1[k * n + j], t);
    A[e] = t;
  }
  for (int i = tid; i < n; i += MLE_THREADS) {
    double t = 0.0;
    for (int k = 0; k < n; ++k) t = fma(K1[i * n + k], al[k], t);
    u[i] = t;
  }
  __syncthreads();
  // traces and quadratic forms; K''_ab = K'_ab (d_ab / theta^2 - 2 / theta)
  double tr1 = 0.0, tr2 = 0.0, tr11 = 0.0, ak1a = 0.0, ak2a = 0.0, uku = 0.0;
  for (int e = tid; e < nn; e += MLE_THREADS) {
    const int i = e / n, k = e - i * n;
    const double k2 = K1[e] * (D[e] / th2 - 2.0 / theta);
    if (i == k) tr1 += A[e];
    tr2 = fma(Ki[k * n + i], k2, tr2);
    tr11 = fma(A[e], A[k * n + i], tr11);
    ak2a = fma(al[i] * k2, al[k], ak2a);
    uku = fma(u[i] * Ki[e], u[k], uku);
  }
  for (int i = tid; i < n; i += MLE_THREADS) ak1a = fma(al[i], u[i], ak1a);
  tr1 = mle_block_sum(tr1, red);
  tr2 = mle_block_sum(tr2, red);
  tr11 = mle_block_sum(tr11, red);
  ak1a = mle_block_sum(ak1a, red);
  ak2a = mle_block_sum(ak2a, red);
  uku = mle_block_sum(uku, red);
  const double hn = 0.5 * (double)n;
  const double ps1 = -ak1a, ps2 = 2.0 * uku - ak2a;
  r.ll = -0.5 * logdet - hn * log(psi / 2.0);
  r.d1 = -0.5 * tr1 - hn * ps1 / psi;
  r.d2 = -0.5 * (tr2 - tr11) - hn * (ps2 / psi - (ps1 / psi) * (ps1 / psi));
  r.psi = psi;
  r.ok = psi > 0.0;
  return r;
}

__global__ void __launch_bounds__(MLE_THREADS) mle_kernel(MleParams P) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double red[MLE_WARPS];
  __shared__ int flag;
  const int n = P.n, p = P.p, tid = threadIdx.x;
  const int64_t loc = blockIdx.x;
  double* S = sm;              // [n][p]
  double* y = S + n * p;       // [n]
  double* D = y + n;           // [n][n] squared distances
  double* Cm = D + n * n;      // [n][n] Cholesky factor
  double* Ki = Cm + n * n;     // [n][n] K^{-1}
  double* K1 = Ki + n * n;     // [n][n] dK/dtheta
  double* A = K1 + n * n;      // [n][n] C^{-1}, then K^{-1} K'
  double* al = A + n * n;      // [n] K^{-1} y
  double* u = al + n;          // [n] K' alpha, then k(x)
  const int32_t* sl = P.sel + loc * n;
  if (tid == 0) flag = 0;
  __syncthreads();
  for (int e = tid; e < n * p; e += MLE_THREADS) {
    const int i = e / p, k = e - i * p;
    const int32_t gi = sl[i];
    if (gi < 0 || gi >= P.N) { flag = 1; S[e] = 0.0; continue; }
    S[e] = P.X[(int64_t)gi * p + k];
  }
  for (int i = tid; i < n; i += MLE_THREADS) {
    const int32_t gi = sl[i];
    y[i] = (gi >= 0 && gi < P.N) ? P.Y[gi] : 0.0;
  }
  __syncthreads();
  const bool bad_index = flag != 0;
  __syncthreads();
  for (int e = tid; e < n * n; e += MLE_THREADS) {
    const int a = e / n, b = e - a * n;
    D[e] = sqdist64(S + a * p, S + b * p, p);
  }
  __syncthreads();

  double lo = P.tmin, hi = P.tmax;
  const double t0 = P.theta0_loc ? P.theta0_loc[loc] : P.theta0;
  double t = t0 < lo ? lo : (t0 > hi ? hi : t0);
  int it = 0;
  bool ok = !bad_index;
  while (ok && it < P.maxit) {
    ++it;
    const MleEval e = mle_eval(n, t, P.g, D, y, Cm, Ki, K1, A, al, u, red, &flag);
    __syncthreads();
    if (!e.ok || !(e.ll == e.ll) || !(e.d1 == e.d1)) break;
    if (e.d1 > 0.0) lo = t; else hi = t;
    if (hi - lo <= P.tol * t) break;
    double tn = t - e.d1 / e.d2;
    if (!(e.d2 < 0.0) || !(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    const double step = tn - t;
    t = tn;
    if (fabs(step) <= P.tol * t) break;
  }
  // predictive equations at the estimate
  double mu = 0.0, s2 = 0.0;
  if (ok) {
    const MleEval e = mle_eval(n, t, P.g, D, y, Cm, Ki, K1, A, al, u, red, &flag);
    __syncthreads();
    ok = e.ok;
    if (ok) {
      const double* x = P.xref + loc * p;
      for (int i = tid; i < n; i += MLE_THREADS) {
        const double d = sqdist64(S + i * p, x, p);
        u[i] = exp_neg_fma(-(d / t));
      }
      __syncthreads();
      double m = 0.0, q = 0.0;
      for (int i = tid; i < n; i += MLE_THREADS) {
        m = fma(u[i], al[i], m);
        double ki = 0.0;
        for (int k = 0; k < n; ++k) ki = fma(Ki[i * n + k], u[k], ki);
        q = fma(u[i], ki, q);
      }
      mu = mle_block_sum(m, red);
      q = mle_block_sum(q, red);
      s2 = e.psi * ((1.0 + P.g) - q) / (double)n;
    }
  }
  if (tid == 0) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    P.theta_out[loc] = ok ? t : nan;
    P.mean[loc] = ok ? mu : nan;
    P.s2[loc] = ok ? s2 : nan;
    if (P.iters) P.iters[loc] = it;
    if (!ok) atomicOr(P.status, LAGP_DEV_BAD_UPDATE);
  }
}

static size_t mle_smem(int n, int p) {
  return sizeof(double) * ((size_t)n * p + 3 * (size_t)n + 5 * (size_t)n * n);
}

}  // namespace lagp

using namespace lagp;

namespace lagp {

cudaError_t launch_mle(const double* X, const double* Y, int64_t N, int p, const double* xref,
                       int64_t M, const int32_t* sel, int n, double theta0,
                       const double* theta0_loc, double g, double tmin, double tmax,
                       double* theta_out, double* mean, double* s2, int32_t* iters,
                       unsigned* status, cudaStream_t s) {
  MleParams P;
  P.X = X; P.Y = Y; P.N = N; P.p = p; P.xref = xref; P.M = M; P.sel = sel; P.n = n;
  P.theta0 = theta0; P.theta0_loc = theta0_loc; P.g = g; P.tmin = tmin; P.tmax = tmax;
  P.tol = 1e-10; P.maxit = 200;
  P.theta_out = theta_out; P.mean = mean; P.s2 = s2; P.iters = iters; P.status = status;
  const size_t sm = mle_smem(n, p);
  cudaError_t e = cudaFuncSetAttribute(mle_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  prof_begin("mle_theta", s);
  mle_kernel<<<(unsigned)M, MLE_THREADS, sm, s>>>(P);
  prof_end(s);
  return cudaGetLastError();
}

bool mle_shape_ok(int p, int n) { return p >= 1 && p <= MLE_PMAX && n >= 1 && n <= MLE_NMAX; }

}  // namespace lagp

extern "C" int laGP_mle_predict(const double* design, const double* y, int64_t N, int p,
                                const double* xref, int64_t M, const int32_t* sel, int n,
                                double theta0, double g, double tmin, double tmax,
                                double* theta_out, double* mean, double* s2, int32_t* iters,
                                unsigned* status, void* stream) {
  if (N < 1 || !mle_shape_ok(p, n) || M < 0 || n > N) return LAGP_ERR_INVALID;
  if (!(g >= 0.0) || !(tmin > 0.0) || !(tmax > tmin) || !(theta0 > 0.0) ||
      !(tmax < 1e300))
    return LAGP_ERR_INVALID;
  if (!status) return LAGP_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(status, 0, sizeof(unsigned), s) != cudaSuccess) return LAGP_ERR_CUDA;
  if (M == 0) return LAGP_OK;
  if (!design || !y || !xref || !sel || !theta_out || !mean || !s2) return LAGP_ERR_INVALID;
  if (M > 0x7fffffffll) return LAGP_ERR_INVALID;
  return launch_mle(design, y, N, p, xref, M, sel, n, theta0, nullptr, g, tmin, tmax, theta_out,
                    mean, s2, iters, status, s) == cudaSuccess
             ? LAGP_OK
             : LAGP_ERR_CUDA;
}
